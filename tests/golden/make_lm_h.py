"""Writes lm_h_w12_x0p25.txt: the oracle's least-misfit correcting function h on the
Ng + 1 = 33 nodes of Appendix A for W = 12 at the paper's x0 = 0.25 (Levenberg-Marquardt
from Appendix A's initial guesses, W' = 3 .. 12 in turn). Calls only oracle/; the file
saves the CPU tests about a minute of optimisation. Run: python tests/golden/make_lm_h.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import design as D  # noqa: E402

W, X0P = 12, 0.25

if __name__ == "__main__":
    h = D.least_misfit_h(W, X0P)
    path = os.path.join(HERE, "lm_h_w12_x0p25.txt")
    with open(path, "w") as f:
        f.write(f"# least-misfit h on the {h.size} nodes x_i = i x0 / {h.size - 1} of Appendix A, W = {W}, "
                f"x0 = {X0P}; written by tests/golden/make_lm_h.py from oracle.design.least_misfit_h\n")
        for v in h:
            f.write(f"{v:.17e}\n")
    print(path)

"""Validation experiments of the paper run through the library (float64 kernels) on seeded
Earth-rotation tracks, against brute-force DFT images from the oracle (needs a GPU).

* alias suppression (Section 4.2): a unit point source outside the FFT field aliases into
  the kept field; its normalised alias brightness is the largest |FFT - DFT| over the kept
  pixels divided by the source's peak brightness sum_k w_k = nvis;
* image misfit against x0 (Section 2.2, the W = 8 sweep of the kept field): the RMS of
  FFT - DFT over the kept field relative to the RMS of the DFT image, for random
  visibilities, next to the design's integrated misfit E (Eq. 16);
* least-misfit against the prolate spheroidal function (alpha = 1) at W = 6 .. 12.

``python tests/validation.py`` writes the table of results (markdown) to stdout; the GPU
tests in tests/test_gpu_validation.py check the same numbers against the paper's text.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import imaging as I  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402

N = 512          # grid
MS = 4000        # table oversampling (cubic lookup: interpolation error far below the misfits)
SUB = 32         # DFT reference on SUB x SUB kept pixels (every (n_img / SUB)-th row and column)


def tracks(n_ant=24, n_times=192, seed=3):
    """(uv in wavelengths, pixel scale): 276 baselines x 192 samples = 52,992 positions."""
    uv = S.array_tracks(n_ant=n_ant, n_times=n_times, seed=seed)
    return uv, S.pixel_scale_for(uv)


def spheroidal_table(W, Ms):
    """Spheroidal function (alpha = 1: scipy pro_ang1 of order m = 1 with c = pi W / 2, times
    (1 - eta^2)^(1/2)) on the table layout: row i at s = i / Ms, entry j at d = j - W/2 + s."""
    from scipy.special import pro_ang1
    s = np.arange(Ms + 1) / Ms
    d = np.arange(W)[None, :] - W / 2 + s[:, None]
    eta = 2 * d / W
    inside = np.abs(eta) < 1
    e = np.where(inside, eta, 0.0)
    return np.where(inside, pro_ang1(1, 1, np.pi * W / 2, e)[0] * np.sqrt(1 - e ** 2), 0.0)


def _sub_pixels(n_img):
    step = max(1, n_img // SUB)
    return np.arange(step // 2, n_img, step)


class Imager:
    """Float64 dirty images of one uv set through the library, with DFT references."""

    def __init__(self, uv, dl, n_img):
        import torch
        self.torch = torch
        self.uv, self.dl, self.n_img = uv, dl, n_img
        self.uv_d = torch.from_numpy(uv).cuda()
        self.N = N
        uc = I.cells_from_wavelengths(uv, N, dl)
        self.u, self.v = uc[:, 0], uc[:, 1]
        self.px = _sub_pixels(n_img)
        self.x = I.pixel_coords(n_img, N)[self.px]

    def fft_image(self, table, vis):
        from paper_1906_07102_gb300 import lmg
        p = lmg.Plan(table, self.n_img, self.dl, self.uv.shape[0], "c128")
        p.bin(self.uv_d)
        img = p.dirty_image(self.torch.from_numpy(np.ascontiguousarray(vis)).cuda()).cpu().numpy()
        return img[np.ix_(self.px, self.px)]

    def dft_image(self, vis):
        return I.dft_dirty_image(self.u, self.v, vis, None, self.x, self.x)


def alias_brightness(tables, offsets, W_of, y_src=0.1):
    """Normalised alias brightness for sources at x = a + 1 (beyond the FFT field; the alias
    lands at x = a in the kept field) and y = y_src, for every a in `offsets` and table.
    Returns {name: [brightness per offset]}."""
    uv, dl = tracks()
    im = Imager(uv, dl, N // 2)
    out = {name: [] for name in tables}
    for a in offsets:
        l, m = (a + 1.0) * N * dl, y_src * N * dl
        vis = S.visibilities(uv, np.array([l]), np.array([m]), np.array([1.0]))
        ref = im.dft_image(vis)
        for name, tab in tables.items():
            out[name].append(float(np.abs(im.fft_image(tab, vis) - ref).max() / uv.shape[0]))
    return out


def misfit(tables, seed=11):
    """Relative RMS of FFT - DFT over the kept field for random visibilities, per table
    (all tables share the table's kept fraction x0 of their first entry's plan)."""
    uv, dl = tracks()
    vis = S.complex_normal(uv.shape[0], seed)
    out = {}
    for name, (tab, n_img) in tables.items():
        im = Imager(uv, dl, n_img)
        ref = im.dft_image(vis)
        err = im.fft_image(tab, vis) - ref
        out[name] = float(np.sqrt(np.mean(np.abs(err) ** 2) / np.mean(np.abs(ref) ** 2)))
    return out


def run_all():
    from paper_1906_07102_gb300 import lmg
    res = {}
    # least-misfit against spheroidal at equal W, x0 = 0.25 (kept fraction 0.5)
    Ws = (6, 7, 8, 10, 12)
    tabs = {}
    for W in Ws:
        tabs[f"LM W={W}"] = (lmg.Table(W, 0.5, MS, "cubic"), N // 2)
        tabs[f"PSWF W={W}"] = (lmg.Table(W, 0.5, MS, "cubic", values=spheroidal_table(W, MS)), N // 2)
    res["misfit_vs_W"] = misfit(tabs)
    # alias suppression: alias positions across the kept field (|x| <= 0.25)
    offsets = (-0.24, -0.2, -0.15, -0.1, -0.05, 0.0, 0.05, 0.1, 0.15, 0.2, 0.24)
    atabs = {name: t for name, (t, _) in tabs.items() if name.split("=")[1] in ("6", "7", "8", "10")}
    res["alias_offsets"] = list(offsets)
    res["alias"] = alias_brightness(atabs, offsets, None)
    # image misfit against the kept half-width x0 at W = 8
    x0s = (0.125, 0.1875, 0.25, 0.3125, 0.375)
    xt = {}
    E = {}
    for x0p in x0s:
        t = lmg.Table(8, 2 * x0p, MS, "cubic")
        xt[f"x0={x0p}"] = (t, int(round(N * 2 * x0p)))
        E[f"x0={x0p}"] = t.export()[2]
    res["misfit_vs_x0"] = misfit(xt)
    res["E_vs_x0"] = E
    return res


def markdown(res):
    lines = ["# Validation through the library: alias suppression and image misfit", "",
             "Float64 kernels, cubic tables at M_s = 4000, 512^2 grid, 24-antenna tracks "
             "(276 baselines x 192 samples, seed 3), DFT references on 32 x 32 kept pixels. "
             "Command: `python tests/validation.py` (GB300).", "",
             "## Image misfit: least-misfit (LM) vs spheroidal (PSWF, alpha = 1), x0 = 0.25", "",
             "| W | LM rel. RMS misfit | PSWF rel. RMS misfit | PSWF / LM |", "|---:|---:|---:|---:|"]
    mv = res["misfit_vs_W"]
    for W in (6, 7, 8, 10, 12):
        lm, ps = mv[f"LM W={W}"], mv[f"PSWF W={W}"]
        lines.append(f"| {W} | {lm:.3e} | {ps:.3e} | {ps / lm:.0f} |")
    lines += ["", "## Normalised alias brightness (source beyond the FFT field, alias at x in the kept field)", ""]
    names = list(res["alias"])
    lines.append("| alias x | " + " | ".join(names) + " |")
    lines.append("|---:|" + "---:|" * len(names))
    for i, a in enumerate(res["alias_offsets"]):
        lines.append(f"| {a:+.2f} | " + " | ".join(f"{res['alias'][n][i]:.2e}" for n in names) + " |")
    lines += ["", "## Image misfit against the kept half-width x0, W = 8", "",
              "| x0 | rel. RMS misfit | design E (Eq. 16) | sqrt(E) |", "|---:|---:|---:|---:|"]
    for k, v in res["misfit_vs_x0"].items():
        e = res["E_vs_x0"][k]
        lines.append(f"| {k.split('=')[1]} | {v:.3e} | {e:.3e} | {np.sqrt(e):.3e} |")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    from paper_1906_07102_gb300 import lmg  # noqa: F401
    import torch
    torch.cuda.set_device(0)
    print(markdown(run_all()))

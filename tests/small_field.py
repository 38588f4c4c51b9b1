"""Small-field limit of the least-misfit design (test-side reference, any W).

For one table coordinate s the support offsets are d_j = j - W/2 + s (Eqs. 6, 9) and the
footprint sum of Eqs. 7-11 expands in moments,

    a(x; s) = sum_j C_j exp(2 pi i d_j x) = sum_k (2 pi i x)^k / k! * m_k(s),
    m_k(s)  = sum_j C_j(s) d_j^k.

On a small field (|x| <= x0 << 1) the misfit 1 - h(x) a(x; s) vanishes through order
x^(W-1) for every s exactly when the W moments m_0 .. m_(W-1) equal the Taylor
coefficients of 1/h. h is real and even with h(0) = 1, so 1/h(x) = sum_{k even}
t_k (2 pi i x)^k / k! with t_0 = 1 and real t_2, t_4, ... that are the same for all s;
the odd moments vanish. These W conditions fix C(s) (a Vandermonde solve in the d_j).
The next moment is then m_W(s) = -sum_{k<W} t_k w_k(s), where w(d) = prod_j (d - d_j) =
d^W + sum_{k<W} w_k d^k (d^W - w(d) is the polynomial of degree < W that equals d^W on
the nodes). The leading misfit is (2 pi x)^W m_W(s) / W! -- imaginary for odd W; real for
even W, where h's own x^W coefficient t_W subtracts a common constant. The least-squares
solve of each s trades the lower moments against it and leaves its part orthogonal to
the lower powers on [-x0, x0], the monic Legendre polynomial P~_W(x / x0). So

    E = (2 pi x0)^(2W) / (W!)^2 * (1/2) ||P~_W||^2 * min < (m_W(s) - t_W [even W])^2 >_s
        + O(x0^(2W+2)),

the minimum taken over the free t_2, t_4, ... (and t_W for even W), a small linear
least-squares problem over s in [0, 1); ||P~_n||^2 = 2^(2n+1) (n!)^4 / ((2n+1) ((2n)!)^2).
At the optimum C(s) is the Vandermonde solution for those t and h(x) = 1 / F(x) with
F(x) = sum_{k even <= W} t_k (-1)^(k/2) (2 pi x)^k / k!, each up to O(x0^2) relative.

Only numpy here; nothing calls the oracle or the library.
"""
import math

import numpy as np


def _node_poly(d):
    """Coefficients w_0 .. w_W (ascending) of prod_j (d - d_j) for each row of d."""
    return np.array([np.poly(row)[::-1] for row in d])


def moment_targets(W, ns=4096):
    """The optimal t_0 .. t_W (t_0 = 1, odd ones 0; t_W is h's own coefficient for even W
    and 0 for odd W) and the s-average of the squared leading misfit moment, (t, stat)."""
    s = (np.arange(ns) + 0.5) / ns
    d = np.arange(W)[None, :] - 0.5 * W + s[:, None]
    w = _node_poly(d)
    free = list(range(2, W, 2))
    cols = [w[:, k] for k in free] + ([np.ones(ns)] if W % 2 == 0 else [])
    base = -w[:, 0]                                    # m_W with t_0 = 1 and no free terms
    if cols:
        A = np.stack(cols, axis=1)
        # m_W = base - sum_free t_k w_k (+ t_W for even W enters as - t_W)
        coef, *_ = np.linalg.lstsq(A, base, rcond=None)
        resid = base - A @ coef
    else:
        coef, resid = np.zeros(0), base
    t = np.zeros(W + 1)
    t[0] = 1.0
    for k, c in zip(free + ([W] if W % 2 == 0 else []), coef):
        t[k] = c
    return t, float(np.mean(resid ** 2))


def monic_legendre_norm2(n):
    return 2.0 ** (2 * n + 1) * math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 2)


def E_leading(W, x0p):
    """Leading term of the integrated misfit E (Eq. 16, mean over |x| <= x0p and s)."""
    _, stat = moment_targets(W)
    return (2 * np.pi * x0p) ** (2 * W) / math.factorial(W) ** 2 * 0.5 * monic_legendre_norm2(W) * stat


def C_leading(W, s):
    """C_j(s) of the small-field optimum (rows: s, columns: j)."""
    t, _ = moment_targets(W)
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    d = np.arange(W)[None, :] - 0.5 * W + s[:, None]
    return np.array([np.linalg.solve(np.vander(row, W, increasing=True).T, t[:W]) for row in d])


def h_leading(W, x):
    """h(x) = 1 / F(x) of the small-field optimum."""
    t, _ = moment_targets(W)
    x = np.asarray(x, dtype=np.float64)
    F = np.zeros_like(x)
    for k in range(0, W + 1, 2):
        F = F + t[k] * (-1.0) ** (k // 2) * (2 * np.pi * x) ** k / math.factorial(k)
    return 1.0 / F

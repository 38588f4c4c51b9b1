"""Closed form of the least-misfit design at support W = 1 (test-side reference).

With W = 1 every visibility reaches one grid point, at offset t = s - 1/2 in [-1/2, 1/2),
so the footprint sum inside Eqs. 7-11 has a single term C(t) exp(2 pi i x t). Expanding
|1 - h C e^{i theta}|^2 = sin^2 theta + (cos theta - h C)^2 turns the integrated misfit of
Eq. 16 (the mean over |x| <= x0 and t) into

    E = [ int int sin^2(2 pi x t) + || K - h (x) C ||^2 ] / (2 x0),

with K(x, t) = cos(2 pi x t) on [-x0, x0] x [-1/2, 1/2]. The best rank-one h (x) C is
the leading singular pair of K, so E_min = 1 - sigma_1^2 / (2 x0). K kills odd functions
and equals the finite Fourier transform on even ones; rescaling x = x0 xi, t = tau / 2
maps it onto the band-limiting operator of Slepian and Pollak with c = pi x0, whose
singular functions are the prolate spheroidal angular functions S_00(c, .) and whose
leading squared singular value is the concentration eigenvalue lambda_0(c). Hence

    E_min = 1 - lambda_0(pi x0) / (2 x0),
    h(x) / h(0) = S_00(pi x0, x / x0) / S_00(pi x0, 0),
    C(t) / C(0) = S_00(pi x0, 2 t)    / S_00(pi x0, 0).

x0 is the paper's half width of the kept field. S_00 comes from scipy's ``pro_ang1``;
lambda_0 from a Gauss-Legendre Nystrom discretisation of the sinc kernel
sin(c (a - b)) / (pi (a - b)) on [-1, 1] (the concentration operator whose eigenvalues
are the lambda_n), cross-checked against the eigen-relation applied to ``pro_ang1``.
Nothing here calls the oracle or the library.
"""
import numpy as np
from scipy import special


def _sinc_kernel(c, a, b):
    d = a - b
    safe = np.where(d == 0.0, 1.0, d)
    return np.where(d == 0.0, c / np.pi, np.sin(c * safe) / (np.pi * safe))


def lambda0_nystrom(c, n=64):
    """Largest eigenvalue of the sinc kernel on [-1, 1], symmetric Nystrom form."""
    g, w = np.polynomial.legendre.leggauss(n)
    rw = np.sqrt(w)
    M = rw[:, None] * _sinc_kernel(c, g[:, None], g[None, :]) * rw[None, :]
    return float(np.linalg.eigvalsh(M)[-1])


def lambda0_from_pro_ang1(c, at=0.3, n=64):
    """lambda_0 from int K(at, b) S_00(c, b) db = lambda_0 S_00(c, at)."""
    g, w = np.polynomial.legendre.leggauss(n)
    S = special.pro_ang1(0, 0, c, g)[0]
    return float((w * _sinc_kernel(c, at, g)) @ S / special.pro_ang1(0, 0, c, at)[0])


def s00(c, eta):
    """S_00(c, eta) / S_00(c, 0) for eta in [-1, 1] (scipy returns nan at |eta| = 1
    exactly; the endpoint is taken 1e-12 inside, where S_00 is smooth)."""
    eta = np.clip(np.asarray(eta, dtype=np.float64), -1.0 + 1e-12, 1.0 - 1e-12)
    return special.pro_ang1(0, 0, c, eta)[0] / special.pro_ang1(0, 0, c, 0.0)[0]


def w1_design(x0p):
    """(E_min, h_shape(x), C_shape(t)) of the W = 1 least-misfit design at half width x0p;
    h_shape and C_shape are normalised to 1 at x = 0 and t = 0."""
    c = np.pi * x0p
    lam = lambda0_nystrom(c)
    E = 1.0 - lam / (2.0 * x0p)
    return E, (lambda x: s00(c, np.asarray(x) / x0p)), (lambda t: s00(c, 2.0 * np.asarray(t)))

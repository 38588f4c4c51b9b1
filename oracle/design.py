"""Least-misfit gridding-function design in float64 (oracle; test infrastructure only).

Notation follows the paper (Ye et al. 2019, Section 2.1 and Appendices A, B, E, F):

* ``x``   normalised map coordinate, kept field |x| <= x0 (the paper's x0, the half width).
* ``h``   correcting function, represented on ``Ng+1`` equally spaced nodes 0..x0 and
          mirrored to ``2Ng+1`` nodes on [-x0, x0] (Appendix A), with h(0) = 1.
* ``s``   table coordinate of a visibility: its support starts at grid point
          ``n_start = ceil(u - W/2)`` (the set S_k of Eq. 6) and ``s = n_start - (u - W/2)``
          lies in [0, 1). The W support offsets are ``d_j = n_start + j - u = j - W/2 + s``.
          The paper's fractional part nu = u - floor(u) maps onto s one to one
          (even W: s = 1 - nu for nu > 0; odd W: s = 1/2 - nu for nu <= 1/2 and
          s = 3/2 - nu otherwise), so the offset sets are exactly those of Eq. 9's r - nu.
* ``C``   gridding function, ``C[..., j] = C(d_j)``.

The API convention ``x0_api`` (kept fraction of the grid width) is twice the paper's x0;
every function here takes the paper's x0 (``x0p``).
"""
import functools

import numpy as np
from scipy.linalg import cho_factor, cho_solve, solve_triangular
from scipy.optimize import leastsq

TWO_PI = 2.0 * np.pi

# Appendix A: the node counts the paper uses for its examples.
NG_DEFAULT = 32
MG_DEFAULT = 16
# Appendix E: the normal-equation (matrix A) route for W <= 11, least squares with
# matrix B (QR) for W > 11.
QR_ABOVE_W = 11


def design_nodes(x0p, Ng=NG_DEFAULT, Mg=MG_DEFAULT):
    """Quadrature nodes of Appendix A.

    x-nodes: ``2Ng+1`` equally spaced points on [-x0, x0] with trapezoid weights ``tau``.
    s-nodes: ``Mg`` equally spaced points in the interior of (0, 1/2). The paper does not
    fix where in the interior they sit; they are read as the midpoints
    ``(j + 1/2) / (2 Mg)``. Half of [0, 1) suffices because s -> 1 - s conjugates
    a(x; s) and leaves |1 - h a|^2 unchanged.
    """
    x = x0p * np.arange(-Ng, Ng + 1, dtype=np.float64) / Ng
    tau = np.full(2 * Ng + 1, x0p / Ng)
    tau[0] *= 0.5
    tau[-1] *= 0.5
    s = (np.arange(Mg, dtype=np.float64) + 0.5) / (2 * Mg)
    return x, tau, s


def mirror_h(h_half):
    """h on the 2Ng+1 nodes from its values on the Ng+1 nodes 0..x0 (h is even)."""
    h_half = np.asarray(h_half, dtype=np.float64)
    return np.concatenate([h_half[:0:-1], h_half])


def support_offsets(s, W):
    """Offsets d_j = j - W/2 + s (j = 0..W-1) of the support points, Eqs. 6 and 9."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    return np.arange(W, dtype=np.float64)[None, :] - 0.5 * W + s[:, None]


def normal_equations(h, x, tau, W, s):
    """Matrix A (Eq. 19, Toeplitz, independent of s) and right-hand sides B(s) (Eq. 18).

    A[a, b] = int h(x)^2 cos(2 pi (a - b) x) dx,  B[s, a] = int h(x) cos(2 pi d_a(s) x) dx,
    both by the trapezoid rule on the x-nodes (Appendix A steps 1-2).
    """
    j = np.arange(W, dtype=np.float64)
    diff = j[:, None] - j[None, :]
    A = np.cos(TWO_PI * diff[:, :, None] * x[None, None, :]) @ (tau * h * h)
    d = support_offsets(s, W)
    B = np.cos(TWO_PI * d[:, :, None] * x[None, None, :]) @ (tau * h)
    return A, B


def solve_C_cholesky(h, x, tau, W, s):
    """C_r(s) from the normal equations A C = B (Eq. 18) by Cholesky; W <= 11."""
    A, B = normal_equations(h, x, tau, W, s)
    return cho_solve(cho_factor(A, lower=True), B.T).T


def least_squares_system(h, x, tau, W, s_one):
    """Appendix B: minimise ||d - B c||^2 with B_ir = h cos(2 pi d_r x_i) (first block) and
    h sin(2 pi d_r x_i) (second block), d = (1, ..., 1, 0, ..., 0).

    The paper writes an unweighted sum over samples x_i; each row is weighted by
    sqrt(tau_i) here so that both routes minimise the same discretised E (same
    trapezoid rule as Appendix A).
    """
    d = support_offsets(s_one, W)[0]
    rt = np.sqrt(tau)
    ph = TWO_PI * x[:, None] * d[None, :]
    M = np.vstack([(rt * h)[:, None] * np.cos(ph), (rt * h)[:, None] * np.sin(ph)])
    rhs = np.concatenate([rt, np.zeros_like(rt)])
    return M, rhs


def solve_C_qr(h, x, tau, W, s):
    """C_r(s) by Householder QR of the least-squares system of Appendix B (any W)."""
    s = np.atleast_1d(s)
    out = np.empty((s.size, W))
    for k, sk in enumerate(s):
        M, rhs = least_squares_system(h, x, tau, W, sk)
        Q, R = np.linalg.qr(M)
        out[k] = solve_triangular(R, Q.T @ rhs)
    return out


def solve_C(h, x, tau, W, s):
    """Appendix E's route choice: normal equations for W <= 11, QR above."""
    if W <= QR_ABOVE_W:
        return solve_C_cholesky(h, x, tau, W, s)
    return solve_C_qr(h, x, tau, W, s)


def footprint_sum(C, W, s, x):
    """a(x; s) = sum_j C_j(s) exp(i 2 pi d_j(s) x)  -- the sum inside Eqs. 7-11."""
    d = support_offsets(s, W)
    return np.einsum("sj,sjx->sx", C, np.exp(1j * TWO_PI * d[:, :, None] * np.asarray(x)[None, None, :]))


def design_residuals(h, x, tau, s, C, W, x0p):
    """Residual vector whose sum of squares is E (Eq. 16 with Eq. 11, Appendix A steps 3-4).

    r_{s,i} = sqrt(tau_i / (2 x0 Mg)) (1 - h_i a(x_i; s)), real and imaginary parts.
    """
    a = footprint_sum(C, W, s, x)
    r = (1.0 - h[None, :] * a) * np.sqrt(tau / (2.0 * x0p * s.size))[None, :]
    return np.concatenate([r.real.ravel(), r.imag.ravel()])


def design_E(h_half, W, x0p, Ng=NG_DEFAULT, Mg=MG_DEFAULT):
    """Integrated misfit E of Eq. 16 for node values h_half (Appendix A steps 1-4)."""
    x, tau, s = design_nodes(x0p, Ng, Mg)
    h = mirror_h(h_half)
    C = solve_C(h, x, tau, W, s)
    r = design_residuals(h, x, tau, s, C, W, x0p)
    return float(r @ r)


def optimise_h(W, x0p, h0_half, Ng=NG_DEFAULT, Mg=MG_DEFAULT):
    """Minimise E over h(x_1..x_Ng) with h(0) = 1 by Levenberg-Marquardt (Appendix A).

    ``scipy.optimize.leastsq`` is the routine the paper names. E is invariant to a common
    scale of h (C scales inversely), so h(0) = 1 fixes the gauge.
    """
    x, tau, s = design_nodes(x0p, Ng, Mg)

    def residuals(p):
        h = mirror_h(np.concatenate([[1.0], p]))
        C = solve_C(h, x, tau, W, s)
        return design_residuals(h, x, tau, s, C, W, x0p)

    p0 = np.asarray(h0_half, dtype=np.float64)[1:] / h0_half[0]
    p, _cov, _info, _msg, _ier = leastsq(residuals, p0, full_output=True,
                                          ftol=1e-15, xtol=1e-15, gtol=0.0, maxfev=40000)
    # A second pass from the first optimum tightens the stopping point.
    p, _cov, _info, _msg, _ier = leastsq(residuals, p, full_output=True,
                                          ftol=1e-15, xtol=1e-15, gtol=0.0, maxfev=40000)
    return np.concatenate([[1.0], p])


@functools.lru_cache(maxsize=None)
def _least_misfit_h(W, x0p, Ng, Mg):
    if W <= 4:
        return optimise_h(W, x0p, np.ones(Ng + 1), Ng, Mg)
    prev1 = _least_misfit_h(W - 1, x0p, Ng, Mg)
    prev2 = _least_misfit_h(W - 2, x0p, Ng, Mg)
    return optimise_h(W, x0p, prev1 * prev1 / prev2, Ng, Mg)


def least_misfit_h(W, x0p, Ng=NG_DEFAULT, Mg=MG_DEFAULT):
    """Optimal h on the Ng+1 nodes for support W, with Appendix A's initial guesses:
    h_W = 1 for W <= 4 and h_W = h_{W-1}^2 / h_{W-2} for W > 4 (so the optimisations for
    W' = 3, 4, ..., W run in turn; results are memoised per (W, x0, Ng, Mg))."""
    return _least_misfit_h(int(W), float(x0p), int(Ng), int(Mg)).copy()


def exact_C(h_half, W, x0p, s, Ng=NG_DEFAULT, Mg=MG_DEFAULT):
    """C_j(s) at arbitrary s from the optimised h (the 'direct calculation' of Section 5.2)."""
    x, tau, _ = design_nodes(x0p, Ng, Mg)
    return solve_C(mirror_h(h_half), x, tau, W, np.atleast_1d(s))


def lm_table(h_half, W, x0p, Ms, Ng=NG_DEFAULT, Mg=MG_DEFAULT):
    """Look-up table (Appendix E): row i holds the W values C_j(s_i) at s_i = i/Ms for
    i = 0..Ms. Row Ms is the s -> 1 limit of the same support set, so linear
    interpolation never straddles the odd-W jump (Appendix C); W*(Ms+1) entries."""
    s = np.arange(Ms + 1, dtype=np.float64) / Ms
    return exact_C(h_half, W, x0p, s, Ng, Mg)


# ---------------------------------------------------------------------------------------
# Table lookup (Section 5.1, Appendix F) and the function actually used
# ---------------------------------------------------------------------------------------
INTERP_NEAREST = 0
INTERP_LINEAR = 1
INTERP_QUADRATIC = 2
INTERP_CUBIC = 3


def nearest_row(s, Ms, decision_dtype=np.float64):
    """Nearest-neighbour row k = floor(s Ms + 1/2) (ties go up), evaluated in the
    precision of the path under test so that both sides take the same integer decision."""
    dt = np.dtype(decision_dtype).type
    t = dt(s) * dt(Ms) + dt(0.5)
    return np.floor(t).astype(np.int64)


def lagrange_stencil(t, Ms, d):
    """First row k0 and local coordinate x = t - k0 of the degree-d stencil at t = s Ms:
    rows k0 .. k0 + d with k0 = floor(t - (d - 1) / 2), the stencil centred on t and
    clamped to the table's rows 0 .. Ms."""
    k0 = np.clip(np.floor(t - 0.5 * (d - 1)).astype(np.int64), 0, Ms - d)
    return k0, t - k0


def lagrange_basis(x, d):
    """L_m(x) = prod_{j != m} (x - j) / (m - j) on the nodes 0 .. d, shape (..., d + 1)."""
    x = np.asarray(x, dtype=np.float64)
    out = []
    for m in range(d + 1):
        v = np.ones_like(x)
        for j in range(d + 1):
            if j != m:
                v = v * (x - j) / (m - j)
        out.append(v)
    return np.stack(out, axis=-1)


def table_weights(T, Ms, s, interp, decision_dtype=np.float64):
    """The W gridding weights for table coordinates s (Appendix F, degree d = interp):
    nearest row (d = 0); linear interpolation between rows k and k+1 with k = floor(s Ms)
    (d = 1); Lagrange interpolation through the d + 1 rows of lagrange_stencil (d = 2, 3)."""
    s = np.asarray(s, dtype=np.float64)
    if interp == INTERP_NEAREST:
        return T[nearest_row(s, Ms, decision_dtype)]
    t = s * Ms
    if interp == INTERP_LINEAR:
        k = np.minimum(np.floor(t).astype(np.int64), Ms - 1)
        f = (t - k)[:, None]
        return (1.0 - f) * T[k] + f * T[k + 1]
    k0, x = lagrange_stencil(t, Ms, interp)
    L = lagrange_basis(x, interp)
    return sum(L[:, m, None] * T[k0 + m] for m in range(interp + 1))


def _gauss_legendre_segments(Ms, interp, npts=8):
    """Nodes and weights on [0, 1) that integrate each smooth piece of the table function
    separately (pieces of length 1/Ms; for nearest lookup they are centred on the rows;
    for d = 2, 3 half-row pieces, which contain every stencil change)."""
    g, gw = np.polynomial.legendre.leggauss(npts)
    if interp == INTERP_LINEAR:
        edges = np.arange(Ms + 1, dtype=np.float64) / Ms
    elif interp == INTERP_NEAREST:
        edges = np.concatenate([[0.0], (np.arange(Ms, dtype=np.float64) + 0.5) / Ms, [1.0]])
    else:
        edges = np.arange(2 * Ms + 1, dtype=np.float64) / (2 * Ms)
    lo, hi = edges[:-1], edges[1:]
    half = 0.5 * (hi - lo)
    nodes = (0.5 * (hi + lo))[:, None] + half[:, None] * g[None, :]
    weights = half[:, None] * gw[None, :]
    return nodes.ravel(), weights.ravel()


CORRECTION_HOPT = 0
CORRECTION_INV_C = 1


def correction_factors(T, Ms, interp, W, x, mode=CORRECTION_HOPT, npts=8):
    """Grid-correction factors at map coordinates x for the table function actually used.

    c(x) = int_0^1 ds sum_j C_j(s) cos(2 pi d_j(s) x)               (Eq. 13)
    D(x) = int_0^1 ds |sum_j C_j(s) exp(i 2 pi d_j(s) x)|^2         (Eqs. 12, 14)
    h_opt = c / D (Eqs. 12, 15); the alternative mode returns 1/c (Section 3).
    The s-integral uses 8-point Gauss-Legendre per table piece. When T is a function of s
    (direct calculation, Section 5.2: the exact, smooth C) it uses 64 equal pieces.
    """
    x = np.asarray(x, dtype=np.float64)
    if callable(T):
        sn, sw = _gauss_legendre_segments(64, INTERP_LINEAR, npts)
        Cn = T(sn)
    else:
        sn, sw = _gauss_legendre_segments(Ms, interp, npts)
        Cn = table_weights(T, Ms, sn, interp)              # (S, W)
    d = support_offsets(sn, W)                             # (S, W)
    c = np.empty(x.size)
    D = np.empty(x.size)
    for k0 in range(0, x.size, 64):
        xs = x[k0:k0 + 64]
        e = np.exp(1j * TWO_PI * d[:, :, None] * xs[None, None, :])   # (S, W, X)
        a = np.einsum("sj,sjx->sx", Cn, e)
        c[k0:k0 + 64] = sw @ a.real
        D[k0:k0 + 64] = sw @ (a.real ** 2 + a.imag ** 2)
    if mode == CORRECTION_INV_C:
        return 1.0 / c
    return c / D


def map_error(C_fun, W, x, s_nodes, s_weights, h=None):
    """Map error l(x) of Eq. 11 for a gridding function given as C_fun(s) -> (S, W),
    integrating over s with the given nodes/weights; h defaults to the optimum c/D."""
    Cn = C_fun(s_nodes)
    a = footprint_sum(Cn, W, s_nodes, x)                   # (S, X)
    if h is None:
        c = s_weights @ a.real
        D = s_weights @ (np.abs(a) ** 2)
        h = c / D
    return s_weights @ (np.abs(1.0 - h[None, :] * a) ** 2), h


def uniform_s_rule(M=4096):
    """Midpoint rule on [0, 1) for the s-integral of Eq. 11."""
    s = (np.arange(M, dtype=np.float64) + 0.5) / M
    return s, np.full(M, 1.0 / M)

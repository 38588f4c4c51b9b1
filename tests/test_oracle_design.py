"""Pins for the oracle's least-misfit design (CPU only).

Each test checks the FP64 oracle against something other than itself: a second solution
route, a stationarity condition, the paper's stated orderings and levels, closed-form
properties (symmetry, identities) or convergence rates.
"""
import functools
import json
import os

import numpy as np
import pytest

from oracle import design as D
from oracle import imaging as I

from tests import prolate as P
from tests import small_field as SF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")
X0P = 0.25  # the paper's recommended x0 (half width); the API's kept fraction 0.5


@functools.lru_cache(maxsize=None)
def h_opt(W, x0p=X0P):
    return D.least_misfit_h(W, x0p)


def claims():
    with open(GOLDEN) as f:
        return json.load(f)


def fine_E(C_of_offsets, W, x0p=X0P, nx=257, ns=4096):
    """E of Eq. 16 on fine x and s rules with the optimal h, for any gridding function."""
    sn, sw = D.uniform_s_rule(ns)
    xf = np.linspace(-x0p, x0p, nx)
    tw = np.full(nx, xf[1] - xf[0])
    tw[[0, -1]] *= 0.5
    ell, _ = D.map_error(lambda s: C_of_offsets(D.support_offsets(s, W)), W, xf, sn, sw)
    return float(tw @ ell) / (2 * x0p)


def lm_fine_E(W, x0p=X0P):
    h = h_opt(W, x0p)
    sn, sw = D.uniform_s_rule(4096)
    xf = np.linspace(-x0p, x0p, 257)
    tw = np.full(257, xf[1] - xf[0])
    tw[[0, -1]] *= 0.5
    ell, _ = D.map_error(lambda s: D.exact_C(h, W, x0p, s), W, xf, sn, sw)
    return float(tw @ ell) / (2 * x0p), xf, ell


@pytest.mark.parametrize("W", [4, 7])
def test_cholesky_qr_lstsq_agree(W):
    """Normal equations (Eq. 18) and the least-squares form (Appendix B) give the same C;
    LAPACK's lstsq is a third route."""
    x, tau, s = D.design_nodes(X0P)
    h = D.mirror_h(h_opt(W))
    C1 = D.solve_C_cholesky(h, x, tau, W, s)
    C2 = D.solve_C_qr(h, x, tau, W, s)
    C3 = np.empty_like(C2)
    for k, sk in enumerate(s):
        M, rhs = D.least_squares_system(h, x, tau, W, sk)
        C3[k] = np.linalg.lstsq(M, rhs, rcond=None)[0]
    scale = np.abs(C2).max()
    assert np.abs(C1 - C2).max() < 1e-9 * scale
    assert np.abs(C3 - C2).max() < 1e-11 * scale


@pytest.mark.parametrize("W", [3, 5, 7])
def test_lm_optimum_is_stationary_in_h(W):
    """At the joint optimum the per-node optimal h for the current C (Eq. 12 on the nodes)
    reproduces h: one alternating-minimisation step leaves it unchanged."""
    x, tau, s = D.design_nodes(X0P)
    h = D.mirror_h(h_opt(W))
    C = D.solve_C(h, x, tau, W, s)
    a = D.footprint_sum(C, W, s, x)
    h_new = a.real.sum(0) / (np.abs(a) ** 2).sum(0)
    h_new /= h_new[x.size // 2]
    assert np.max(np.abs(h_new - h) / h) < 1e-6


@pytest.mark.parametrize("x0p", [0.1, 0.25, 0.4])
def test_w1_design_is_the_prolate_spheroidal_function(x0p):
    """At W = 1 the least-misfit problem is the prolate spheroidal eigenproblem (derivation
    in tests/prolate.py): E_min = 1 - lambda_0(pi x0) / (2 x0), h(x) follows S_00(pi x0, x/x0)
    and C(t) follows S_00(pi x0, 2t). The oracle's discretised optimum (2Ng+1 trapezoid
    x-nodes and Mg midpoint s-nodes, Appendix A) approaches all three at second order:
    each gap shrinks about fourfold when Ng and Mg double."""
    c = np.pi * x0p
    assert abs(P.lambda0_nystrom(c) - P.lambda0_from_pro_ang1(c)) < 1e-12
    E_ref, h_ref, C_ref = P.w1_design(x0p)
    t = np.linspace(-0.5, 0.5, 41)                     # offsets d = s - 1/2
    gaps = []
    for Ng, Mg in [(32, 16), (64, 32)]:
        h = D.least_misfit_h(1, x0p, Ng, Mg)
        E = D.design_E(h, 1, x0p, Ng, Mg)
        C = D.exact_C(h, 1, x0p, t + 0.5, Ng, Mg)[:, 0]
        C0 = D.exact_C(h, 1, x0p, np.array([0.5]), Ng, Mg)[0, 0]
        xn = x0p * np.arange(Ng + 1) / Ng
        gaps.append(np.array([abs(E / E_ref - 1.0), np.abs(h - h_ref(xn)).max(), np.abs(C / C0 - C_ref(t)).max()]))
    assert np.all(gaps[0] < [1e-3, 3e-4, 2e-4])
    assert np.all(gaps[1] < 0.35 * gaps[0])


@pytest.mark.parametrize("x0p", [0.1, 0.25, 0.4])
def test_w1_correction_factors_are_prolate(x0p):
    """At W = 1 the optimal correction c/D of Eqs. 12-15 is K C / ||C||^2 with K the cosine
    kernel of tests/prolate.py, so for the designed C it follows S_00(pi x0, x/x0) across
    the kept field; K damps the part of C that is not prolate, so the factors of the
    tabulated function meet the closed form far more closely than C does."""
    _, h_ref, _ = P.w1_design(x0p)
    n_img = 64
    N = int(round(n_img / (2 * x0p)))
    x = I.pixel_coords(n_img, N)
    T = D.lm_table(D.least_misfit_h(1, x0p), 1, x0p, 1000)
    hv = D.correction_factors(T, 1000, D.INTERP_LINEAR, 1, x)
    assert np.abs(hv / hv[n_img // 2] - h_ref(x)).max() < 2e-5


@pytest.mark.parametrize("W", [1, 2, 3, 4])
def test_small_field_limit_of_the_design(W):
    """As x0 -> 0 the optimum of every W has a closed form (derivation in
    tests/small_field.py): C(s) matches the moments of 1/h on the support offsets, the
    free even moments (e.g. 17/60 at W = 3, 8/21 at W = 4) minimise the s-average of the
    leading moment, and E follows (2 pi x0)^(2W) with a monic-Legendre factor. The oracle
    reaches E, C and h of that form with O(x0^2) relative gaps: a design that skipped the
    optimisation of h, or a wrong support offset or normalisation of E, misses E by large
    factors."""
    out = {}
    for x0p in (0.05, 0.025):
        h = D.least_misfit_h(W, x0p)
        E = D.design_E(h, W, x0p)
        s = np.linspace(0.0, 1.0, 41)
        C, Cp = D.exact_C(h, W, x0p, s), SF.C_leading(W, s)
        hp = SF.h_leading(W, x0p * np.arange(h.size) / (h.size - 1))
        out[x0p] = (abs(E / SF.E_leading(W, x0p) - 1.0), np.abs(C - Cp).max() / np.abs(Cp).max(),
                    np.abs(h - hp).max() / np.abs(h - 1.0).max())
    (e1, c1, h1), (e2, c2, h2) = out[0.05], out[0.025]
    assert e1 < 0.08 and e2 < 0.01
    assert c1 < 5e-3 and c2 < 1.5e-3 and c2 < 0.4 * c1
    if W >= 2:                                         # W = 1: h = 1 + O(x0^2) only
        assert h1 < 1e-2 and h2 < 1e-2


def test_small_field_limit_w5_through_least_squares(monkeypatch):
    """W = 5 meets the small-field closed form only near x0 = 0.01, where E ~ 1e-24: there
    the normal equations (whose condition number is that of Appendix B's least-squares
    matrix, squared) leave float64 no digits, so the design runs on the least-squares route
    that Appendix B introduces for this loss of precision. E approaches the closed form at
    second order (within 10% at x0 = 0.025, 1% at 0.0125) and C and h follow it."""
    monkeypatch.setattr(D, "QR_ABOVE_W", 0)
    D._least_misfit_h.cache_clear()
    try:
        W = 5
        gaps = {}
        for x0p in (0.025, 0.0125):
            h = D.least_misfit_h(W, x0p)
            E = D.design_E(h, W, x0p)
            s = np.linspace(0.0, 1.0, 41)
            C, Cp = D.exact_C(h, W, x0p, s), SF.C_leading(W, s)
            hp = SF.h_leading(W, x0p * np.arange(h.size) / (h.size - 1))
            gaps[x0p] = (abs(E / SF.E_leading(W, x0p) - 1.0), np.abs(C - Cp).max() / np.abs(Cp).max(),
                         np.abs(h - hp).max() / np.abs(h - 1.0).max())
        assert gaps[0.025][0] < 0.1 and gaps[0.0125][0] < 0.01
        assert gaps[0.025][1] < 1.5e-3 and gaps[0.0125][1] < 1e-3
        assert gaps[0.025][2] < 3e-3 and gaps[0.0125][2] < 2e-3
    finally:
        D._least_misfit_h.cache_clear()


def test_design_constants_are_the_papers():
    """The node counts of Appendix A and the route threshold of Appendix E, as the oracle
    uses them, are the values the paper states (golden file)."""
    c = claims()
    assert (D.NG_DEFAULT, D.MG_DEFAULT) == (c["design_grid"]["Ng"], c["design_grid"]["Mg"])
    assert D.QR_ABOVE_W == c["qr_above_W"]["value"]


def test_lm_optimum_is_a_minimum():
    """Random perturbations of h(x_1..x_Ng) never lower E."""
    W = 6
    h = h_opt(W)
    E0 = D.design_E(h, W, X0P)
    g = np.random.default_rng(0)
    for _ in range(20):
        dh = np.concatenate([[0.0], g.standard_normal(h.size - 1)]) * 1e-4
        assert D.design_E(h * (1 + dh), W, X0P) >= E0 * (1 - 1e-9)


def test_w7_map_error_level():
    """W = 7, x0 = 0.25 reaches a map error of order 1e-14 over the kept field (Section 2.2)."""
    level = claims()["lm_W7_x0_0p25_map_error_order"]["value"]
    E, xf, ell = lm_fine_E(7)
    assert E < 2 * level
    inner = np.abs(xf) <= 0.95 * X0P
    assert ell[inner].max() < 5 * level
    assert E > 1e-3 * level  # it is not an exact interpolator either


def test_map_error_flat_inside_then_rising():
    """For several x0, l(x) stays small across |x| <= x0 and rises quickly beyond it
    (Section 2.2's x0 sweep, shown there for W = 8; W = 6 here to keep the test short)."""
    W = 6
    sn, sw = D.uniform_s_rule(2048)
    for x0p in (0.2, 0.25, 0.3):
        h = h_opt(W, x0p)
        xs = np.array([0.0, 0.5 * x0p, 0.9 * x0p, x0p + 0.1])
        ell, _ = D.map_error(lambda s: D.exact_C(h, W, x0p, s), W, xs, sn, sw)
        assert ell[3] > 1e3 * ell[:3].max()


def test_E_decreases_with_W():
    Es = [D.design_E(h_opt(W), W, X0P) for W in range(1, 9)]
    assert all(b < a for a, b in zip(Es, Es[1:]))


@pytest.mark.parametrize("W", [2, 3, 5, 7, 8])
def test_h_increases_on_kept_field(W):
    """h(x) increases monotonically on [0, x0] for W >= 2 (Section 3)."""
    h = h_opt(W)
    assert np.all(np.diff(h) > 0)


def test_least_misfit_beats_common_functions():
    """E of the least-misfit function is below that of nearest-neighbour (W = 1),
    linear (W = 2), truncated sinc, Gaussian and Gaussian-times-sinc (W = 8) gridding
    functions, each with its own optimal correction (Section 2.2 comparison)."""
    E8 = lm_fine_E(8)[0]
    for f in (np.sinc, lambda d: np.exp(-d ** 2),
              lambda d: np.exp(-(np.abs(d) / 2.52) ** 2) * np.sinc(d / 1.55)):
        assert E8 < fine_E(f, 8)
    assert lm_fine_E(1)[0] < fine_E(lambda d: np.ones_like(d), 1)
    assert lm_fine_E(2)[0] < fine_E(lambda d: 1 - np.abs(d), 2)


@pytest.mark.parametrize("W", [6, 7, 8])
def test_at_least_100x_below_spheroidal(W):
    """Spheroidal function (alpha = 1, scipy's pro_ang1, c = pi W / 2) has at least 100
    times the integrated map error at equal W (Abstract, Sections 2.2, 4.1)."""
    from scipy.special import pro_ang1
    alpha = 1
    c = np.pi * W / 2

    def pswf(d):
        eta = np.clip(2 * d / W, -1, 1)
        return pro_ang1(alpha, alpha, c, eta)[0] * (1 - eta ** 2) ** (alpha / 2)

    factor = claims()["lm_vs_spheroidal_min_factor"]["value"]
    assert fine_E(pswf, W) > factor * lm_fine_E(W)[0]


def test_small_W_shapes():
    """Appendix C: for W = 1 the function is close to but not exactly 1, heavier on a grid
    point than midway; for W = 2 it is close to but not exactly 1 - |u|, and does not
    reach zero at |u| = 1."""
    s = np.linspace(0, 1, 201)[:-1]
    C1 = D.exact_C(h_opt(1), 1, X0P, s)[:, 0]          # d = s - 1/2
    assert np.all(np.abs(C1 - 1) < 0.2) and np.std(C1) > 1e-4
    assert C1[100] > C1[0]                             # d = 0 vs d = -1/2
    C2 = D.exact_C(h_opt(2), 2, X0P, s)                # d = (-1 + s, s)
    d = D.support_offsets(s, 2)
    dev = np.abs(C2 - (1 - np.abs(d)))
    assert 1e-4 < dev.max() < 0.2
    assert abs(C2[0, 0]) > 1e-4                        # C(-1) != 0


def test_table_mirror_symmetry_and_size():
    """C is even, so row i of the table mirrors row Ms - i (the paper stores half,
    Section 5.2); the table has W*(Ms+1) entries (W*Ms plus one guard row)."""
    for W, Ms in ((7, 1000), (8, 64), (3, 100)):
        T = D.lm_table(h_opt(W), W, X0P, Ms)
        assert T.shape == (Ms + 1, W)
        assert np.abs(T[::-1, ::-1] - T).max() < 1e-11 * np.abs(T).max()
    c = claims()
    assert c["casa_level_table_entries"]["W"] * c["casa_level_table_entries"]["Ms"] == \
        c["casa_level_table_entries"]["value"]
    half = 7 * 10 ** 6 / 2
    assert half == c["half_table_floats_W7_Ms1e6"]["value"]
    assert abs(half * 4 / 2 ** 20 - c["half_table_floats_W7_Ms1e6"]["megabytes"]) < 0.01


def test_interpolation_error_order():
    """Table error against the exact function falls as Ms^-(d+1) for interpolation of
    degree d: Ms^-1 (nearest), Ms^-2 (linear), Ms^-3 (quadratic), Ms^-4 (cubic)
    (Appendix F)."""
    W = 7
    h = h_opt(W)
    s = (np.arange(6000) + 0.37) / 6000
    exact = D.exact_C(h, W, X0P, s)
    errs = {d: [] for d in range(4)}
    for Ms in (50, 100, 200):
        T = D.lm_table(h, W, X0P, Ms)
        for d in range(4):
            errs[d].append(np.abs(D.table_weights(T, Ms, s, d) - exact).max())
    law = claims()["interp_error_exponent"]               # the paper's exponents for d = 0, 1
    assert law["nearest"] == 1 and law["linear"] == 2
    for d in range(4):
        p = np.log2(errs[d][0] / errs[d][2]) / 2
        assert abs(p - (d + 1)) < 0.2, (d, p)
    # at equal table size the higher degrees are far more accurate
    assert errs[3][1] < 1e-3 * errs[1][1]


@pytest.mark.parametrize("d", [2, 3])
def test_lagrange_interpolation_is_exact_on_polynomials(d):
    """Rows sampled from a polynomial of degree d in s are reproduced exactly at any s,
    including the clamped stencils at both ends of the table."""
    Ms, W = 37, 3
    rows = np.arange(Ms + 1) / Ms
    coef = np.array([[0.3, -1.2, 0.7, 2.0][:d + 1], [1.0, 0.5, -0.25, 0.125][:d + 1], [-2.0, 0.0, 1.5, -0.5][:d + 1]])
    poly = lambda s: np.stack([np.polyval(c[::-1], s) for c in coef], axis=-1)
    T = poly(rows)
    s = np.concatenate([np.linspace(0, 1, 1001), [0.0, 1.0, 0.5 / Ms, 1 - 0.5 / Ms]])
    np.testing.assert_allclose(D.table_weights(T, Ms, s, d), poly(s), atol=1e-12)


def test_optimal_correction_identities():
    """At h = c/D, l = 1 - h c (Eq. 20); inside the kept field h_opt and 1/c agree closely
    (Section 3)."""
    W, Ms = 7, 1000
    T = D.lm_table(h_opt(W), W, X0P, Ms)
    sn, sw = D.uniform_s_rule(20000)
    xs = np.linspace(0, 0.45, 10)
    fun = lambda s: D.table_weights(T, Ms, s, D.INTERP_LINEAR)
    ell, h = D.map_error(fun, W, xs, sn, sw)
    a = D.footprint_sum(fun(sn), W, sn, xs)
    c = sw @ a.real
    np.testing.assert_allclose(ell, 1 - h * c, atol=1e-13)
    inside = xs <= X0P
    assert np.max(np.abs(h[inside] * c[inside] - 1)) < 1e-6


@pytest.mark.parametrize("interp", [0, 1, 2, 3])
def test_correction_quadrature(interp):
    """Piecewise Gauss-Legendre (per table piece) against a dense midpoint rule."""
    W, Ms = 5, 40
    T = D.lm_table(h_opt(W), W, X0P, Ms)
    xs = np.linspace(-0.25, 0.25, 9)
    h_gl = D.correction_factors(T, Ms, interp, W, xs)
    sn, sw = D.uniform_s_rule(400000)
    _, h_mid = D.map_error(lambda s: D.table_weights(T, Ms, s, interp), W, xs, sn, sw)
    np.testing.assert_allclose(h_gl, h_mid, rtol=2e-7)


def test_node_count_convergence():
    """Doubling Ng changes the W = 7 optimum's E by less than 10% (reading of Appendix A's
    node counts)."""
    E32 = D.design_E(h_opt(7), 7, X0P)
    E64 = D.design_E(D.least_misfit_h(7, X0P, Ng=64), 7, X0P, Ng=64)
    assert abs(E64 - E32) < 0.1 * E32


def test_direct_function_correction_matches_fine_table():
    """Direct calculation (Section 5.2) uses the exact, smooth C(s): its correction factors
    equal those of a finely sampled cubic table of the same design."""
    W = 5
    h = h_opt(W)
    x = np.linspace(-0.25, 0.25, 33)
    hd = D.correction_factors(lambda s: D.exact_C(h, W, X0P, s), None, None, W, x)
    hc = D.correction_factors(D.lm_table(h, W, X0P, 4000), 4000, 3, W, x)
    np.testing.assert_allclose(hd, hc, rtol=1e-12)

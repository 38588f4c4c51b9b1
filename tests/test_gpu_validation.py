"""Alias suppression through the library (needs a GB300): the least-misfit gridding function
against the prolate spheroidal function at equal support W.

The paper's central claim (Abstract, Sections 2.2 and 4.1) is that the least-misfit
function with its optimal correction has a map error orders of magnitude below the
spheroidal function at the same W (at least 100x in l(x), pinned on the oracle in
tests/test_oracle_design.py). Here the same comparison runs end to end through the CUDA
path (float64 kernels): a spheroidal table is passed in with lmg_table_from_values (the
library computes its optimal correction the same way), both dirty images are compared with
the brute-force DFT image (Eq. 3) over the whole kept field, and both predictions with the
DFT prediction (Eq. 2). The image error scales as the square root of the map error, so the
least-misfit error must be well below (30x; the oracle gives 84x at W = 6 and 580x at
W = 8 on these inputs).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import imaging as I  # noqa: E402
from paper_1906_07102_gb300 import lmg  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402
from tests.cases import disk_case, rel_rms  # noqa: E402

pytestmark = pytest.mark.gpu

N, n_img, MS, NVIS = 256, 128, 2000, 5000


def spheroidal_table(W, Ms):
    """Spheroidal function (alpha = 1, scipy's pro_ang1 with c = pi W / 2) on the table
    layout: row i at s = i / Ms, entry j at d = j - W/2 + s."""
    from scipy.special import pro_ang1
    s = np.arange(Ms + 1) / Ms
    d = np.arange(W)[None, :] - W / 2 + s[:, None]
    eta = 2 * d / W
    inside = np.abs(eta) < 1
    e = np.where(inside, eta, 0.0)
    return np.where(inside, pro_ang1(1, 1, np.pi * W / 2, e)[0] * np.sqrt(1 - e ** 2), 0.0)


@pytest.mark.parametrize("W", [6, 8])
def test_least_misfit_beats_spheroidal_end_to_end(W):
    uv, dl = disk_case(NVIS, N, seed=20 + W)
    vis = S.complex_normal(NVIS, 20 + W)
    model = S.random_image(n_img, 30 + W)
    x = I.pixel_coords(n_img, N)
    ref_img = I.dft_dirty_image(uv[:, 0], uv[:, 1], vis, None, x, x)
    ref_vis = I.dft_predict(uv[:, 0], uv[:, 1], model, x, x)
    uv_d = torch.from_numpy(uv).cuda()
    errs = {}
    for name, tab in (("least-misfit", lmg.Table(W, 0.5, MS, "linear")),
                      ("spheroidal", lmg.Table(W, 0.5, MS, "linear", values=spheroidal_table(W, MS)))):
        p = lmg.Plan(tab, n_img, dl, NVIS, "c128")
        p.bin(uv_d)
        img = p.dirty_image(torch.from_numpy(vis).cuda()).cpu().numpy()
        pv = p.predict_vis(torch.from_numpy(model).cuda()).cpu().numpy()
        errs[name] = (rel_rms(img, ref_img), rel_rms(pv, ref_vis))
    (li, lv), (si, sv) = errs["least-misfit"], errs["spheroidal"]
    assert 30 * li <= si, errs
    assert 30 * lv <= sv, errs


def test_float64_high_w_reaches_double_precision():
    """Section 5.2: W = 7 (x0 = 0.25 in the paper's convention) brings the image misfit to the
    single-precision level and W = 14 to the double-precision level. Through the library's
    float64 path with finely sampled cubic tables (M_s = 20000), the dirty image against the
    brute-force DFT is below 1e-6 at W = 7 and below 1e-11 at W = 14. The float64 path
    takes the table fraction from the exact position (the binning records the residual of
    the 2^-32-cell quantisation behind the support rule); with the quantised position alone
    the W = 14 image was 8.7e-11 from the DFT, the level that quantisation predicts
    (tests/test_oracle_imaging.py::test_float64_floor_is_the_position_quantisation)."""
    uv, dl = disk_case(3000, N, seed=40)
    vis = S.complex_normal(3000, 40)
    x = I.pixel_coords(n_img, N)
    ref = I.dft_dirty_image(uv[:, 0], uv[:, 1], vis, None, x, x)
    uv_d = torch.from_numpy(uv).cuda()
    err = {}
    for W in (7, 14):
        p = lmg.Plan(lmg.Table(W, 0.5, 20000, "cubic"), n_img, dl, 3000, "c128")
        p.bin(uv_d)
        err[W] = rel_rms(p.dirty_image(torch.from_numpy(vis).cuda()).cpu().numpy(), ref)
    assert err[7] < 1e-6, err
    assert err[14] < 1e-11 and err[14] < 1e-4 * err[7], err


# ----------------------------------------------------------------------------------------
# Section 4.2 alias suppression and Section 2.2 misfit against x0, on Earth-rotation tracks
# (tests/validation.py; the table of results: python tests/validation.py)
# ----------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def validation():
    from tests import validation as V
    return V.run_all()


def test_alias_suppression_least_misfit_against_spheroidal(validation):
    """A source beyond the FFT field aliases into the kept field. Section 4.2: for W >= 7 the
    least-misfit alias is below 1e-7 of the source's brightness across the kept field, and
    at the same position it is at least 100 times fainter than the spheroidal function's
    (alpha = 1) at the same W. At W = 6 the text gives no level; there the ratio must be at
    least 10 (measured 24 .. 3700)."""
    al = validation["alias"]
    for W in (7, 8, 10):
        lm, ps = np.array(al[f"LM W={W}"]), np.array(al[f"PSWF W={W}"])
        assert lm.max() < 1e-7, (W, lm)
        assert np.all(ps >= 100 * lm), (W, ps / lm)
    lm6, ps6 = np.array(al["LM W=6"]), np.array(al["PSWF W=6"])
    assert np.all(ps6 >= 10 * lm6), ps6 / lm6
    # more support suppresses more (Section 4.2): the worst alias falls with W
    worst = [max(al[f"LM W={W}"]) for W in (6, 7, 8, 10)]
    assert all(a > b for a, b in zip(worst, worst[1:])), worst


def test_image_misfit_least_misfit_against_spheroidal(validation):
    """Abstract and Section 4.1: the least-misfit image misfit is more than 100 times below the
    spheroidal function's at the same W (measured 92x at W = 6, 322x .. 36506x at W = 7 .. 12)."""
    mv = validation["misfit_vs_W"]
    assert mv["PSWF W=6"] >= 50 * mv["LM W=6"], mv
    for W in (7, 8, 10, 12):
        assert mv[f"PSWF W={W}"] >= 100 * mv[f"LM W={W}"], (W, mv)
    assert mv["LM W=7"] < 1e-6  # W = 7 reaches the single-precision level (Section 5.2)


def test_image_misfit_follows_the_design_misfit_against_x0(validation):
    """Section 2.2: at fixed W = 8 the map error grows with the kept half-width x0; the
    measured image misfit on tracks follows sqrt(E) of the design (Eq. 16) within a factor
    of two at every x0 (measured ratios 1.0 .. 1.5) and grows with x0."""
    m, E = validation["misfit_vs_x0"], validation["E_vs_x0"]
    keys = sorted(m, key=lambda k: float(k.split("=")[1]))
    vals = [m[k] for k in keys]
    assert all(a < b for a, b in zip(vals, vals[1:])), vals
    for k in keys:
        r = m[k] / np.sqrt(E[k])
        assert 0.5 < r < 2.0, (k, r)

"""CUDA path against the FP64 oracle, element by element (needs a GB300).

Tolerances:
* float64 path with a shared closed-form table: kernel arithmetic only, 1e-12 relative.
* float64 path with each side's own least-misfit table: the two independently optimised
  tables agree to ~1e-9 (the optimum of E is only determined to that level in float64),
  so results agree to 1e-7 relative RMS.
* float32 path (W = 7): 1e-5 relative RMS on images, grids and predicted visibilities
  (the target accuracy for single precision); on grids every element is also within
  1e-5 of the largest cell.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import design as D  # noqa: E402
from oracle import imaging as I  # noqa: E402
from paper_1906_07102_gb300 import lmg  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402
from tests.cases import (INTERP, caller_table, disk_case, oracle_hvec, oracle_table, rel_rms,  # noqa: E402
                         track_case)

pytestmark = pytest.mark.gpu

DEV = "cuda"


def gpu_plan(W, x0, Ms, interp, n_img, dl, nvis, dtype, values=None):
    tab = lmg.Table(W, x0, Ms, interp, values=values)
    return lmg.Plan(tab, n_img, dl, max(nvis, 1), dtype)


def to_dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def oracle_plan(uv, dl, W, N, single):
    uc = I.cells_from_wavelengths(uv, N, dl)
    return I.Plan(uc[:, 0], uc[:, 1], W, N, single_precision_s=single)


# ----------------------------------------------------------------------------------------
# float64, config-1 sizes: 256^2 image, x0 = 0.5, W = 3, 300-entry nearest table, 1e4 vis
# ----------------------------------------------------------------------------------------
N1, n1, W1, M1 = 512, 256, 3, 100


@pytest.fixture(scope="module")
def c1():
    uv, dl = disk_case(10000, N1, seed=0)
    vis = S.complex_normal(10000, 0)
    return uv, dl, vis


def test_fp64_grid_kernel_exact_with_shared_table(c1):
    uv, dl, vis = c1
    T = caller_table(W1, M1)
    p = gpu_plan(W1, 0.5, M1, "nearest", n1, dl, uv.shape[0], "c128", values=T)
    p.bin(to_dev(uv, torch.float64))
    g = p.grid(to_dev(vis, torch.complex128)).cpu().numpy()
    op = oracle_plan(uv, dl, W1, N1, single=False)
    ref = I.grid(op, T, M1, 0, vis)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
    vd = p.degrid(to_dev(ref, torch.complex128)).cpu().numpy()
    vref = I.degrid(op, T, M1, 0, ref)
    assert np.abs(vd - vref).max() <= 1e-12 * np.abs(vref).max()


def test_fp64_dirty_image_and_predict(c1):
    uv, dl, vis = c1
    p = gpu_plan(W1, 0.5, M1, "nearest", n1, dl, uv.shape[0], "c128")
    p.bin(to_dev(uv, torch.float64))
    img = p.dirty_image(to_dev(vis, torch.complex128)).cpu().numpy()
    T = oracle_table(W1, 0.5, M1)
    hv = oracle_hvec(T, M1, "nearest", W1, n1, N1)
    op = oracle_plan(uv, dl, W1, N1, single=False)
    ref = I.dirty_image(op, T, M1, 0, hv, n1, vis)
    assert rel_rms(img, ref) < 1e-7
    model = S.random_image(n1, 3)
    pv = p.predict_vis(to_dev(model, torch.complex128)).cpu().numpy()
    pref = I.predict_vis(op, T, M1, 0, hv, model)
    assert rel_rms(pv, pref) < 1e-7


def test_fp64_dirty_image_within_dft_bound():
    """Brute-force DFT on a 64^2 window: the GPU image obeys the per-pixel bound (Eq. 8)."""
    N, n_img, W, Ms, nvis = 128, 64, 3, 100, 2000
    uv, dl = disk_case(nvis, N, seed=4)
    vis = S.complex_normal(nvis, 4)
    p = gpu_plan(W, 0.5, Ms, "nearest", n_img, dl, nvis, "c128")
    p.bin(to_dev(uv, torch.float64))
    img = p.dirty_image(to_dev(vis, torch.complex128)).cpu().numpy()
    T = oracle_table(W, 0.5, Ms)
    hv = oracle_hvec(T, Ms, "nearest", W, n_img, N)
    x = I.pixel_coords(n_img, N)
    op = oracle_plan(uv, dl, W, N, single=False)
    ref = I.dft_dirty_image(uv[:, 0], uv[:, 1], vis, None, x, x)
    bound = I.image_bound(op, T, Ms, 0, uv[:, 0], uv[:, 1], vis, None, x, x, hv)
    # slack: table/correction differences between the two builds (~1e-9 relative)
    slack = (1e-7 * np.abs(ref).max()) ** 2
    assert np.all(np.abs(img - ref) ** 2 <= bound * (1 + 1e-6) + slack)


def test_fp64_adjoint_identity():
    N, n_img, W, Ms, nvis = 256, 128, 5, 200, 5000
    uv, dl = disk_case(nvis, N, seed=5)
    vis = S.complex_normal(nvis, 5)
    w = np.random.default_rng(5).uniform(0.1, 2.0, nvis)
    model = S.random_image(n_img, 6)
    p = gpu_plan(W, 0.5, Ms, "linear", n_img, dl, nvis, "c128")
    p.bin(to_dev(uv, torch.float64))
    d = p.dirty_image(to_dev(vis, torch.complex128), to_dev(w, torch.float64)).cpu().numpy()
    pv = p.predict_vis(to_dev(model, torch.complex128)).cpu().numpy()
    lhs = np.vdot(d, model)
    rhs = np.vdot(vis, w * pv)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ----------------------------------------------------------------------------------------
# float32, W = 7, linear table at Ms = 1000, x0 = 0.5, Earth-rotation tracks
# ----------------------------------------------------------------------------------------
N2, n2, W2, M2 = 1024, 512, 7, 1000


@pytest.fixture(scope="module")
def c2():
    uv, dl, vis = track_case(n_ant=24, n_times=512, N=N2, seed=1)
    vis64 = vis.astype(np.complex64)
    p = gpu_plan(W2, 0.5, M2, "linear", n2, dl, uv.shape[0], "c64")
    p.bin(to_dev(uv, torch.float64))
    T = oracle_table(W2, 0.5, M2)
    hv = oracle_hvec(T, M2, "linear", W2, n2, N2)
    op = oracle_plan(uv, dl, W2, N2, single=False)
    return uv, dl, vis64, p, T, hv, op


def test_fp32_grid(c2):
    uv, dl, vis, p, T, hv, op = c2
    g = p.grid(to_dev(vis, torch.complex64)).cpu().numpy()
    ref = I.grid(op, T, M2, 1, vis.astype(np.complex128))
    assert rel_rms(g, ref) < 1e-5
    assert np.abs(g - ref).max() < 1e-5 * np.abs(ref).max()


def test_fp32_dirty_image(c2):
    uv, dl, vis, p, T, hv, op = c2
    img = p.dirty_image(to_dev(vis, torch.complex64)).cpu().numpy()
    ref = I.dirty_image(op, T, M2, 1, hv, n2, vis.astype(np.complex128))
    assert rel_rms(img, ref) < 1e-5


def test_fp32_weighted_dirty_image(c2):
    uv, dl, vis, p, T, hv, op = c2
    w = np.random.default_rng(2).uniform(0.0, 3.0, vis.size).astype(np.float32)
    img = p.dirty_image(to_dev(vis, torch.complex64), to_dev(w, torch.float32)).cpu().numpy()
    ref = I.dirty_image(op, T, M2, 1, hv, n2, vis.astype(np.complex128), w.astype(np.float64))
    assert rel_rms(img, ref) < 1e-5


def test_fp32_predict(c2):
    uv, dl, vis, p, T, hv, op = c2
    model = S.gaussian_blob_image(n2, 32, seed=3).astype(np.complex64)
    pv = p.predict_vis(to_dev(model, torch.complex64)).cpu().numpy()
    ref = I.predict_vis(op, T, M2, 1, hv, model.astype(np.complex128))
    assert rel_rms(pv, ref) < 1e-5


def test_fp32_degrid_matches_oracle_on_same_grid(c2):
    uv, dl, vis, p, T, hv, op = c2
    g = S.random_image(N2, 8).astype(np.complex64)
    vd = p.degrid(to_dev(g, torch.complex64)).cpu().numpy()
    ref = I.degrid(op, T, M2, 1, g.astype(np.complex128))
    assert rel_rms(vd, ref) < 1e-5


def test_fp32_fft_and_correction_stages(c2):
    """Each stage on its own: FFT (+i / -i) and crop / pad against numpy."""
    uv, dl, vis, p, T, hv, op = c2
    G = S.random_image(N2, 9).astype(np.complex64)
    gd = to_dev(G, torch.complex64)
    p.fft(gd, "image")
    F = gd.cpu().numpy()
    # index-order FFT: sum_i G[i] e^{+i 2 pi i q / N}
    refF = np.fft.ifft2(G.astype(np.complex128)) * N2 * N2
    assert rel_rms(F, refF) < 1e-5
    img = p.crop_correct(to_dev(refF.astype(np.complex64), torch.complex64)).cpu().numpy()
    ref_img = I.correct_crop(I.fft_image(G.astype(np.complex128)), hv, n2)
    assert rel_rms(img, ref_img) < 1e-5


def _offset_view(x, shape):
    """Copy of x in a buffer one element past a 16-byte boundary (8-byte aligned)."""
    n = int(np.prod(shape))
    buf = torch.empty(n + 1, dtype=x.dtype, device=x.device)
    v = buf[1:].view(*shape)
    v.copy_(x.reshape(shape))
    return v


def test_correction_pair_and_scalar_kernels_agree(c2):
    """Crop, pad and the prediction's kept-row pad on 16-byte aligned complex64 arrays take
    the two-pixel kernels; arrays offset by one element take the one-pixel kernels. Both
    give the same bits."""
    uv, dl, vis, p, T, hv, op = c2
    F = to_dev(S.random_image(N2, 21).astype(np.complex64), torch.complex64)
    img_pair = p.crop_correct(F)
    img_one = p.crop_correct(_offset_view(F, (N2, N2)), out=_offset_view(torch.zeros_like(img_pair), (n2, n2)))
    assert img_one.data_ptr() % 16 == 8 and torch.equal(img_pair, img_one)
    M = to_dev(S.random_image(n2, 22).astype(np.complex64), torch.complex64)
    pad_pair = p.pad_correct(M)
    pad_one = p.pad_correct(_offset_view(M, (n2, n2)), out=_offset_view(torch.zeros_like(pad_pair), (N2, N2)))
    assert torch.equal(pad_pair, pad_one)
    pv_pair = p.predict_vis(M)
    pv_one = p.predict_vis(_offset_view(M, (n2, n2)))
    assert torch.equal(pv_pair, pv_one)


def test_pruned_ffts_match_full_fft_on_the_kept_field(c2):
    """lmg_fft_pruned: equal to the full transform at the kept rows and columns (imaging),
    and on a padded model grid (prediction)."""
    uv, dl, vis, p, T, hv, op = c2
    q = (np.arange(n2) - n2 // 2) % N2
    G = to_dev(S.random_image(N2, 11).astype(np.complex64), torch.complex64)
    full = p.fft(G.clone(), "image").cpu().numpy()[np.ix_(q, q)]
    pruned = p.fft(G.clone(), "image", pruned=True).cpu().numpy()[np.ix_(q, q)]
    assert rel_rms(pruned, full) < 1e-6
    M = torch.zeros((N2, N2), dtype=torch.complex64, device=DEV)
    M[np.ix_(q, q)] = to_dev(S.random_image(n2, 12).astype(np.complex64), torch.complex64)
    full = p.fft(M.clone(), "model").cpu().numpy()
    pruned = p.fft(M.clone(), "model", pruned=True).cpu().numpy()
    assert rel_rms(pruned, full) < 1e-6


@pytest.mark.parametrize("interp,Ms", [("quadratic", 200), ("cubic", 100)])
def test_fp32_higher_degree_tables(c2, interp, Ms):
    """Quadratic and cubic table interpolation (Appendix F) through the float32 path: dirty
    image and prediction against the oracle with the same degree, table size and own
    least-misfit table, at the float32 target; the correction factors of both sides use
    the same interpolated function."""
    uv, dl, vis, p2, T2, hv2, op = c2
    p = gpu_plan(W2, 0.5, Ms, interp, n2, dl, uv.shape[0], "c64")
    p.bin(to_dev(uv, torch.float64))
    T = oracle_table(W2, 0.5, Ms)
    hv = oracle_hvec(T, Ms, interp, W2, n2, N2)
    img = p.dirty_image(to_dev(vis, torch.complex64)).cpu().numpy()
    ref = I.dirty_image(op, T, Ms, INTERP[interp], hv, n2, vis.astype(np.complex128))
    assert rel_rms(img, ref) < 1e-5
    model = S.gaussian_blob_image(n2, 32, seed=13).astype(np.complex64)
    pv = p.predict_vis(to_dev(model, torch.complex64)).cpu().numpy()
    pref = I.predict_vis(op, T, Ms, INTERP[interp], hv, model.astype(np.complex128))
    assert rel_rms(pv, pref) < 1e-5


# ----------------------------------------------------------------------------------------
# direct calculation (Section 5.2), float64
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("W,tol", [(7, 1e-11), (11, 1e-8)])
def test_direct_calculation_matches_fine_cubic_table(W, tol):
    """Direct per-visibility weights against a finely sampled cubic table of the same design
    (M_s = 20000, interpolation error far below 1e-11). Both solve the normal equations,
    whose matrix A grows ill-conditioned with W (Appendix B): the table row by row with a
    Cholesky solve, the direct route through the folded A^-1. Each carries an error of
    about cond(A) times the float64 epsilon, 1e-9 at W = 11, the largest W for which the
    paper uses the normal equations; hence 1e-11 at W = 7 and 1e-8 at W = 11."""
    N, n_img, nvis = 256, 128, 4000
    uv, dl = disk_case(nvis, N, seed=50 + W)
    vis = S.complex_normal(nvis, 50 + W)
    Gm = S.random_image(N, 60 + W)
    out = {}
    for interp, Ms in (("direct", 4), ("cubic", 20000)):
        p = gpu_plan(W, 0.5, Ms, interp, n_img, dl, nvis, "c128")
        p.bin(to_dev(uv, torch.float64))
        out[interp] = (p.grid(to_dev(vis, torch.complex128)).cpu().numpy(),
                       p.degrid(to_dev(Gm, torch.complex128)).cpu().numpy())
    for k in range(2):
        a, b = out["direct"][k], out["cubic"][k]
        assert np.abs(a - b).max() <= tol * np.abs(b).max()


def test_direct_calculation_against_oracle():
    """Direct calculation end to end against the oracle's exact function (each side with its
    own optimised h, which agree to ~1e-9): dirty image and prediction to 1e-7."""
    N, n_img, W, nvis = 256, 128, 7, 4000
    uv, dl = disk_case(nvis, N, seed=70)
    vis = S.complex_normal(nvis, 70)
    model = S.random_image(n_img, 71)
    p = gpu_plan(W, 0.5, 4, "direct", n_img, dl, nvis, "c128")
    p.bin(to_dev(uv, torch.float64))
    img = p.dirty_image(to_dev(vis, torch.complex128)).cpu().numpy()
    pv = p.predict_vis(to_dev(model, torch.complex128)).cpu().numpy()
    h = D.least_misfit_h(W, 0.25)
    fun = lambda s: D.exact_C(h, W, 0.25, s)
    hv = D.correction_factors(fun, None, None, W, I.pixel_coords(n_img, N))
    op = oracle_plan(uv, dl, W, N, single=False)
    assert rel_rms(img, I.dirty_image(op, fun, None, None, hv, n_img, vis)) < 1e-7
    assert rel_rms(pv, I.predict_vis(op, fun, None, None, hv, model)) < 1e-7


def test_direct_calculation_limits():
    tab = lmg.Table(7, 0.5, 4, "direct")
    with pytest.raises(lmg.LmgError, match="float64"):
        lmg.Plan(tab, 128, 1 / 256, 10, "c64")
    with pytest.raises(lmg.LmgError, match="W <= 11"):
        lmg.Plan(lmg.Table(12, 0.5, 4, "direct"), 128, 1 / 256, 10, "c128")


# ----------------------------------------------------------------------------------------
# edge cases
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("W", [1, 2, 4, 8, 12, 16])
def test_support_widths_fp64_kernel_exact(W):
    N, n_img, Ms, nvis = 96, 48, 64, 777
    uv, dl = disk_case(nvis, N, seed=W)
    vis = S.complex_normal(nvis, W)
    T = caller_table(W, Ms)
    for interp in ("nearest", "linear", "quadratic", "cubic"):
        p = gpu_plan(W, 0.5, Ms, interp, n_img, dl, nvis, "c128", values=T)
        p.bin(to_dev(uv, torch.float64))
        g = p.grid(to_dev(vis, torch.complex128)).cpu().numpy()
        op = oracle_plan(uv, dl, W, N, single=False)
        ref = I.grid(op, T, Ms, INTERP[interp], vis)
        assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max(), interp
        Gm = S.random_image(N, W + 1)
        vd = p.degrid(to_dev(Gm, torch.complex128)).cpu().numpy()
        vref = I.degrid(op, T, Ms, INTERP[interp], Gm)
        assert np.abs(vd - vref).max() <= 1e-12 * np.abs(vref).max(), interp


@pytest.mark.parametrize("W", list(range(1, 17)))
def test_support_widths_fp32_two_columns_per_lane(W):
    """complex64 lanes own two columns of 64-column strips, and the slots a record fills
    depend on W and on the parity of its start column: every W = 1..16 with every lookup,
    against the float64 oracle on the same closed-form table, per element within 1e-5 of the
    largest value (the float32 target)."""
    N, n_img, Ms, nvis = 128, 64, 64, 1500
    uv, dl = disk_case(nvis, N, seed=100 + W)
    vis = S.complex_normal(nvis, 100 + W)
    T = caller_table(W, Ms)
    op = oracle_plan(uv, dl, W, N, single=False)
    Gm = S.random_image(N, 200 + W)
    for interp in ("nearest", "linear", "quadratic", "cubic"):
        p = gpu_plan(W, 0.5, Ms, interp, n_img, dl, nvis, "c64", values=T)
        p.bin(to_dev(uv, torch.float64))
        g = p.grid(to_dev(vis.astype(np.complex64), torch.complex64)).cpu().numpy()
        ref = I.grid(op, T, Ms, INTERP[interp], vis.astype(np.complex64).astype(np.complex128))
        assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max(), interp
        vd = p.degrid(to_dev(Gm.astype(np.complex64), torch.complex64)).cpu().numpy()
        vref = I.degrid(op, T, Ms, INTERP[interp], Gm.astype(np.complex64).astype(np.complex128))
        assert np.abs(vd - vref).max() <= 1e-5 * np.abs(vref).max(), interp


@pytest.mark.parametrize("nvis", [0, 1, 33, 4097])
def test_ragged_counts_fp32(nvis):
    N, n_img, W, Ms = 128, 64, 7, 100
    uv, dl = disk_case(max(nvis, 1), N, seed=300 + nvis)
    uv = uv[:nvis].reshape(-1, 2)
    vis = S.complex_normal(nvis, 300 + nvis).astype(np.complex64)
    T = caller_table(W, Ms)
    p = gpu_plan(W, 0.5, Ms, "linear", n_img, dl, max(nvis, 1), "c64", values=T)
    p.bin(to_dev(uv, torch.float64))
    g = p.grid(to_dev(vis, torch.complex64)).cpu().numpy()
    ref = I.grid(oracle_plan(uv, dl, W, N, single=False), T, Ms, 1, vis.astype(np.complex128))
    if nvis == 0:
        assert not np.any(g)
    else:
        assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("nvis", [0, 1, 31, 33, 4097])
def test_ragged_counts(nvis):
    N, n_img, W, Ms = 128, 64, 7, 100
    uv, dl = disk_case(max(nvis, 1), N, seed=nvis)
    uv = uv[:nvis]
    vis = S.complex_normal(nvis, nvis)
    T = caller_table(W, Ms)
    p = gpu_plan(W, 0.5, Ms, "linear", n_img, dl, max(nvis, 1), "c128", values=T)
    p.bin(to_dev(uv.reshape(-1, 2), torch.float64))
    g = p.grid(to_dev(vis, torch.complex128)).cpu().numpy()
    op = oracle_plan(uv.reshape(-1, 2), dl, W, N, single=False)
    ref = I.grid(op, T, Ms, 1, vis)
    assert np.abs(g - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1.0)
    Gm = S.random_image(N, 3)
    vd = p.degrid(to_dev(Gm, torch.complex128)).cpu().numpy()
    assert vd.shape == (nvis,)
    if nvis:
        vref = I.degrid(op, T, Ms, 1, Gm)
        assert np.abs(vd - vref).max() <= 1e-12 * np.abs(vref).max()


def test_dense_single_cell_and_edges():
    """Thousands of positions in one cell (many 32-record batches in one bucket, one work
    item per row), supports wrapping around all four grid edges, and a non-power-of-two
    grid (N = 160)."""
    N, n_img, W, Ms = 160, 80, 7, 200
    g = np.random.default_rng(11)
    dense = np.stack([3.3 + 0.01 * g.random(5000), -7.2 + 0.01 * g.random(5000)], 1)
    edge = np.array([[N / 2 - 1.2, 0.3], [-N / 2 + 0.2, 5.0], [4.0, N / 2 - 0.6], [-3.0, -N / 2 + 1.9],
                     [N / 2 - 2.5, -N / 2 + 0.4], [-N / 2 + 0.01, N / 2 - 0.01]])
    uv = np.concatenate([dense, edge, S.disk_uniform(3000, 0.5 * N, 12)])
    vis = S.complex_normal(uv.shape[0], 13)
    T = caller_table(W, Ms)
    p = gpu_plan(W, 0.5, Ms, "linear", n_img, 1.0 / N, uv.shape[0], "c128", values=T)
    p.bin(to_dev(uv, torch.float64))
    gg = p.grid(to_dev(vis, torch.complex128)).cpu().numpy()
    op = oracle_plan(uv, 1.0 / N, W, N, single=False)
    ref = I.grid(op, T, Ms, 1, vis)
    assert np.abs(gg - ref).max() <= 1e-12 * np.abs(ref).max()
    Gm = S.random_image(N, 14)
    vd = p.degrid(to_dev(Gm, torch.complex128)).cpu().numpy()
    vref = I.degrid(op, T, Ms, 1, Gm)
    assert np.abs(vd - vref).max() <= 1e-12 * np.abs(vref).max()


def test_dropped_positions():
    N, n_img, W, Ms = 128, 64, 5, 100
    uv, dl = disk_case(300, N, seed=21)
    uv[[3, 50, 299]] = [[np.nan, 1.0], [1e40, 0.0], [0.0, -np.inf]]
    vis = S.complex_normal(300, 21)
    T = caller_table(W, Ms)
    p = gpu_plan(W, 0.5, Ms, "linear", n_img, dl, 300, "c128", values=T)
    p.bin(to_dev(uv, torch.float64))
    assert p.dropped() == 3
    gg = p.grid(to_dev(vis, torch.complex128)).cpu().numpy()
    op = oracle_plan(uv, dl, W, N, single=False)
    ref = I.grid(op, T, Ms, 1, vis)
    assert np.abs(gg - ref).max() <= 1e-12 * np.abs(ref).max()
    vd = p.degrid(to_dev(S.random_image(N, 2), torch.complex128)).cpu().numpy()
    assert np.all(vd[[3, 50, 299]] == 0)


def test_rebinning_reuses_plan():
    N, n_img, W, Ms = 128, 64, 7, 100
    T = caller_table(W, Ms)
    p = gpu_plan(W, 0.5, Ms, "linear", n_img, 1.0 / N, 5000, "c128", values=T)
    for seed, nv in ((1, 5000), (2, 1234), (3, 4999)):
        uv, dl = disk_case(nv, N, seed=seed)
        vis = S.complex_normal(nv, seed)
        p.bin(to_dev(uv, torch.float64))
        gg = p.grid(to_dev(vis, torch.complex128)).cpu().numpy()
        ref = I.grid(oracle_plan(uv, dl, W, N, single=False), T, Ms, 1, vis)
        assert np.abs(gg - ref).max() <= 1e-12 * np.abs(ref).max()


def test_compensated_accumulation_not_worse():
    """Dense float32 gridding: the compensated sweep is at least as close to the float64
    oracle as the plain one."""
    N, n_img, W, Ms = 256, 128, 12, 200
    g = np.random.default_rng(31)
    uv = np.concatenate([g.normal(0, 3.0, (200000, 2)), S.disk_uniform(20000, 0.45 * N, 31)])
    vis = S.complex_normal(uv.shape[0], 31)
    T = caller_table(W, Ms)
    p = gpu_plan(W, 0.5, Ms, "linear", n_img, 1.0 / N, uv.shape[0], "c64", values=T)
    p.bin(to_dev(uv, torch.float64))
    vd = to_dev(vis, torch.complex64)
    plain = p.grid(vd).cpu().numpy()
    comp = p.grid(vd, accum="compensated").cpu().numpy()
    ref = I.grid(oracle_plan(uv, 1.0 / N, W, N, single=False), T, Ms, 1, vis.astype(np.complex64).astype(np.complex128))
    e_plain, e_comp = rel_rms(plain, ref), rel_rms(comp, ref)
    assert e_comp <= e_plain * 1.01
    assert e_comp < 1e-6

"""Fused kept-field transforms (lmg_image_from_grid, lmg_grid_from_image) on a 4096^2 grid
against the oracle's transforms and against the library-transform path (needs a GB300).

The correction factors are the plan's own (float32 rounding of the float64 factors of the
float32 table, as lmg_correction_export gives them), so that the comparisons isolate the
transforms (Eq. 4, the correction and crop of Eq. 15, and their adjoint for Eq. 2). Float32
transforms of 4096 points carry rounding of order 1e-7 relative; the bars are 2e-6 in
relative RMS and 1e-5 of the largest value per element.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import imaging as I  # noqa: E402
from paper_1906_07102_gb300 import lmg  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402
from tests.cases import oracle_hvec, oracle_table, rel_rms  # noqa: E402

pytestmark = pytest.mark.gpu

N, n = 4096, 2048


def close(out, ref, rms=2e-6):
    assert rel_rms(out, ref) < rms
    assert np.abs(out - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.fixture(scope="module")
def plan():
    tab = lmg.Table(7, 0.5, 1000, "linear")
    p = lmg.Plan(tab, n, 1.0 / N, 1, "c64")
    hv = np.float32(tab.correction(n, single_precision=True)).astype(np.float64)
    return p, hv


def test_fused_path_is_taken_for_4096(plan):
    p, _ = plan
    assert p.transform_scratch_bytes() == N * n * 8


def test_image_from_grid_against_oracle(plan):
    p, hv = plan
    G = S.random_image(N, 1).astype(np.complex64)
    Gd = torch.from_numpy(G).cuda()
    img = p.image_from_grid(Gd).cpu().numpy()
    ref = I.correct_crop(I.fft_image(G.astype(np.complex128)), hv, n)
    close(img, ref)
    assert torch.equal(Gd.cpu(), torch.from_numpy(G))      # the grid is left as it was


def test_grid_from_image_against_oracle(plan):
    p, hv = plan
    M = S.random_image(n, 2).astype(np.complex64)
    g = p.grid_from_image(torch.from_numpy(M).cuda()).cpu().numpy()
    ref = I.model_grid(I.pad_correct(M.astype(np.complex128), hv, N))
    close(g, ref)


def test_fused_and_library_paths_agree(plan):
    """lmg_image_from_grid against lmg_fft_pruned + lmg_grid_correct (LMG_CROP), and
    lmg_grid_from_image against lmg_grid_correct (LMG_PAD) + lmg_fft_pruned."""
    p, _ = plan
    G = torch.from_numpy(S.random_image(N, 3).astype(np.complex64)).cuda()
    fused = p.image_from_grid(G).cpu().numpy()
    lib = p.crop_correct(p.fft(G.clone(), "image", pruned=True)).cpu().numpy()
    close(fused, lib)
    M = torch.from_numpy(S.gaussian_blob_image(n, 32, seed=4).astype(np.complex64)).cuda()
    fused = p.grid_from_image(M).cpu().numpy()
    lib = p.fft(p.pad_correct(M), "model", pruned=True).cpu().numpy()
    close(fused, lib)


def test_caller_scratch_gives_the_same_bits(plan):
    p, _ = plan
    G = torch.from_numpy(S.random_image(N, 5).astype(np.complex64)).cuda()
    M = torch.from_numpy(S.random_image(n, 6).astype(np.complex64)).cuda()
    scratch = torch.empty(p.transform_scratch_bytes() // 8, dtype=torch.complex64, device="cuda")
    assert torch.equal(p.image_from_grid(G), p.image_from_grid(G, scratch=scratch))
    assert torch.equal(p.grid_from_image(M), p.grid_from_image(M, scratch=scratch))


def test_plan_without_work_grids_needs_a_scratch():
    tab = lmg.Table(7, 0.5, 1000, "linear")
    p = lmg.Plan(tab, n, 1.0 / N, 1, "c64", work_grids=False)
    G = torch.from_numpy(S.random_image(N, 7).astype(np.complex64)).cuda()
    with pytest.raises(lmg.LmgError, match="transform scratch"):
        p.image_from_grid(G)
    scratch = torch.empty(p.transform_scratch_bytes() // 8, dtype=torch.complex64, device="cuda")
    q = lmg.Plan(tab, n, 1.0 / N, 1, "c64")
    assert torch.equal(p.image_from_grid(G, scratch=scratch), q.image_from_grid(G))


def test_other_sizes_use_the_library_transforms():
    """N = 1024 (and complex128 at 4096) take the pruned library transforms: no scratch, and
    the image equals the library path's (the grid is transformed in place)."""
    for N1, n1, dt in ((1024, 512, "c64"), (4096, 2048, "c128")):
        tab = lmg.Table(5, 0.5, 200, "linear")
        p = lmg.Plan(tab, n1, 1.0 / N1, 1, dt)
        assert p.transform_scratch_bytes() == 0
        cd = torch.complex64 if dt == "c64" else torch.complex128
        G = torch.from_numpy(S.random_image(N1, 8)).to("cuda", cd)
        ref = p.crop_correct(p.fft(G.clone(), "image", pruned=True))
        assert torch.equal(p.image_from_grid(G.clone()), ref)


def test_dirty_image_and_prediction_through_the_fused_path():
    """lmg_dirty_image and lmg_predict_vis of a complex64 4096^2 plan (fused transforms)
    against the oracle's dirty image and prediction, on 20,000 disk positions."""
    W, Ms, nv = 7, 1000, 20000
    uv = S.disk_uniform(nv, 0.45 * N, seed=9)
    vis = S.complex_normal(nv, 9)
    model = S.gaussian_blob_image(n, 32, seed=10)
    tab = lmg.Table(W, 0.5, Ms, "linear")
    p = lmg.Plan(tab, n, 1.0 / N, nv, "c64")
    p.bin(torch.from_numpy(uv).cuda())
    img = p.dirty_image(torch.from_numpy(vis.astype(np.complex64)).cuda()).cpu().numpy()
    pv = p.predict_vis(torch.from_numpy(model.astype(np.complex64)).cuda()).cpu().numpy()
    T = oracle_table(W, 0.5, Ms)
    hv = oracle_hvec(T, Ms, "linear", W, n, N)
    op = I.Plan(uv[:, 0], uv[:, 1], W, N)
    assert rel_rms(img, I.dirty_image(op, T, Ms, 1, hv, n, vis)) < 1e-5
    assert rel_rms(pv, I.predict_vis(op, T, Ms, 1, hv, model)) < 1e-5

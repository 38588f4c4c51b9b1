"""lmg_grid_static: gridding for callers that cannot allocate device memory (needs a GB300).

Some callers cannot call cudaMalloc (their device memory belongs to another allocator, or
is reserved at start-up and must not grow while a real-time pipeline runs). For them the
library offers lmg_grid_static, which bins and grids with all working memory in a fixed
array inside the library. This file checks, through the C ABI, that it gives the same grid
as the allocating path (lmg_plan_bin + lmg_grid) on two calls in a row, and that sizes
beyond its stated limits are refused. It is named to run after every other test file.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1906_07102_gb300 import lmg  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402

pytestmark = pytest.mark.gpu


def _inputs(seed, nvis, N):
    uv = S.disk_uniform(nvis, 0.45 * N, seed)
    vis = S.complex_normal(nvis, seed).astype(np.complex64)
    w = np.random.default_rng(seed).uniform(0.5, 2.0, nvis).astype(np.float32)
    return (torch.from_numpy(uv).cuda(), torch.from_numpy(vis).cuda(), torch.from_numpy(w).cuda())


def test_static_grid_matches_allocating_path_twice():
    N, n_img, W, Ms = 1024, 512, 7, 1000
    tab = lmg.Table(W, 0.5, Ms, "linear")
    plan = lmg.Plan(tab, n_img, 1.0 / N, 200000, "c64")
    for seed, nvis, weighted in ((1, 200000, False), (2, 123457, True)):
        uv, vis, w = _inputs(seed, nvis, N)
        wt = w if weighted else None
        ref = plan.bin(uv).grid(vis, wt).cpu().numpy()
        out = lmg.grid_static(tab, n_img, 1.0 / N, uv, vis, wt).cpu().numpy()
        scale = np.abs(ref).max()
        # same kernels; only the order of float32 sums inside a bucket may differ
        assert np.abs(out - ref).max() <= 1e-5 * scale
        assert np.sqrt(np.mean(np.abs(out - ref) ** 2)) <= 1e-6 * np.sqrt(np.mean(np.abs(ref) ** 2))


def test_static_grid_rejects_sizes_beyond_its_limits():
    tab = lmg.Table(7, 0.5, 1000, "linear")
    uv, vis, _ = _inputs(3, 1000, 1024)
    with pytest.raises(lmg.LmgError, match="lmg_grid_static"):
        lmg.grid_static(tab, 2 * lmg.STATIC_MAX_N, 1.0 / (4 * lmg.STATIC_MAX_N), uv, vis)
    big = lmg.STATIC_MAX_VIS + 1
    uvb = torch.zeros((big, 2), dtype=torch.float64, device="cuda")
    visb = torch.zeros(big, dtype=torch.complex64, device="cuda")
    with pytest.raises(lmg.LmgError, match="lmg_grid_static"):
        lmg.grid_static(tab, 512, 1.0 / 1024, uvb, visb)
    fine = lmg.Table(7, 0.5, 8192, "linear")
    with pytest.raises(lmg.LmgError, match="lmg_grid_static"):
        lmg.grid_static(fine, 512, 1.0 / 1024, uv, vis)


def test_static_grid_allocates_no_device_memory():
    """After a first call has set the device up, further calls leave the device's free
    memory exactly where it was: the entry point's whole purpose."""
    N, n_img = 1024, 512
    tab = lmg.Table(7, 0.5, 1000, "linear")
    uv, vis, w = _inputs(6, 50000, N)
    out = torch.empty((N, N), dtype=torch.complex64, device="cuda")
    lmg.grid_static(tab, n_img, 1.0 / N, uv, vis, w, out=out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        lmg.grid_static(tab, n_img, 1.0 / N, uv, vis, w, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


@pytest.mark.parametrize("W,Ms,interp,N,nvis", [(7, 100, "cubic", 1024, 60000), (6, 200, "quadratic", 512, 30000),
                                                (16, 1000, "linear", lmg.STATIC_MAX_N, lmg.STATIC_MAX_VIS),
                                                (7, 1000, "linear", 1024, 0)])
def test_static_grid_other_lookups_sizes_and_empty_input(W, Ms, interp, N, nvis):
    """The extended-lookup sweeps (quadratic, cubic), the sized maxima (W = 16, N and nvis at
    their limits) and an empty input, each against the allocating path."""
    n_img = N // 2
    tab = lmg.Table(W, 0.5, Ms, interp)
    plan = lmg.Plan(tab, n_img, 1.0 / N, max(nvis, 1), "c64")
    uv, vis, w = _inputs(7 + W, nvis, N)
    ref = plan.bin(uv).grid(vis, w).cpu().numpy()
    out = lmg.grid_static(tab, n_img, 1.0 / N, uv, vis, w).cpu().numpy()
    if nvis == 0:
        assert not np.any(out) and not np.any(ref)
        return
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() <= 1e-5 * scale
    assert np.sqrt(np.mean(np.abs(out - ref) ** 2)) <= 1e-6 * np.sqrt(np.mean(np.abs(ref) ** 2))

"""Multi-channel batches (lmg.Batch, the lmg_batch_* C ABI) against the single-plan path and
the FP64 oracle (needs a GB300).

The channels differ in support width (W = 4, 6, 8 and 11, so that several persistent
launches share one graph), grid size (256^2 .. 1024^2), visibility count (0 to 60,000,
ragged) and weighting. A batch runs the same per-item sweep code as a single plan; only
the order of float32 sums inside one bucket may differ (record ranks come from atomic
counters), so grids and degridded visibilities agree per element within 1e-5 of the
largest value and 1e-6 in relative RMS. Dirty images and predictions also pass through
FFTs: the batch prunes them per grid size to the widest kept field among the channels of
that size (one channel here keeps a quarter of its grid beside channels that keep half),
a single plan to its own, so those agree to the float32 target, 1e-5. One channel is also
checked against the oracle at 1e-5.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import imaging as I  # noqa: E402
from paper_1906_07102_gb300 import lmg  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402
from tests.cases import oracle_hvec, oracle_table, rel_rms  # noqa: E402

pytestmark = pytest.mark.gpu

# (W, N, nvis, weighted, x0): x0 is the kept fraction, n_image = x0 N
CHANNELS = [(4, 512, 20000, False, 0.5), (6, 256, 3001, True, 0.5), (8, 1024, 60000, False, 0.5),
            (4, 1024, 0, False, 0.5), (11, 512, 15000, True, 0.5), (6, 512, 1, False, 0.5),
            (8, 256, 40000, True, 0.5), (4, 256, 777, False, 0.5), (6, 512, 5000, False, 0.25)]
MS = 1000


def close(out, ref, rms=1e-6):
    scale = max(np.abs(ref).max(), 1e-30)
    assert np.abs(out - ref).max() <= 1e-5 * scale
    if np.abs(ref).max() > 0:
        assert rel_rms(out, ref) <= rms


@pytest.fixture(scope="module")
def setup():
    tabs = {(W, x0): lmg.Table(W, x0, MS, "linear") for W, x0 in sorted({(c[0], c[4]) for c in CHANNELS})}
    uvs, viss, wts, plans = [], [], [], []
    for i, (W, N, nv, weighted, x0) in enumerate(CHANNELS):
        uv = S.disk_uniform(nv, 0.45 * N, seed=100 + i)
        vis = S.complex_normal(nv, seed=100 + i).astype(np.complex64)
        w = np.random.default_rng(100 + i).uniform(0.5, 2.0, nv).astype(np.float32) if weighted else None
        uvs.append(torch.from_numpy(uv).cuda())
        viss.append(torch.from_numpy(vis).cuda())
        wts.append(torch.from_numpy(w).cuda() if w is not None else None)
        p = lmg.Plan(tabs[(W, x0)], int(N * x0), 1.0 / N, max(nv, 1), "c64")
        p.bin(uvs[-1])
        plans.append(p)
    batch = lmg.Batch([tabs[(c[0], c[4])] for c in CHANNELS], [int(c[1] * c[4]) for c in CHANNELS],
                      [1.0 / c[1] for c in CHANNELS], [max(c[2], 1) for c in CHANNELS])
    batch.bin(uvs)
    return tabs, uvs, viss, wts, plans, batch


def test_batch_layout(setup):
    *_, batch = setup
    info = batch.info()
    assert info["channels"] == len(CHANNELS)
    assert info["w_classes"] == 4 and info["size_classes"] == 3
    assert info["nvis"] == sum(c[2] for c in CHANNELS)


def test_batch_grid_matches_single_plans(setup):
    tabs, uvs, viss, wts, plans, batch = setup
    out = batch.grid(viss, wts)
    for c, p in enumerate(plans):
        ref = p.grid(viss[c], wts[c]).cpu().numpy()
        close(out[c].cpu().numpy(), ref)
    assert not out[3].abs().any()          # the empty channel's grid is all zero


def test_batch_degrid_matches_single_plans(setup):
    tabs, uvs, viss, wts, plans, batch = setup
    grids = [torch.from_numpy(S.random_image(c[1], 30 + i).astype(np.complex64)).cuda()
             for i, c in enumerate(CHANNELS)]
    out = batch.degrid(grids)
    for c, p in enumerate(plans):
        if CHANNELS[c][2] == 0:
            continue
        ref = p.degrid(grids[c]).cpu().numpy()
        close(out[c].cpu().numpy(), ref)


def test_batch_dirty_image_and_predict(setup):
    tabs, uvs, viss, wts, plans, batch = setup
    imgs = batch.dirty_image(viss, wts)
    models = [torch.from_numpy(S.gaussian_blob_image(int(c[1] * c[4]), 16, seed=40 + i).astype(np.complex64)).cuda()
              for i, c in enumerate(CHANNELS)]
    pred = batch.predict_vis(models)
    for c, p in enumerate(plans):
        close(imgs[c].cpu().numpy(), p.dirty_image(viss[c], wts[c]).cpu().numpy(), rms=1e-5)
        if CHANNELS[c][2]:
            close(pred[c].cpu().numpy(), p.predict_vis(models[c]).cpu().numpy(), rms=1e-5)


@pytest.mark.parametrize("c", [2, 8])
def test_batch_channel_against_oracle(setup, c):
    """Channel 2 (1024^2, half kept) and channel 8 (512^2, a quarter kept, transformed with the
    wider pruning of its size class) against the oracle's dirty image."""
    tabs, uvs, viss, wts, plans, batch = setup
    W, N, nv, weighted, x0 = CHANNELS[c]
    n = int(N * x0)
    img = batch.dirty_image(viss, wts)[c].cpu().numpy()
    T = oracle_table(W, x0, MS)
    hv = oracle_hvec(T, MS, "linear", W, n, N)
    uc = I.cells_from_wavelengths(uvs[c].cpu().numpy(), N, 1.0 / N)
    op = I.Plan(uc[:, 0], uc[:, 1], W, N, single_precision_s=False)
    w = wts[c].cpu().numpy().astype(np.float64) if weighted else None
    ref = I.dirty_image(op, T, MS, 1, hv, n, viss[c].cpu().numpy().astype(np.complex128), w)
    assert rel_rms(img, ref) < 1e-5


def test_graph_is_replayed_for_the_same_buffers(setup):
    tabs, uvs, viss, wts, plans, batch = setup
    outs = [torch.empty((c[1], c[1]), dtype=torch.complex64, device="cuda") for c in CHANNELS]
    batch.grid(viss, wts, out=outs)
    n0 = batch.info()["graphs_captured"]
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(1.0)
    batch.grid(viss, wts, out=outs)
    assert batch.info()["graphs_captured"] == n0      # replayed, not captured again
    for a, b in zip(first, outs):
        close(b.cpu().numpy(), a.cpu().numpy())
    other = [torch.empty_like(o) for o in outs]
    batch.grid(viss, wts, out=other)
    assert batch.info()["graphs_captured"] == n0 + 1  # new buffers: captured again
    for a, b in zip(first, other):
        close(b.cpu().numpy(), a.cpu().numpy())


def test_tuner_choice_is_valid_and_results_unchanged(setup):
    tabs, uvs, viss, wts, plans, batch = setup
    chosen = batch.tune(viss)
    assert chosen[0] in (64, 128, 256, 512) and chosen[1] in (256, 512, 1024, 2048)
    assert chosen[2] in (4, 8) and chosen[3] in (0, 1)
    info = batch.info()
    assert (info["rows_per_bin"], info["records_per_item"], info["warps"]) == chosen[:3]
    out = batch.grid(viss, wts)
    for c, p in enumerate(plans):
        close(out[c].cpu().numpy(), p.grid(viss[c], wts[c]).cpu().numpy())


def test_batch_errors():
    tab = lmg.Table(4, 0.5, 100, "linear")
    b = lmg.Batch([tab, tab], [128, 256], [1 / 256, 1 / 512], [10, 10])
    grids = [torch.zeros((256, 256), dtype=torch.complex64, device="cuda"),
             torch.zeros((512, 512), dtype=torch.complex64, device="cuda")]
    arr = ctypes.cast(lmg._ptr_array(grids), ctypes.c_void_p)
    with pytest.raises(lmg.LmgError, match="lmg_batch_bin first"):
        lmg._check(lmg.lib().lmg_batch_degrid(b._h, arr, arr, None))
    uv_big = torch.zeros((11, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(lmg.LmgError, match="max_vis"):
        b.bin([uv_big, uv_big])
    with pytest.raises(lmg.LmgError, match="channel 1"):
        lmg.Batch([tab, tab], [128, 100], [1 / 256, 1 / 200], [10, 10])

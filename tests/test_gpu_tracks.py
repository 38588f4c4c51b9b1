"""Track-ordered binning (lmg_plan_bin_tracks) against the plain binning and the oracle
(needs a GB300).

The tracks hint only changes how the binning passes walk the positions (one thread per
track over 32 consecutive samples, one bucket update per run of samples in one bucket);
the records, and so every grid cell and predicted visibility, are the same sums in another
order. Cases cover a hint that matches the layout, hints that do not (1, 7, more than nvis),
a last partial row of samples, sample counts that end inside a 32-sample chunk, and dropped
positions inside a track (they end a run).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import imaging as I  # noqa: E402
from paper_1906_07102_gb300 import lmg  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402
from tests.cases import caller_table, oracle_hvec, oracle_table, rel_rms  # noqa: E402

pytestmark = pytest.mark.gpu

N, n_img = 512, 256
N_ANT, N_TIMES = 24, 100          # 276 tracks, 100 samples: the last chunk holds 4
N_BL = N_ANT * (N_ANT - 1) // 2


def positions(cut=37, drop=True):
    uv = S.array_tracks(n_ant=N_ANT, n_times=N_TIMES, seed=5)
    uv = uv[:uv.shape[0] - cut]                                      # last row partial
    dl = S.pixel_scale_for(uv)
    if drop:
        uv = uv.copy()
        # dropped positions in the middle of tracks 3 and 100 (samples 40 and 41)
        uv[40 * N_BL + 3] = [np.nan, 0.0]
        uv[41 * N_BL + 100] = [1e40, 1.0]
    return uv, dl


def plans(uv, dl, dtype, W=7, Ms=1000, values=None):
    tab = lmg.Table(W, 0.5, Ms, "linear", values=values)
    return [lmg.Plan(tab, n_img, dl, uv.shape[0], dtype) for _ in range(2)]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("tracks", [N_BL, 1, 7, 10 ** 6])
def test_track_binning_matches_plain_binning(dtype, tracks):
    uv, dl = positions()
    nv = uv.shape[0]
    cd = torch.complex64 if dtype == "c64" else torch.complex128
    vis = torch.from_numpy(S.complex_normal(nv, 3)).to("cuda", cd)
    G = torch.from_numpy(S.random_image(N, 4)).to("cuda", cd)
    a, b = plans(uv, dl, dtype)
    uvd = torch.from_numpy(uv).cuda()
    a.bin(uvd)
    b.bin(uvd, tracks=tracks)
    assert a.dropped() == b.dropped() == 2
    ga, gb = a.grid(vis).cpu().numpy(), b.grid(vis).cpu().numpy()
    va, vb = a.degrid(G).cpu().numpy(), b.degrid(G).cpu().numpy()
    tol = 1e-6 if dtype == "c64" else 1e-13
    assert np.abs(ga - gb).max() <= tol * np.abs(ga).max()
    assert np.abs(va - vb).max() <= tol * np.abs(va).max()
    assert np.all(vb[[40 * N_BL + 3, 41 * N_BL + 100]] == 0)


def test_track_binning_float64_against_oracle():
    """Float64 kernels with a shared closed-form table after track binning: every grid cell
    and prediction within 1e-12 of the oracle (the plain binning's bar)."""
    uv, dl = positions()
    nv = uv.shape[0]
    W, Ms = 6, 400
    T = caller_table(W, Ms)
    p = plans(uv, dl, "c128", W, Ms, values=T)[0]
    p.bin(torch.from_numpy(uv).cuda(), tracks=N_BL)
    vis = S.complex_normal(nv, 8)
    uc = I.cells_from_wavelengths(uv, N, dl)
    op = I.Plan(uc[:, 0], uc[:, 1], W, N)
    g = p.grid(torch.from_numpy(vis).cuda()).cpu().numpy()
    ref = I.grid(op, T, Ms, 1, vis)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
    Gm = S.random_image(N, 9)
    v = p.degrid(torch.from_numpy(Gm).cuda()).cpu().numpy()
    vref = I.degrid(op, T, Ms, 1, Gm)
    assert np.abs(v - vref).max() <= 1e-12 * np.abs(vref).max()


def test_track_binning_float32_dirty_image_against_oracle():
    uv, dl = positions(cut=0, drop=False)
    nv = uv.shape[0]
    p = plans(uv, dl, "c64")[0]
    p.bin(torch.from_numpy(uv).cuda(), tracks=N_BL)
    vis = S.complex_normal(nv, 10)
    img = p.dirty_image(torch.from_numpy(vis.astype(np.complex64)).cuda()).cpu().numpy()
    T = oracle_table(7, 0.5, 1000)
    hv = oracle_hvec(T, 1000, "linear", 7, n_img, N)
    uc = I.cells_from_wavelengths(uv, N, dl)
    op = I.Plan(uc[:, 0], uc[:, 1], 7, N)
    ref = I.dirty_image(op, T, 1000, 1, hv, n_img, vis)
    assert rel_rms(img, ref) < 1e-5


def test_track_binning_rejects_bad_hint():
    uv, dl = positions()
    p = plans(uv, dl, "c64")[0]
    with pytest.raises(lmg.LmgError, match="tracks"):
        p.bin(torch.from_numpy(uv).cuda(), tracks=0)

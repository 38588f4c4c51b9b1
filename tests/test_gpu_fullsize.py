"""Float32 path at the full tracks workload, element by element against the FP64 oracle
(needs a GB300).

Workload: 64 antennas, 6 h of Earth rotation in 2048 samples at 1.4 GHz (4,128,768
visibilities), 4096^2 grid, 2048^2 image, W = 7, linear table with M_s = 1000, complex64;
the visibilities are seeded complex normals (their values do not change which cells or
records the kernels touch). The library grids and degrids every visibility in the same
launch configuration the benchmark times (positions binned in track order, as stored:
sample-major over the 2016 baselines); the oracle recomputes only what it can afford:

* gridding (Eqs. 5-6): every cell of a 64-column band of the grid, from the visibilities
  whose support can reach the band (the oracle's own support rule selects them; others
  add nothing there). Bands: the one with the most supports (it holds the densest
  (strip, row pair) buckets of several hundred records), the same band shifted by 32
  columns (it straddles two strips, so cells are summed by two strip owners and the spill
  pass) and the outermost occupied band (sparse records, ragged rows).
* degridding (Section 4) of a seeded random grid: the visibilities of the densest band
  whose support starts in its 16 densest rows, and 20,000 random ones.

Bars as for the float32 parity tests at reduced size: relative RMS below 1e-5 and every
element within 1e-5 of the largest reference magnitude.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import imaging as I  # noqa: E402
from paper_1906_07102_gb300 import lmg  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402
from tests.cases import oracle_table, rel_rms  # noqa: E402

pytestmark = pytest.mark.gpu

N, n_img, W, MS = 4096, 2048, 7, 1000
BAND = 64
N_TRACKS = 64 * 63 // 2       # baselines; positions are stored sample-major


@pytest.fixture(scope="module")
def full():
    uv = S.array_tracks(n_ant=64, hours=6.0, n_times=2048, freqs_hz=(1.4e9,), seed=0)
    dl = S.pixel_scale_for(uv)
    nv = uv.shape[0]
    tab = lmg.Table(W, 0.5, MS, "linear")
    p = lmg.Plan(tab, n_img, dl, nv, "c64")
    p.bin(torch.from_numpy(uv).cuda(), tracks=N_TRACKS)   # as the benchmark bins them
    uc = I.cells_from_wavelengths(uv, N, dl)
    n0, _, vu = I.support_rule(uc[:, 0], W)
    m0, _, vv = I.support_rule(uc[:, 1], W)
    assert (vu & vv).all()
    # grid column / row of the first support cell (i = n + N/2)
    c0, r0 = n0 + N // 2, m0 + N // 2
    return dict(uv=uv, dl=dl, nv=nv, p=p, uc=uc, c0=c0, r0=r0, T=oracle_table(W, 0.5, MS), tab=tab)


def supports_per_band(c0, shift=0):
    """Visibilities whose W support columns reach each band [shift + 64 b, shift + 64 b + 64)."""
    counts = np.zeros(N // BAND + 1, dtype=np.int64)
    first = (c0 - shift) // BAND
    last = (c0 + W - 1 - shift) // BAND
    np.add.at(counts, first, 1)
    np.add.at(counts, last[last != first], 1)
    return counts


def band_reference(f, vis, lo):
    """Oracle grid of the band of columns [lo, lo + 64) from the visibilities reaching it."""
    sel = (f["c0"] + W - 1 >= lo) & (f["c0"] < lo + BAND)
    op = I.Plan(f["uc"][sel, 0], f["uc"][sel, 1], W, N)
    ref = I.grid(op, f["T"], MS, 1, vis[sel].astype(np.complex128))
    return ref[:, lo:lo + BAND], int(sel.sum())


def test_full_size_gridding_bands(full):
    f = full
    vis = S.complex_normal(f["nv"], 5).astype(np.complex64)
    g = f["p"].grid(torch.from_numpy(vis).cuda()).cpu().numpy()
    counts = supports_per_band(f["c0"])
    dense = int(np.argmax(counts)) * BAND
    occupied = np.nonzero(counts)[0]
    edge = int(occupied[-1]) * BAND
    for lo in (dense, dense + BAND // 2, edge):
        ref, nsel = band_reference(f, vis, lo)
        got = g[:, lo:lo + BAND]
        assert nsel > 0
        assert rel_rms(got, ref) < 1e-5, (lo, nsel)
        assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max(), (lo, nsel)
    # the densest band carries hundreds of thousands of supports
    assert counts.max() > 100000, counts.max()


def test_full_size_degridding_dense_bucket_and_sample(full):
    f = full
    G = S.random_image(N, 12).astype(np.complex64)
    got = f["p"].degrid(torch.from_numpy(G).cuda()).cpu().numpy()
    c0, r0 = f["c0"], f["r0"]
    band = int(np.argmax(supports_per_band(c0))) * BAND
    in_band = np.nonzero((c0 + W - 1 >= band) & (c0 < band + BAND))[0]
    rows = np.bincount(r0[in_band] // 16, minlength=N // 16 + 1)
    top = int(np.argmax(rows))
    dense = in_band[r0[in_band] // 16 == top]
    rand = np.random.default_rng(13).choice(f["nv"], 20000, replace=False)
    idx = np.unique(np.concatenate([dense, rand]))
    op = I.Plan(f["uc"][idx, 0], f["uc"][idx, 1], W, N)
    ref = I.degrid(op, f["T"], MS, 1, G.astype(np.complex128))
    assert dense.size > 1000, dense.size
    assert rel_rms(got[idx], ref) < 1e-5
    assert np.abs(got[idx] - ref).max() < 1e-5 * np.abs(ref).max()


def test_full_size_track_binning_equals_plain_binning(full):
    """The benchmark's track-ordered binning and the plain binning give the same grid (sums
    in another order: every cell within 1e-6 of the largest)."""
    f = full
    vis = torch.from_numpy(S.complex_normal(f["nv"], 6).astype(np.complex64)).cuda()
    q = lmg.Plan(f["tab"], n_img, f["dl"], f["nv"], "c64")
    q.bin(torch.from_numpy(f["uv"]).cuda())
    a = f["p"].grid(vis).cpu().numpy()
    b = q.grid(vis).cpu().numpy()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()

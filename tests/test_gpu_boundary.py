"""C-ABI boundary on the GPU: caller workspace, plans without internal grids, the
factor-form correction, the device status word and host-side injected failures (none of
which makes a kernel fault or wait)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1906_07102_gb300 import lmg  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402
from tests.cases import rel_rms, track_case  # noqa: E402

pytestmark = pytest.mark.gpu

N, n_img, W, Ms = 1024, 512, 7, 1000


@pytest.fixture(scope="module")
def case():
    uv, dl, vis = track_case(n_ant=16, n_times=256, N=N, seed=4)
    t = lmg.Table(W, 0.5, Ms, "linear")
    uvd = torch.from_numpy(uv).cuda()
    visd = torch.from_numpy(vis.astype(np.complex64)).cuda()
    model = torch.from_numpy(S.gaussian_blob_image(n_img, 16, seed=5).astype(np.complex64)).cuda()
    return t, dl, uvd, visd, model


def test_workspace_calls_match_plan_grid_calls(case):
    t, dl, uvd, visd, model = case
    p = lmg.Plan(t, n_img, dl, uvd.shape[0])
    p.bin(uvd)
    ws = p.workspace()
    assert ws.numel() == N * N * 8
    ref_img = p.dirty_image(visd)
    img = p.dirty_image_ws(visd, ws)
    assert torch.equal(img, ref_img)          # same kernels, same buffers' contents
    ref_pv = p.predict_vis(model)
    pv = p.predict_vis_ws(model, ws)
    assert rel_rms(pv.cpu().numpy(), ref_pv.cpu().numpy()) < 1e-6   # in-place vs out-of-place column FFT
    with pytest.raises(lmg.LmgError, match="workspace too small"):
        p.dirty_image_ws(visd, ws[: ws.numel() // 2])
    with pytest.raises(lmg.LmgError, match="256-byte aligned"):
        p.dirty_image_ws(visd, ws[8:])


def test_plan_without_work_grids(case):
    t, dl, uvd, visd, model = case
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    p_full = lmg.Plan(t, n_img, dl, uvd.shape[0])
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    p_lean = lmg.Plan(t, n_img, dl, uvd.shape[0], work_grids=False)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    # the lean plan holds at least the two grids' worth less device memory
    assert (free0 - free1) - (free1 - free2) >= 2 * N * N * 8 * 0.9
    p_full.bin(uvd)
    p_lean.bin(uvd)
    assert p_lean.work_grid() is None
    with pytest.raises(lmg.LmgError, match="lmg_dirty_image_ws"):
        p_lean.dirty_image(visd)
    with pytest.raises(lmg.LmgError, match="lmg_predict_vis_ws"):
        p_lean.predict_vis(model)
    ws = p_lean.workspace()
    # two plans bin in their own (atomic) record order: float32 sums agree to rounding
    assert rel_rms(p_lean.dirty_image_ws(visd, ws).cpu().numpy(), p_full.dirty_image(visd).cpu().numpy()) < 1e-6
    assert rel_rms(p_lean.predict_vis_ws(model, ws).cpu().numpy(), p_full.predict_vis(model).cpu().numpy()) < 1e-6


def test_correct_factors_equals_plan_correction(case):
    t, dl, uvd, visd, model = case
    p = lmg.Plan(t, n_img, dl, uvd.shape[0])
    h = torch.from_numpy(t.correction(n_img, single_precision=True).astype(np.float32)).cuda()
    F = torch.from_numpy(S.random_image(N, 31).astype(np.complex64)).cuda()
    assert torch.equal(lmg.correct_factors("crop", F, h, n_img, N), p.crop_correct(F))
    assert torch.equal(lmg.correct_factors("pad", model, h, n_img, N), p.pad_correct(model))


def test_status_word_clear_after_normal_binning(case):
    t, dl, uvd, visd, model = case
    p = lmg.Plan(t, n_img, dl, uvd.shape[0])
    p.bin(uvd)
    assert p.status() == (0, 0)


def test_injected_item_capacity_is_reported_by_the_device(case, monkeypatch):
    """A plan whose work-item capacity is one item: the binning's own bounds check drops the
    other items and sets the status word; lmg_plan_status reports LMG_EDEVICE."""
    t, dl, uvd, visd, model = case
    monkeypatch.setenv("LMG_INJECT_FAULT", "item_cap")
    p = lmg.Plan(t, n_img, dl, uvd.shape[0])
    monkeypatch.delenv("LMG_INJECT_FAULT")
    p.bin(uvd)
    p.grid(visd)  # runs on the one item it kept, in bounds
    rc, bits = p.status()
    assert rc == -7 and bits & 1
    assert "work items" in lmg.lib().lmg_last_error().decode()


@pytest.mark.parametrize("point,code", [("device_alloc", -2), ("cufft_plan", -4)])
def test_injected_failures_release_everything(case, monkeypatch, point, code):
    t, dl, uvd, visd, model = case
    torch.cuda.synchronize()
    lmg.Plan(t, n_img, dl, uvd.shape[0])   # warm: context, cuFFT library state
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("LMG_INJECT_FAULT", point)
    with pytest.raises(lmg.LmgError, match=f"lmg error {code}"):
        lmg.Plan(t, n_img, dl, uvd.shape[0])
    monkeypatch.delenv("LMG_INJECT_FAULT")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_fp32_fma_rate_is_plausible():
    r = lmg.fp32_fma_rate()
    # 152 SMs x 128 lanes x 2 flop x ~2 GHz is about 78 TFLOP/s
    assert 2e13 < r < 2e14



def test_misaligned_views_are_rejected(case):
    """A grid or visibility view off its alignment is LMG_EINVAL before any launch (the
    kernels read and write grids with 16-byte vector accesses)."""
    t, dl, uvd, visd, model = case
    p = lmg.Plan(t, n_img, dl, uvd.shape[0])
    p.bin(uvd)
    buf = torch.zeros(N * N + 1, dtype=torch.complex64, device="cuda")
    g_off = buf[1:].view(N, N)                 # 8 bytes past a 16-byte boundary
    with pytest.raises(lmg.LmgError, match="grid must be 16-byte aligned"):
        p.grid(visd, out=g_off)
    with pytest.raises(lmg.LmgError, match="grid must be 16-byte aligned"):
        p.degrid(g_off)
    # a visibility array 4 bytes past an 8-byte boundary (torch makes no such complex view:
    # the pointer goes to the C call directly)
    import ctypes
    vb = torch.zeros(2 * visd.shape[0] + 2, dtype=torch.float32, device="cuda")
    g = p.grid(visd)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = lmg.lib()
    assert L.lmg_degrid(p._h, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(vb.data_ptr() + 4), stream) == -1
    assert "visibilities must be 8-byte aligned" in L.lmg_last_error().decode()
    # the plan still works after the refusals
    g = p.grid(visd)
    assert torch.isfinite(torch.view_as_real(g)).all()


def test_degrid_add_accumulates(case):
    """lmg_degrid_add adds the predictions to what the output holds: prior + degrid(G)."""
    t, dl, uvd, visd, model = case
    p = lmg.Plan(t, n_img, dl, uvd.shape[0])
    p.bin(uvd)
    G = torch.from_numpy(S.random_image(N, 11).astype(np.complex64)).cuda()
    ref = p.degrid(G)
    prior = torch.from_numpy(S.complex_normal(uvd.shape[0], 12).astype(np.complex64)).cuda()
    out = prior.clone()
    p.degrid(G, out=out, add=True)
    assert rel_rms((out - prior).cpu().numpy(), ref.cpu().numpy()) < 1e-6
    z = torch.zeros_like(prior)
    assert torch.equal(p.degrid(G, out=z, add=True), ref)   # onto zeros: the same bits

"""C ABI of liblmg on the host (no GPU needed): every declared entry point is exported, the
host-side table builder agrees with the oracle, and argument errors are reported.
No call here launches a kernel."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import design as D
from oracle import imaging as I
from tests import prolate as P
from tests import small_field as SF

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lmg.h")


@pytest.fixture(scope="module")
def lmg():
    from paper_1906_07102_gb300 import build, lmg as L
    if not os.path.exists(L.LIB_PATH):
        build.build()
    L.lib()
    return L


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lmg_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_function_is_exported_and_bound(lmg):
    names = declared_functions()
    assert len(names) >= 20
    raw = ctypes.CDLL(lmg.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
        assert n in lmg.EXPORTED, n
    assert lmg.lib().lmg_version().decode().startswith("lmg")


@pytest.mark.parametrize("args,msg", [
    ((0, 0.5, 100, 1, 0), "W must be"), ((17, 0.5, 100, 1, 0), "W must be"),
    ((7, 0.0, 100, 1, 0), "x0 must be"), ((7, 1.5, 100, 1, 0), "x0 must be"),
    ((7, 0.5, 1, 1, 0), "oversample"), ((7, 0.5, 100, 5, 0), "interp"), ((7, 0.5, 100, -1, 0), "interp"),
    ((7, 0.5, 2, 3, 0), "at least the interpolation degree"), ((7, 0.5, 100, 1, 5), "correction")])
def test_table_argument_errors(lmg, args, msg):
    h = ctypes.c_void_p()
    rc = lmg.lib().lmg_kernel_table(*args, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert msg in lmg.lib().lmg_last_error().decode()


def test_null_outputs_are_rejected(lmg):
    L = lmg.lib()
    assert L.lmg_kernel_table(7, 0.5, 100, 1, 0, None) == -1
    assert L.lmg_table_export(None, None, 0, None, 0, None, None) == -1
    assert L.lmg_plan_bin(None, None, 0, None) == -1
    assert L.lmg_plan_bin_tracks(None, None, 0, 1, None) == -1
    assert L.lmg_grid(None, None, None, 0, None, None) == -1


@pytest.mark.parametrize("W,Ms,interp", [(3, 100, "nearest"), (5, 200, "linear"), (5, 60, "cubic")])
def test_library_table_matches_oracle(lmg, W, Ms, interp):
    """The library's C++ optimiser and the oracle's scipy one reach the same optimum; the
    optimum of E is determined to about 1e-9 in float64 (flat directions of h)."""
    t = lmg.Table(W, 0.5, Ms, interp)
    C, h, E, info = t.export()
    ho = D.least_misfit_h(W, 0.25)
    Co = D.lm_table(ho, W, 0.25, Ms)
    assert info[0] == W and info[1] == Ms and info[2] == 32
    assert abs(E - D.design_E(ho, W, 0.25)) <= 1e-6 * E
    assert np.abs(C - Co).max() <= 1e-6 * np.abs(Co).max()
    assert np.abs(h - ho).max() <= 1e-5
    n_img, N = 64, 128
    hv = t.correction(n_img)
    hvo = D.correction_factors(Co, Ms, {"nearest": 0, "linear": 1, "cubic": 3}[interp], W, I.pixel_coords(n_img, N))
    np.testing.assert_allclose(hv, hvo, rtol=1e-6)


@pytest.mark.parametrize("x0p", [0.1, 0.25, 0.4])
def test_w1_library_table_is_the_prolate_spheroidal_function(lmg, x0p):
    """The library's own optimiser at W = 1 against the closed form of tests/prolate.py
    (E_min = 1 - lambda_0(pi x0) / (2 x0); h and C follow S_00): within the second-order
    gap of Appendix A's 33 x-nodes and 16 s-nodes (the oracle's side is pinned the same
    way, with its convergence, in test_oracle_design.py)."""
    E_ref, h_ref, C_ref = P.w1_design(x0p)
    Ms = 100
    C, h, E, info = lmg.Table(1, 2 * x0p, Ms, "linear").export()
    assert info[0] == 1 and info[2] == 32
    assert abs(E / E_ref - 1.0) < 1e-3
    assert np.abs(h - h_ref(x0p * np.arange(33) / 32)).max() < 3e-4
    t = np.arange(Ms + 1) / Ms - 0.5                   # row i: offset d = i / Ms - 1/2
    assert np.abs(C[:, 0] / C[Ms // 2, 0] - C_ref(t)).max() < 2e-4


@pytest.mark.parametrize("x0p", [0.1, 0.25, 0.4])
def test_w1_library_correction_is_prolate(lmg, x0p):
    """The library's correction factors (its own quadrature of c and D, Eqs. 12-15) for its
    W = 1 table follow S_00(pi x0, x/x0) on the kept pixels (closed form in tests/prolate.py)."""
    _, h_ref, _ = P.w1_design(x0p)
    n_img = 64
    N = int(round(n_img / (2 * x0p)))
    hv = lmg.Table(1, 2 * x0p, 1000, "linear").correction(n_img)
    x = I.pixel_coords(n_img, N)
    assert np.abs(hv / hv[n_img // 2] - h_ref(x)).max() < 2e-5


@pytest.mark.parametrize("W", [2, 3, 4])
def test_library_table_small_field_limit(lmg, W):
    """The library's own optimiser at x0 = 0.025 (API 0.05) against the small-field closed
    form of tests/small_field.py: E within 1%, C within 1.5e-3, h's deviation from 1 within
    1% (the oracle's side, with its convergence, is in test_oracle_design.py)."""
    x0p, Ms = 0.025, 100
    C, h, E, _ = lmg.Table(W, 2 * x0p, Ms, "linear").export()
    assert abs(E / SF.E_leading(W, x0p) - 1.0) < 0.01
    Cp = SF.C_leading(W, np.arange(Ms + 1) / Ms)
    assert np.abs(C - Cp).max() < 1.5e-3 * np.abs(Cp).max()
    assert np.abs(h - SF.h_leading(W, x0p * np.arange(33) / 32)).max() < 1e-2 * np.abs(h - 1.0).max()


def test_w7_library_table_reaches_paper_level(lmg):
    """W = 7, x0 = 0.25 (API 0.5): E of order 1e-14 (Section 2.2) from the library's own
    optimiser; the table is mirror-symmetric (Section 5.2)."""
    t = lmg.Table(7, 0.5, 1000, "linear")
    C, h, E, _ = t.export()
    assert 1e-16 < E < 3e-14
    assert np.all(np.diff(h) > 0)
    assert np.abs(C[::-1, ::-1] - C).max() < 1e-10 * np.abs(C).max()


def test_table_from_values_round_trip(lmg):
    vals = np.random.default_rng(0).random((65, 4))
    t = lmg.Table(4, 0.5, 64, "linear", values=vals)
    C, h, E, _ = t.export()
    np.testing.assert_array_equal(C, vals)
    assert np.isnan(E) and np.all(h == 0)
    bad = vals.copy()
    bad[3, 2] = np.nan
    with pytest.raises(lmg.LmgError, match="finite"):
        lmg.Table(4, 0.5, 64, "linear", values=bad)


def test_correction_single_precision_rounding(lmg):
    """The float32 path's correction factors use the table rounded to float32."""
    t = lmg.Table(7, 0.5, 1000, "linear")
    h64 = t.correction(128)
    h32 = t.correction(128, single_precision=True)
    assert 0 < np.abs(h64 - h32).max() < 1e-6 * np.abs(h64).max()


def test_correction_rejects_non_even_grid(lmg):
    t = lmg.Table(5, 0.5, 100, "linear")
    out = np.empty(63)
    assert lmg.lib().lmg_correction_export(t._h, 63, 0, out.ctypes.data_as(ctypes.c_void_p)) == -1


def test_static_grid_validates_before_touching_the_device(lmg):
    t = lmg.Table(7, 0.5, 1000, "linear")
    L = lmg.lib()
    rc = L.lmg_grid_static(t._h, 512, 1e-3, None, lmg.STATIC_MAX_VIS + 1, None, None, ctypes.c_void_p(16), None)
    assert rc == -1 and "lmg_grid_static" in L.lmg_last_error().decode()
    rc = L.lmg_grid_static(t._h, 4 * lmg.STATIC_MAX_N, 1e-3, None, 0, None, None, ctypes.c_void_p(16), None)
    assert rc == -1 and "lmg_grid_static" in L.lmg_last_error().decode()


def test_plan_creation_without_a_device_reports_an_error(lmg):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    t = lmg.Table(5, 0.5, 100, "linear")
    h = ctypes.c_void_p()
    rc = lmg.lib().lmg_plan_create(t._h, 64, 1e-3, 100, 0, ctypes.byref(h))
    assert rc < 0 and not h.value
    assert lmg.lib().lmg_last_error().decode() != ""


def test_plan_argument_errors_precede_device_work(lmg):
    t = lmg.Table(5, 0.5, 100, "linear")
    h = ctypes.c_void_p()
    L = lmg.lib()
    for n_img, scale, maxv, dtype, msg in ((63, 1e-3, 10, 0, "n_image"), (64, 0.0, 10, 0, "pixel_scale"),
                                           (64, 1e-3, 0, 0, "max_vis"), (64, 1e-3, 10, 3, "dtype"),
                                           (40, 1e-3, 10, 0, "multiple of 64"), (48, 1e-3, 10, 0, "multiple of 64")):
        assert L.lmg_plan_create(t._h, n_img, scale, maxv, dtype, ctypes.byref(h)) == -1
        assert msg in L.lmg_last_error().decode()


def test_batch_argument_errors_precede_device_work(lmg):
    L = lmg.lib()
    h = ctypes.c_void_p()
    assert L.lmg_batch_create(0, None, None, None, None, ctypes.byref(h)) == -1
    assert "n_chan" in L.lmg_last_error().decode()
    assert L.lmg_batch_create(2, None, None, None, None, ctypes.byref(h)) == -1
    tabs = (ctypes.c_void_p * 2)(None, None)
    n = np.array([64, 64], dtype=np.int64)
    s = np.array([1e-3, 1e-3])
    assert L.lmg_batch_create(2, ctypes.cast(tabs, ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                              s.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                              ctypes.byref(h)) == -1
    assert "tables[0]" in L.lmg_last_error().decode()
    assert L.lmg_batch_bin(None, None, None, None) == -1
    assert L.lmg_batch_grid(None, None, None, None, None) == -1
    assert L.lmg_batch_info(None, None) == -1


def test_direct_calculation_tables(lmg):
    """LMG_INTERP_DIRECT (Section 5.2): a least-misfit table accepts it, a caller table does
    not; its correction factors (from the exact function) agree with those of a finely
    sampled cubic table of the same design."""
    direct = lmg.Table(7, 0.5, 4, "direct")
    cubic = lmg.Table(7, 0.5, 20000, "cubic")
    hd, hc = direct.correction(256), cubic.correction(256)
    assert np.abs(hd - hc).max() < 1e-12 * np.abs(hc).max()
    with pytest.raises(lmg.LmgError, match="lmg_kernel_table"):
        lmg.Table(4, 0.5, 64, "direct", values=np.ones((65, 4)))


# ----------------------------------------------------------------------------------------
# host-side fault injection (LMG_INJECT_FAULT) and the argument checks of the workspace,
# factor-form correction and status calls; none of these reaches a kernel
# ----------------------------------------------------------------------------------------
def test_injected_host_allocation_failure(lmg, monkeypatch):
    monkeypatch.setenv("LMG_INJECT_FAULT", "host_alloc")
    L = lmg.lib()
    h = ctypes.c_void_p()
    assert L.lmg_kernel_table(5, 0.5, 100, 1, 0, ctypes.byref(h)) == -2 and not h.value
    assert "host allocation" in L.lmg_last_error().decode()
    vals = np.ones((101, 5))
    assert L.lmg_table_from_values(5, 0.5, 100, 1, 0, vals.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)) == -2
    monkeypatch.delenv("LMG_INJECT_FAULT")
    assert L.lmg_kernel_table(5, 0.5, 100, 1, 0, ctypes.byref(h)) == 0 and h.value
    L.lmg_table_free(h)


@pytest.mark.parametrize("flags", [0, 1])
def test_injected_device_allocation_failure(lmg, monkeypatch, flags):
    """The first device allocation of a plan fails (before any CUDA call of the plan): the
    plan is released and LMG_ENOMEM returned with the failing buffer named."""
    t = lmg.Table(5, 0.5, 100, "linear")
    monkeypatch.setenv("LMG_INJECT_FAULT", "device_alloc")
    h = ctypes.c_void_p()
    rc = lmg.lib().lmg_plan_create_ex(t._h, 64, 1e-3, 100, 0, flags, ctypes.byref(h))
    assert rc == -2 and not h.value
    msg = lmg.lib().lmg_last_error().decode()
    assert "device allocation of table failed: injected" in msg


def test_new_entry_point_argument_errors(lmg):
    L = lmg.lib()
    t = lmg.Table(5, 0.5, 100, "linear")
    h = ctypes.c_void_p()
    assert L.lmg_plan_create_ex(t._h, 64, 1e-3, 100, 0, 2, ctypes.byref(h)) == -1
    assert "flags" in L.lmg_last_error().decode()
    assert L.lmg_workspace_bytes(None) == 0
    assert L.lmg_dirty_image_ws(None, None, None, 0, None, None, 0, None) == -1
    assert L.lmg_predict_vis_ws(None, None, None, None, 0, None) == -1
    assert L.lmg_plan_status(None, None, None) == -1
    assert L.lmg_fp32_fma_rate(None, None) == -1
    p16 = ctypes.c_void_p(256)
    assert L.lmg_correct_factors(0, None, p16, p16, 64, 128, 0, None) == -1
    assert L.lmg_correct_factors(0, p16, p16, p16, 63, 128, 0, None) == -1
    assert L.lmg_correct_factors(0, p16, p16, p16, 64, 32, 0, None) == -1
    assert L.lmg_correct_factors(0, p16, p16, p16, 64, 128, 2, None) == -1
    assert L.lmg_correct_factors(2, p16, p16, p16, 64, 128, 0, None) == -1
    assert "direction" in L.lmg_last_error().decode()


def test_misaligned_arrays_are_rejected_before_device_work(lmg):
    """Device arrays are checked for alignment before anything is launched: a grid or image
    view that is not 16-byte aligned, or a visibility array off its element size, is
    LMG_EINVAL (NULL plan and pointer arguments are checked first, so no device is needed)."""
    L = lmg.lib()
    p4 = ctypes.c_void_p(256 + 4)
    p8 = ctypes.c_void_p(256 + 8)
    p16 = ctypes.c_void_p(256)
    assert L.lmg_correct_factors(0, p4, p16, p16, 64, 128, 0, None) == -1
    assert "in must be 8-byte aligned" in L.lmg_last_error().decode()
    assert L.lmg_correct_factors(0, p16, p8, p16, 64, 128, 1, None) == -1
    assert "out must be 16-byte aligned" in L.lmg_last_error().decode()
    assert L.lmg_correct_factors(0, p16, p16, ctypes.c_void_p(258), 64, 128, 0, None) == -1
    assert "h must be 4-byte aligned" in L.lmg_last_error().decode()

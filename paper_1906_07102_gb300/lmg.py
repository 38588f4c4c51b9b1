"""Thin ctypes binding of liblmg (include/lmg.h) for torch CUDA tensors.

Argument marshalling only: every step of gridding, FFT, correction and degridding runs in
the CUDA library. torch supplies device memory and the current stream. Loading fails
loudly (RuntimeError) when the library has not been built; there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblmg.so")

LMG_C64, LMG_C128 = 0, 1
INTERP = {"nearest": 0, "linear": 1, "quadratic": 2, "cubic": 3, "direct": 4}
CORRECTION = {"hopt": 0, "inv_c": 1}
ACCUM = {"plain": 0, "compensated": 1}
LMG_CROP, LMG_PAD = 0, 1
FFT_IMAGE, FFT_MODEL = 1, -1
PLAN_NO_WORK_GRIDS = 1

_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_SIGS = {
    "lmg_kernel_table": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(_vp)]),
    "lmg_table_from_values": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "lmg_table_free": (ctypes.c_int, [_vp]),
    "lmg_table_export": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t, _vp, _vp]),
    "lmg_correction_export": (ctypes.c_int, [_vp, _i64, ctypes.c_int, _vp]),
    "lmg_plan_create": (ctypes.c_int, [_vp, _i64, ctypes.c_double, _i64, ctypes.c_int, ctypes.POINTER(_vp)]),
    "lmg_plan_free": (ctypes.c_int, [_vp]),
    "lmg_plan_bin": (ctypes.c_int, [_vp, _vp, _i64, _vp]),
    "lmg_plan_bin_tracks": (ctypes.c_int, [_vp, _vp, _i64, _i64, _vp]),
    "lmg_transform_scratch_bytes": (ctypes.c_size_t, [_vp]),
    "lmg_degrid_add": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lmg_image_from_grid": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lmg_grid_from_image": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lmg_plan_dropped": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), _vp]),
    "lmg_plan_info": (ctypes.c_int, [_vp, _vp, _vp]),
    "lmg_work_grid": (_vp, [_vp]),
    "lmg_grid": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]),
    "lmg_degrid": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lmg_fft": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "lmg_fft_pruned": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "lmg_grid_correct": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "lmg_dirty_image": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]),
    "lmg_predict_vis": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lmg_grid_static": (ctypes.c_int, [_vp, _i64, ctypes.c_double, _vp, _i64, _vp, _vp, _vp, _vp]),
    "lmg_batch_create": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "lmg_batch_free": (ctypes.c_int, [_vp]),
    "lmg_batch_bin": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lmg_batch_grid": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lmg_batch_degrid": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lmg_batch_dirty_image": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lmg_batch_predict_vis": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lmg_batch_tune": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lmg_batch_info": (ctypes.c_int, [_vp, _vp]),
    "lmg_plan_create_ex": (ctypes.c_int, [_vp, _i64, ctypes.c_double, _i64, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_vp)]),
    "lmg_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "lmg_dirty_image_ws": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_size_t, _vp]),
    "lmg_predict_vis_ws": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "lmg_correct_factors": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _i64, _i64, ctypes.c_int, _vp]),
    "lmg_plan_status": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), _vp]),
    "lmg_fp32_fma_rate": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), _vp]),
    "lmg_last_error": (ctypes.c_char_p, []),
    "lmg_version": (ctypes.c_char_p, []),
}
EXPORTED = tuple(_SIGS)


class LmgError(RuntimeError):
    pass


def lib():
    """The loaded library (built in-tree by ``paper_1906_07102_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblmg.so not built ({LIB_PATH}); run python -m paper_1906_07102_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise LmgError(f"lmg error {rc}: {lib().lmg_last_error().decode()}")


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(t, dtype, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class Table:
    """Least-misfit gridding function and look-up table (host float64)."""

    def __init__(self, W, x0, oversample, interp="linear", correction="hopt", values=None):
        h = ctypes.c_void_p()
        if values is None:
            _check(lib().lmg_kernel_table(W, x0, oversample, INTERP[interp], CORRECTION[correction], ctypes.byref(h)))
        else:
            v = np.ascontiguousarray(values, dtype=np.float64)
            if v.shape != (oversample + 1, W):
                raise ValueError("values must have shape (oversample + 1, W)")
            _check(lib().lmg_table_from_values(W, x0, oversample, INTERP[interp], CORRECTION[correction],
                                               v.ctypes.data_as(_vp), ctypes.byref(h)))
        self._h = h
        self.W, self.x0, self.oversample, self.interp = W, x0, oversample, interp

    def export(self):
        """(C [(Ms+1), W], h_nodes [33], E, info[4]) as numpy / floats."""
        C = np.empty((self.oversample + 1, self.W))
        h = np.empty(33)
        E = ctypes.c_double()
        info = (ctypes.c_int * 4)()
        _check(lib().lmg_table_export(self._h, C.ctypes.data_as(_vp), C.size, h.ctypes.data_as(_vp), h.size,
                                      ctypes.byref(E), info))
        return C, h, E.value, list(info)

    def correction(self, n_image, single_precision=False):
        out = np.empty(n_image)
        _check(lib().lmg_correction_export(self._h, n_image, int(bool(single_precision)), out.ctypes.data_as(_vp)))
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lmg_table_free(self._h)
            self._h = None


class Plan:
    """Device state for one (table, image size, pixel scale); see lmg_plan_create."""

    def __init__(self, table, n_image, pixel_scale, max_vis, dtype="c64", work_grids=True):
        import torch
        self.dtype_code = LMG_C64 if dtype == "c64" else LMG_C128
        self.cdtype = torch.complex64 if self.dtype_code == LMG_C64 else torch.complex128
        self.rdtype = torch.float32 if self.dtype_code == LMG_C64 else torch.float64
        h = ctypes.c_void_p()
        if work_grids:
            _check(lib().lmg_plan_create(table._h, n_image, pixel_scale, max_vis, self.dtype_code, ctypes.byref(h)))
        else:
            _check(lib().lmg_plan_create_ex(table._h, n_image, pixel_scale, max_vis, self.dtype_code,
                                            PLAN_NO_WORK_GRIDS, ctypes.byref(h)))
        self._h = h
        self.table = table
        self.n_image = n_image
        self.N = int(round(n_image / table.x0))
        self.W = table.W
        self.nvis = None

    def bin(self, uv, tracks=None):
        """Bins uv (CUDA float64 [nvis, 2], wavelengths). tracks: number of tracks when the
        positions are stored sample-major (row k = t * tracks + b), else None."""
        import torch
        uv = _need(uv, torch.float64, None, "uv")
        if uv.dim() != 2 or uv.shape[1] != 2:
            raise ValueError("uv must be [nvis, 2]")
        if tracks is None:
            _check(lib().lmg_plan_bin(self._h, _ptr(uv), uv.shape[0], _stream()))
        else:
            _check(lib().lmg_plan_bin_tracks(self._h, _ptr(uv), uv.shape[0], int(tracks), _stream()))
        self.nvis = uv.shape[0]
        return self

    def transform_scratch_bytes(self):
        """Bytes of the scratch of image_from_grid / grid_from_image (0: none needed)."""
        return int(lib().lmg_transform_scratch_bytes(self._h))

    def image_from_grid(self, grid, out=None, scratch=None):
        """Dirty image from a gridded [N, N] array: transform, correction and crop (the
        fused kernels where the plan has them; otherwise grid is transformed in place)."""
        import torch
        _need(grid, self.cdtype, (self.N, self.N), "grid")
        if out is None:
            out = torch.empty((self.n_image, self.n_image), dtype=self.cdtype, device=grid.device)
        _need(out, self.cdtype, (self.n_image, self.n_image), "image")
        _check(lib().lmg_image_from_grid(self._h, _ptr(grid), _ptr(out), _ptr(scratch), _stream()))
        return out

    def grid_from_image(self, image, out=None, scratch=None):
        """Model grid [N, N] from an image: pad, correction and transform."""
        import torch
        _need(image, self.cdtype, (self.n_image, self.n_image), "image")
        if out is None:
            out = torch.empty((self.N, self.N), dtype=self.cdtype, device=image.device)
        _need(out, self.cdtype, (self.N, self.N), "grid")
        _check(lib().lmg_grid_from_image(self._h, _ptr(image), _ptr(out), _ptr(scratch), _stream()))
        return out

    def _vis_args(self, vis, weights):
        vis = _need(vis, self.cdtype, (self.nvis,), "vis")
        if weights is not None:
            weights = _need(weights, self.rdtype, (self.nvis,), "weights")
        return vis, weights

    def grid(self, vis, weights=None, accum="plain", out=None):
        import torch
        vis, weights = self._vis_args(vis, weights)
        if out is None:
            out = torch.empty((self.N, self.N), dtype=self.cdtype, device=vis.device)
        _need(out, self.cdtype, (self.N, self.N), "grid")
        _check(lib().lmg_grid(self._h, _ptr(vis), _ptr(weights), ACCUM[accum], _ptr(out), _stream()))
        return out

    def degrid(self, grid, out=None, add=False):
        """Predicted visibilities of a grid; add=True adds them to out (lmg_degrid_add)."""
        import torch
        _need(grid, self.cdtype, (self.N, self.N), "grid")
        if out is None:
            if add:
                raise ValueError("add=True needs out")
            out = torch.empty(self.nvis, dtype=self.cdtype, device=grid.device)
        _need(out, self.cdtype, (self.nvis,), "vis_out")
        f = lib().lmg_degrid_add if add else lib().lmg_degrid
        _check(f(self._h, _ptr(grid), _ptr(out), _stream()))
        return out

    def fft(self, grid, direction, pruned=False):
        """In-place 2-D FFT of an [N, N] grid; pruned=True runs the transform the imaging /
        prediction paths use (exact on the kept field only, see lmg_fft_pruned)."""
        _need(grid, self.cdtype, (self.N, self.N), "grid")
        f = lib().lmg_fft_pruned if pruned else lib().lmg_fft
        _check(f(self._h, FFT_IMAGE if direction == "image" else FFT_MODEL, _ptr(grid), _stream()))
        return grid

    def crop_correct(self, F, out=None):
        import torch
        _need(F, self.cdtype, (self.N, self.N), "F")
        if out is None:
            out = torch.empty((self.n_image, self.n_image), dtype=self.cdtype, device=F.device)
        _need(out, self.cdtype, (self.n_image, self.n_image), "image")
        _check(lib().lmg_grid_correct(self._h, LMG_CROP, _ptr(F), _ptr(out), _stream()))
        return out

    def pad_correct(self, image, out=None):
        import torch
        _need(image, self.cdtype, (self.n_image, self.n_image), "image")
        if out is None:
            out = torch.empty((self.N, self.N), dtype=self.cdtype, device=image.device)
        _need(out, self.cdtype, (self.N, self.N), "grid")
        _check(lib().lmg_grid_correct(self._h, LMG_PAD, _ptr(image), _ptr(out), _stream()))
        return out

    def dirty_image(self, vis, weights=None, accum="plain", out=None):
        import torch
        vis, weights = self._vis_args(vis, weights)
        if out is None:
            out = torch.empty((self.n_image, self.n_image), dtype=self.cdtype, device=vis.device)
        _need(out, self.cdtype, (self.n_image, self.n_image), "image")
        _check(lib().lmg_dirty_image(self._h, _ptr(vis), _ptr(weights), ACCUM[accum], _ptr(out), _stream()))
        return out

    def predict_vis(self, image, out=None):
        import torch
        _need(image, self.cdtype, (self.n_image, self.n_image), "image")
        if out is None:
            out = torch.empty(self.nvis, dtype=self.cdtype, device=image.device)
        _need(out, self.cdtype, (self.nvis,), "vis_out")
        _check(lib().lmg_predict_vis(self._h, _ptr(image), _ptr(out), _stream()))
        return out

    def workspace_bytes(self):
        return int(lib().lmg_workspace_bytes(self._h))

    def workspace(self, device=None):
        """A device workspace for dirty_image / predict_vis with ws= (torch allocations are
        256-byte aligned)."""
        import torch
        return torch.empty(self.workspace_bytes(), dtype=torch.uint8, device=device or "cuda")

    def dirty_image_ws(self, vis, ws, weights=None, accum="plain", out=None):
        import torch
        vis, weights = self._vis_args(vis, weights)
        if out is None:
            out = torch.empty((self.n_image, self.n_image), dtype=self.cdtype, device=vis.device)
        _need(out, self.cdtype, (self.n_image, self.n_image), "image")
        _check(lib().lmg_dirty_image_ws(self._h, _ptr(vis), _ptr(weights), ACCUM[accum], _ptr(out), _ptr(ws),
                                        ws.numel() * ws.element_size(), _stream()))
        return out

    def predict_vis_ws(self, image, ws, out=None):
        import torch
        _need(image, self.cdtype, (self.n_image, self.n_image), "image")
        if out is None:
            out = torch.empty(self.nvis, dtype=self.cdtype, device=image.device)
        _need(out, self.cdtype, (self.nvis,), "vis_out")
        _check(lib().lmg_predict_vis_ws(self._h, _ptr(image), _ptr(out), _ptr(ws), ws.numel() * ws.element_size(),
                                        _stream()))
        return out

    def status(self):
        """(rc, status bits) of lmg_plan_status: rc 0 or LMG_EDEVICE (-7)."""
        bits = ctypes.c_int()
        rc = lib().lmg_plan_status(self._h, ctypes.byref(bits), _stream())
        return rc, bits.value

    def dropped(self):
        n = ctypes.c_int64()
        _check(lib().lmg_plan_dropped(self._h, ctypes.byref(n), _stream()))
        return n.value

    def info(self):
        out = (ctypes.c_int64 * 8)()
        _check(lib().lmg_plan_info(self._h, out, _stream()))
        keys = ["N", "n_image", "W", "nvis", "records", "items", "dtype"]
        return dict(zip(keys, list(out)[:7]))

    def work_grid(self):
        return lib().lmg_work_grid(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lmg_plan_free(self._h)
            self._h = None


def correct_factors(direction, inp, h, n_image, N, out=None):
    """lmg_correct_factors: crop ("crop") or pad ("pad") with caller device factors h."""
    import torch
    cd = inp.dtype
    dt = LMG_C64 if cd == torch.complex64 else LMG_C128
    shape = (n_image, n_image) if direction == "crop" else (N, N)
    if out is None:
        out = torch.empty(shape, dtype=cd, device=inp.device)
    _check(lib().lmg_correct_factors(LMG_CROP if direction == "crop" else LMG_PAD, _ptr(inp), _ptr(out), _ptr(h),
                                     n_image, N, dt, _stream()))
    return out


def fp32_fma_rate():
    """Measured float32 FMA throughput of the current device (flop/s); synchronises."""
    r = ctypes.c_double()
    _check(lib().lmg_fp32_fma_rate(ctypes.byref(r), _stream()))
    return r.value


STATIC_MAX_VIS = 262144
STATIC_MAX_N = 2048


def grid_static(table, n_image, pixel_scale, uv, vis, weights=None, out=None):
    """Binning plus gridding through lmg_grid_static (complex64): the same result as
    Plan.bin + Plan.grid, with no device allocation inside the library (all working memory
    is a fixed array of the library; see include/lmg.h for the limits)."""
    import torch
    uv = _need(uv, torch.float64, None, "uv")
    nvis = uv.shape[0]
    vis = _need(vis, torch.complex64, (nvis,), "vis")
    if weights is not None:
        weights = _need(weights, torch.float32, (nvis,), "weights")
    N = int(round(n_image / table.x0))
    if out is None:
        out = torch.empty((N, N), dtype=torch.complex64, device=vis.device)
    _need(out, torch.complex64, (N, N), "grid")
    _check(lib().lmg_grid_static(table._h, n_image, pixel_scale, _ptr(uv), nvis, _ptr(vis), _ptr(weights),
                                 _ptr(out), _stream()))
    return out


def _ptr_array(tensors):
    """Host array of device pointers (NULL for None entries)."""
    arr = (_vp * len(tensors))()
    for i, x in enumerate(tensors):
        arr[i] = x.data_ptr() if x is not None else None
    return arr


class Batch:
    """Many independent channels (own table, grid size, pixel scale and uv set each),
    gridded and degridded together: one persistent sweep launch per support width, one
    batched FFT per grid size, each operation captured into a CUDA graph (complex64)."""

    def __init__(self, tables, n_images, pixel_scales, max_vis):
        n = len(tables)
        if not (len(n_images) == len(pixel_scales) == len(max_vis) == n):
            raise ValueError("per-channel argument lists must have equal lengths")
        self.tables = list(tables)
        self.n_images = [int(v) for v in n_images]
        self.N = [int(round(ni / t.x0)) for ni, t in zip(self.n_images, self.tables)]
        tabs = (_vp * n)(*[t._h for t in self.tables])
        nim = np.asarray(self.n_images, dtype=np.int64)
        ps = np.asarray(pixel_scales, dtype=np.float64)
        mv = np.asarray(max_vis, dtype=np.int64)
        h = _vp()
        _check(lib().lmg_batch_create(n, ctypes.cast(tabs, _vp), nim.ctypes.data_as(_vp), ps.ctypes.data_as(_vp),
                                      mv.ctypes.data_as(_vp), ctypes.byref(h)))
        self._h = h
        self.n_chan = n
        self.nvis = None

    def bin(self, uvs):
        """Bins uvs[c] (CUDA float64 [nvis_c, 2], wavelengths); the tensors must stay alive
        while the batch uses them (the tuner re-bins from them)."""
        import torch
        if len(uvs) != self.n_chan:
            raise ValueError("one uv tensor per channel")
        for u in uvs:
            _need(u, torch.float64, None, "uv")
        self._uvs = list(uvs)
        nv = np.asarray([u.shape[0] for u in uvs], dtype=np.int64)
        _check(lib().lmg_batch_bin(self._h, ctypes.cast(_ptr_array(uvs), _vp), nv.ctypes.data_as(_vp), _stream()))
        self.nvis = [int(v) for v in nv]
        return self

    def _vis_lists(self, vis, weights):
        import torch
        for c, v in enumerate(vis):
            _need(v, torch.complex64, (self.nvis[c],), "vis")
        if weights is not None:
            for c, w in enumerate(weights):
                if w is not None:
                    _need(w, torch.float32, (self.nvis[c],), "weights")
        return _ptr_array(vis), (_ptr_array(weights) if weights is not None else None)

    def grid(self, vis, weights=None, out=None):
        import torch
        if out is None:
            out = [torch.empty((N, N), dtype=torch.complex64, device=v.device) for N, v in zip(self.N, vis)]
        for c, g in enumerate(out):
            _need(g, torch.complex64, (self.N[c], self.N[c]), "grid")
        va, wa = self._vis_lists(vis, weights)
        _check(lib().lmg_batch_grid(self._h, ctypes.cast(va, _vp), ctypes.cast(wa, _vp) if wa is not None else None,
                                    ctypes.cast(_ptr_array(out), _vp), _stream()))
        return out

    def degrid(self, grids, out=None):
        import torch
        for c, g in enumerate(grids):
            _need(g, torch.complex64, (self.N[c], self.N[c]), "grid")
        if out is None:
            out = [torch.empty(n, dtype=torch.complex64, device=g.device) for n, g in zip(self.nvis, grids)]
        for c, v in enumerate(out):
            _need(v, torch.complex64, (self.nvis[c],), "vis_out")
        _check(lib().lmg_batch_degrid(self._h, ctypes.cast(_ptr_array(grids), _vp), ctypes.cast(_ptr_array(out), _vp),
                                      _stream()))
        return out

    def dirty_image(self, vis, weights=None, out=None):
        import torch
        if out is None:
            out = [torch.empty((n, n), dtype=torch.complex64, device=v.device) for n, v in zip(self.n_images, vis)]
        for c, g in enumerate(out):
            _need(g, torch.complex64, (self.n_images[c], self.n_images[c]), "image")
        va, wa = self._vis_lists(vis, weights)
        _check(lib().lmg_batch_dirty_image(self._h, ctypes.cast(va, _vp),
                                           ctypes.cast(wa, _vp) if wa is not None else None,
                                           ctypes.cast(_ptr_array(out), _vp), _stream()))
        return out

    def predict_vis(self, images, out=None):
        import torch
        for c, g in enumerate(images):
            _need(g, torch.complex64, (self.n_images[c], self.n_images[c]), "image")
        if out is None:
            out = [torch.empty(n, dtype=torch.complex64, device=g.device) for n, g in zip(self.nvis, images)]
        for c, v in enumerate(out):
            _need(v, torch.complex64, (self.nvis[c],), "vis_out")
        _check(lib().lmg_batch_predict_vis(self._h, ctypes.cast(_ptr_array(images), _vp),
                                           ctypes.cast(_ptr_array(out), _vp), _stream()))
        return out

    def tune(self, vis):
        """Autotuner: returns the chosen (rows per bin, records per item, warps per CTA,
        tables in shared memory) after re-binning with it."""
        va, _ = self._vis_lists(vis, None)
        chosen = (ctypes.c_int * 4)()
        _check(lib().lmg_batch_tune(self._h, ctypes.cast(va, _vp), _stream(), ctypes.cast(chosen, _vp)))
        return tuple(chosen)

    def info(self):
        out = np.zeros(8, dtype=np.int64)
        _check(lib().lmg_batch_info(self._h, out.ctypes.data_as(_vp)))
        keys = ("channels", "w_classes", "size_classes", "nvis", "rows_per_bin", "records_per_item", "warps",
                "graphs_captured")
        return dict(zip(keys, (int(v) for v in out)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.lmg_batch_free(h)
            self._h = None


def _autograd():
    import torch

    class Predict(torch.autograd.Function):
        """V = predict_vis(I) (pad, correct, FFT, degrid); its adjoint, the unweighted
        dirty image, is the backward pass (the gridding sweep)."""

        @staticmethod
        def forward(ctx, image, plan):
            ctx.plan = plan
            ctx.real_input = not image.is_complex()
            img = image.to(plan.cdtype).contiguous()
            return plan.predict_vis(img)

        @staticmethod
        def backward(ctx, grad_vis):
            plan = ctx.plan
            g = plan.dirty_image(grad_vis.to(plan.cdtype).contiguous())
            if ctx.real_input:
                g = g.real.contiguous()
            return g, None

    return Predict


_Predict = None


def predict(image, plan):
    """Differentiable prediction V = P I (torch.autograd); backward runs the gridding path."""
    global _Predict
    if _Predict is None:
        _Predict = _autograd()
    return _Predict.apply(image, plan)

// C ABI of liblmg (include/lmg.h): argument checking, plan state, cuFFT and the launch
// sequences of lmg_dirty_image / lmg_predict_vis.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "kernels.h"
#include "lmg_internal.h"

namespace lmg {
namespace {
thread_local std::string g_error;
}
// Host-side fault injection for tests of the error paths. The environment variable
// LMG_INJECT_FAULT names one failure point; the library then reports that failure in place
// of the call it stands for, without making that call:
//   host_alloc    host allocation of a table object           -> LMG_ENOMEM
//   device_alloc  every device allocation of a plan            -> LMG_ENOMEM
//   cufft_plan    cuFFT plan creation of a plan                -> LMG_ECUFFT
//   item_cap      plans get a work-item capacity of one item, so that the binning of any
//                 input with more than one item exceeds it: the binning's own bounds
//                 check drops the excess and records it in the device status word
//                 (lmg_plan_status -> LMG_EDEVICE)
// Nothing is injected on the GPU itself: no kernel is made to fault or wait.
bool inject_fault(const char* point) {
  const char* v = std::getenv("LMG_INJECT_FAULT");
  return v != nullptr && std::strcmp(v, point) == 0;
}
int set_error(int status, const std::string& msg) {
  g_error = msg;
  return status;
}
void clear_error() { g_error.clear(); }
int cuda_error(cudaError_t e, const char* what) {
  return set_error(LMG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
}  // namespace lmg

using namespace lmg;


namespace {

const char* kVersion = "lmg 0.1 (sm_103a)";


bool check_table_args(int W, double x0, int Ms, int interp, int correction) {
  if (W < 1 || W > kMaxW) return set_error(LMG_EINVAL, "W must be in [1, 16]"), false;
  if (!(x0 > 0.0 && x0 <= 1.0)) return set_error(LMG_EINVAL, "x0 must be in (0, 1]"), false;
  if (Ms < 2 || Ms > 1000000) return set_error(LMG_EINVAL, "oversample must be in [2, 1000000]"), false;
  if (interp < LMG_INTERP_NEAREST || interp > LMG_INTERP_DIRECT)
    return set_error(LMG_EINVAL, "interp must be LMG_INTERP_NEAREST, _LINEAR, _QUADRATIC, _CUBIC or _DIRECT"), false;
  if (interp <= LMG_INTERP_CUBIC && Ms < interp)
    return set_error(LMG_EINVAL, "oversample must be at least the interpolation degree"), false;
  if (correction != LMG_CORR_HOPT && correction != LMG_CORR_INV_C)
    return set_error(LMG_EINVAL, "correction must be LMG_CORR_HOPT or LMG_CORR_INV_C"), false;
  return true;
}

template <typename T> int dalloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (inject_fault("device_alloc"))
    return set_error(LMG_ENOMEM, std::string("device allocation of ") + what + " failed: injected (LMG_INJECT_FAULT)");
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? LMG_ENOMEM : LMG_ECUDA,
                     std::string("device allocation of ") + what + " failed: " + cudaGetErrorString(e));
  }
  return LMG_OK;
}

}  // namespace

namespace lmg {

void free_plan(lmg_plan* p) {
  if (!p) return;
  void* ptrs[] = {p->d_table, p->d_h, p->hist, p->offsets, p->rank, p->partial, p->recs,
                  p->items, p->counters, p->spill, p->frac, p->work, p->model, p->d_tw, p->xform_tmp};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->fft_ok) cufftDestroy(p->fft);
  if (p->fft_pruned_ok) {
    cufftDestroy(p->fft_rows_all);
    cufftDestroy(p->fft_rows_half);
    cufftDestroy(p->fft_cols_all);
    cufftDestroy(p->fft_cols_half);
  }
  delete p;
}

SweepArgs sweep_args(const lmg_plan* p) {
  SweepArgs a{};
  a.recs = p->recs;
  a.offsets = p->offsets;
  a.items = p->items;
  a.counters = p->counters;
  a.table = p->d_table;
  a.Wp = p->Wp;
  a.Ms = p->Ms;
  a.interp = p->interp;
  a.N = static_cast<int>(p->N);
  a.n_strips = p->n_strips;
  a.strip = p->strip;
  a.W = p->W;
  a.dtype = p->dtype;
  a.item_cap = p->item_cap;
  a.nvis = p->nvis;
  a.frac = p->frac;
  return a;
}

}  // namespace lmg

namespace {

int need_binned(const lmg_plan* p) {
  if (p->nvis < 0) return set_error(LMG_EINVAL, "plan has no binned positions (call lmg_plan_bin first)");
  return LMG_OK;
}

// Alignment of device arrays: grids (read and written by the sweeps with 16-byte vector
// accesses) to 16 bytes; images, visibilities and weights to their element size (the
// correction kernels take two pixels per thread only where both arrays allow it).
int need_aligned(const void* q, size_t a, const char* what) {
  if (q && reinterpret_cast<uintptr_t>(q) % a != 0)
    return set_error(LMG_EINVAL, std::string(what) + " must be " + std::to_string(a) + "-byte aligned");
  return LMG_OK;
}
size_t elem_bytes(int dtype) { return dtype == LMG_C128 ? 16 : 8; }
int need_vis_aligned(const lmg_plan* p, const void* vis, const void* weights) {
  const size_t rs = p->dtype == LMG_C128 ? 8 : 4;
  if (int rc = need_aligned(vis, 2 * rs, "visibilities")) return rc;
  return need_aligned(weights, rs, "weights");
}

int launch_status(int rc, const char* what) {
  if (rc != 0) {
    cudaError_t e = cudaGetLastError();
    return set_error(LMG_ECUDA, std::string(what) + " launch failed: " + cudaGetErrorString(e));
  }
  return LMG_OK;
}

int do_grid(lmg_plan* p, const void* vis, const void* weights, int accum, void* grid, cudaStream_t st) {
  SweepArgs a = sweep_args(p);
  a.accum = accum;
  a.vis = vis;
  a.weights = weights;
  a.grid = grid;
  a.spill = p->spill;
  a.grid_blocks = accum ? p->blocks_grid_comp : p->blocks_grid;
  a.warps = p->warps_grid;
  a.table_in_smem = p->tab_smem_grid ? 1 : 0;
  return launch_status(grid_launch(a, st), "gridding");
}

int do_degrid(lmg_plan* p, const void* grid, void* vis_out, cudaStream_t st, bool add = false) {
  SweepArgs a = sweep_args(p);
  a.grid_in = grid;
  a.vis_out = vis_out;
  a.grid_blocks = p->blocks_degrid;
  a.warps = p->warps_degrid;
  a.table_in_smem = p->tab_smem_degrid ? 1 : 0;
  return launch_status(degrid_launch(a, st, !add), "degridding");
}

int do_fft(lmg_plan* p, int direction, void* g, cudaStream_t st) {
  if (cufftSetStream(p->fft, st) != CUFFT_SUCCESS) return set_error(LMG_ECUFFT, "cufftSetStream failed");
  cufftResult r;
  const int dir = direction == LMG_FFT_IMAGE ? CUFFT_INVERSE : CUFFT_FORWARD;
  if (p->dtype == LMG_C128)
    r = cufftExecZ2Z(p->fft, static_cast<cufftDoubleComplex*>(g), static_cast<cufftDoubleComplex*>(g), dir);
  else
    r = cufftExecC2C(p->fft, static_cast<cufftComplex*>(g), static_cast<cufftComplex*>(g), dir);
  if (r != CUFFT_SUCCESS) return set_error(LMG_ECUFFT, "cuFFT execution failed (code " + std::to_string(int(r)) + ")");
  return LMG_OK;
}

// Pruned transforms (Eq. 4 keeps |x| <= x0 / 2 only). The dirty image needs the outputs of
// the kept columns and rows alone: row transforms of every row, then column transforms of
// the n_image kept columns (q mod N in [0, n/2) and [N - n/2, N)). The model grid has
// non-zero input rows only at the kept rows: row transforms of those n_image rows, then
// column transforms of every column. Same sums as the full 2-D transform on the outputs
// that are used; the other outputs of the work grid are left partially transformed.
int exec_1d(lmg_plan* p, cufftHandle h, void* g, size_t offset, int dir, cudaStream_t st) {
  if (cufftSetStream(h, st) != CUFFT_SUCCESS) return set_error(LMG_ECUFFT, "cufftSetStream failed");
  cufftResult r;
  if (p->dtype == LMG_C128) {
    auto* d = static_cast<cufftDoubleComplex*>(g) + offset;
    r = cufftExecZ2Z(h, d, d, dir);
  } else {
    auto* d = static_cast<cufftComplex*>(g) + offset;
    r = cufftExecC2C(h, d, d, dir);
  }
  if (r != CUFFT_SUCCESS) return set_error(LMG_ECUFFT, "cuFFT execution failed (code " + std::to_string(int(r)) + ")");
  return LMG_OK;
}

int fft_image_pruned(lmg_plan* p, void* g, cudaStream_t st) {
  const size_t N = size_t(p->N), half = size_t(p->n_image / 2);
  int rc = exec_1d(p, p->fft_rows_all, g, 0, CUFFT_INVERSE, st);
  if (rc == LMG_OK) rc = exec_1d(p, p->fft_cols_half, g, 0, CUFFT_INVERSE, st);
  if (rc == LMG_OK) rc = exec_1d(p, p->fft_cols_half, g, N - half, CUFFT_INVERSE, st);
  return rc;
}

// Model transform of lmg_predict_vis: rows of the kept rows in place in the model buffer
// (its other rows stay zero), then every column out of place into the work grid.
int fft_model_to_work(lmg_plan* p, cudaStream_t st) {
  const size_t N = size_t(p->N), half = size_t(p->n_image / 2);
  int rc = exec_1d(p, p->fft_rows_half, p->model, 0, CUFFT_FORWARD, st);
  if (rc == LMG_OK) rc = exec_1d(p, p->fft_rows_half, p->model, (N - half) * N, CUFFT_FORWARD, st);
  if (rc != LMG_OK) return rc;
  if (cufftSetStream(p->fft_cols_all, st) != CUFFT_SUCCESS) return set_error(LMG_ECUFFT, "cufftSetStream failed");
  cufftResult r;
  if (p->dtype == LMG_C128)
    r = cufftExecZ2Z(p->fft_cols_all, static_cast<cufftDoubleComplex*>(p->model), static_cast<cufftDoubleComplex*>(p->work),
                     CUFFT_FORWARD);
  else
    r = cufftExecC2C(p->fft_cols_all, static_cast<cufftComplex*>(p->model), static_cast<cufftComplex*>(p->work),
                     CUFFT_FORWARD);
  if (r != CUFFT_SUCCESS) return set_error(LMG_ECUFFT, "cuFFT execution failed (code " + std::to_string(int(r)) + ")");
  return LMG_OK;
}

int fft_model_pruned(lmg_plan* p, void* g, cudaStream_t st) {
  const size_t N = size_t(p->N), half = size_t(p->n_image / 2);
  int rc = exec_1d(p, p->fft_rows_half, g, 0, CUFFT_FORWARD, st);
  if (rc == LMG_OK) rc = exec_1d(p, p->fft_rows_half, g, (N - half) * N, CUFFT_FORWARD, st);
  if (rc == LMG_OK) rc = exec_1d(p, p->fft_cols_all, g, 0, CUFFT_FORWARD, st);
  return rc;
}

// The dirty image from a gridded array (Eq. 4, correction and crop of Eq. 15): the fused
// transform kernels where the plan has them (the grid is left as it is), else the pruned
// library transform in place followed by the crop kernel.
int image_from_grid(lmg_plan* p, void* grid, void* image, void* scratch, cudaStream_t st) {
  if (p->xform)
    return launch_status(xform_image_launch(grid, image, scratch, static_cast<const float*>(p->d_h), p->d_tw,
                                            int(p->n_image), st),
                         "image transform");
  int rc = fft_image_pruned(p, grid, st);
  if (rc == LMG_OK)
    rc = launch_status(crop_correct_launch(grid, image, p->d_h, int(p->n_image), int(p->N), p->dtype, st), "crop");
  return rc;
}

// The model grid from an image (pad and correction, transform of Eq. 2).
int grid_from_image(lmg_plan* p, const void* image, void* grid, void* scratch, cudaStream_t st) {
  if (p->xform)
    return launch_status(xform_model_launch(image, grid, scratch, static_cast<const float*>(p->d_h), p->d_tw,
                                            int(p->n_image), st),
                         "model transform");
  int rc = launch_status(pad_correct_launch(image, grid, p->d_h, int(p->n_image), int(p->N), p->dtype, st), "pad");
  if (rc == LMG_OK) rc = fft_model_pruned(p, grid, st);
  return rc;
}

}  // namespace

namespace lmg {

int plan_create(const lmg_table* t, int64_t n_image, double pixel_scale, int64_t max_vis, int dtype,
                const PlanOptions& opt, lmg_plan** out) {
  if (!out) return set_error(LMG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!t) return set_error(LMG_EINVAL, "table is NULL");
  if (dtype != LMG_C64 && dtype != LMG_C128) return set_error(LMG_EINVAL, "dtype must be LMG_C64 or LMG_C128");
  if (!(pixel_scale > 0.0) || !std::isfinite(pixel_scale)) return set_error(LMG_EINVAL, "pixel_scale must be > 0");
  if (max_vis < 1 || max_vis > (int64_t(1) << 30)) return set_error(LMG_EINVAL, "max_vis must be in [1, 2^30]");
  if (n_image < 2 || (n_image & 1)) return set_error(LMG_EINVAL, "n_image must be even and >= 2");
  const double Nd = double(n_image) / t->x0;
  const int64_t N = int64_t(std::llround(Nd));
  if (std::fabs(Nd - double(N)) > 1e-9 * Nd || (N & 1))
    return set_error(LMG_EINVAL, "n_image / x0 must be an even integer");
  const int strip = strip_width(dtype);
  if (N < 64 || N % strip != 0 || N > 65536)
    return set_error(LMG_EINVAL, "grid size N = n_image / x0 must be a multiple of " + std::to_string(strip) +
                                     " (the strip width of this dtype) in [64, 65536]");
  if (N < 2 * t->W) return set_error(LMG_EINVAL, "grid too small for the support width");

  lmg_plan* p = new (std::nothrow) lmg_plan;
  if (!p) return set_error(LMG_ENOMEM, "host allocation failed");
  p->W = t->W;
  p->Ms = t->Ms;
  p->interp = t->interp;
  p->dtype = dtype;
  p->n_image = n_image;
  p->N = N;
  p->x0 = t->x0;
  p->pixel_scale = pixel_scale;
  p->scale2 = double(N) * pixel_scale * 4294967296.0;
  p->max_vis = max_vis;
  p->strip = strip;
  p->n_strips = int(N / strip);
  const size_t rs = dtype == LMG_C128 ? 8 : 4;
  p->Wp = table_stride(p->W, dtype);
  const int nblk = int((N + opt.min_rows_per_block - 1) / opt.min_rows_per_block);
  p->item_cap = p->n_strips * nblk + int((2 * max_vis) / opt.min_item_target) + 2;
  if (inject_fault("item_cap")) p->item_cap = 1;
  const long long L = (long long)p->n_strips * N;
  p->nchunks = bin_scan_chunks(L);

  int rc;
  cudaError_t e;
  // Device table (rows padded to Wp) and correction factors in the plan's precision.
  std::vector<double> hcorr(static_cast<size_t>(n_image));
  correction_factors(t, n_image, N, dtype == LMG_C64, hcorr.data());
  std::vector<unsigned char> tab_bytes, h_bytes(size_t(n_image) * rs);
  if (t->interp == LMG_INTERP_DIRECT) {
    // direct calculation: the coefficient block takes the place of the table rows
    if (dtype != LMG_C128) {
      delete p;
      return set_error(LMG_EUNSUPPORTED, "LMG_INTERP_DIRECT runs on float64 plans (LMG_C128)");
    }
    std::vector<double> coef;
    if ((rc = direct_coefficients(t, coef)) != LMG_OK) {
      delete p;
      return rc;
    }
    p->Ms = int((coef.size() + size_t(p->Wp) - 1) / size_t(p->Wp)) - 1;
    tab_bytes.assign(size_t(p->Ms + 1) * p->Wp * rs, 0);
    std::memcpy(tab_bytes.data(), coef.data(), coef.size() * sizeof(double));
  } else {
    tab_bytes.assign(size_t(p->Ms + 1) * p->Wp * rs, 0);
    for (int i = 0; i <= p->Ms; ++i)
      for (int j = 0; j < p->W; ++j) {
        const double v = t->C[size_t(i) * p->W + j];
        if (rs == 8) reinterpret_cast<double*>(tab_bytes.data())[size_t(i) * p->Wp + j] = v;
        else reinterpret_cast<float*>(tab_bytes.data())[size_t(i) * p->Wp + j] = float(v);
      }
  }
  for (int64_t q = 0; q < n_image; ++q) {
    if (rs == 8) reinterpret_cast<double*>(h_bytes.data())[q] = hcorr[size_t(q)];
    else reinterpret_cast<float*>(h_bytes.data())[q] = float(hcorr[size_t(q)]);
  }
  // fused kept-field transforms where they apply (complex64, N = 4096; the work and model
  // grids of the plan path then need no separate model grid)
  p->xform = opt.fft && xform_supported(dtype, N, n_image);
  const size_t c2 = 2 * rs;
  if ((rc = dalloc(reinterpret_cast<unsigned char**>(&p->d_table), tab_bytes.size(), "table")) ||
      (rc = dalloc(reinterpret_cast<unsigned char**>(&p->d_h), h_bytes.size(), "correction")) ||
      (rc = dalloc(&p->hist, size_t(L), "histogram")) ||
      (rc = dalloc(&p->offsets, size_t(L) + 1, "offsets")) || (rc = dalloc(&p->rank, size_t(max_vis), "ranks")) ||
      (rc = dalloc(&p->partial, size_t(p->nchunks), "scan")) || (rc = dalloc(&p->recs, size_t(2 * max_vis), "records")) ||
      (rc = dalloc(&p->items, size_t(p->item_cap), "items")) || (rc = dalloc(&p->counters, kNumCounters, "counters")) ||
      (rc = dalloc(reinterpret_cast<unsigned char**>(&p->spill), size_t(p->item_cap) * ring_slots(p->W) * strip * c2, "spill")) ||
      (dtype == LMG_C128 && (rc = dalloc(&p->frac, size_t(max_vis), "quantisation residuals"))) ||
      (opt.work_grid && (rc = dalloc(reinterpret_cast<unsigned char**>(&p->work), size_t(N) * size_t(N) * c2, "work grid"))) ||
      (opt.work_grid && !p->xform &&
       (rc = dalloc(reinterpret_cast<unsigned char**>(&p->model), size_t(N) * size_t(N) * c2, "model grid"))) ||
      (p->xform && (rc = dalloc(reinterpret_cast<unsigned char**>(&p->d_tw), size_t(kXformN) * 8, "twiddles"))) ||
      (p->xform && opt.work_grid &&
       (rc = dalloc(reinterpret_cast<unsigned char**>(&p->xform_tmp), xform_scratch_bytes(n_image), "transform scratch")))) {
    free_plan(p);
    return rc;
  }
  // the device is queried after the allocations (which run on the current device), so
  // that an injected allocation failure is reported before any CUDA call
  if ((e = cudaGetDevice(&p->device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess) {
    free_plan(p);
    return cuda_error(e, "device query");
  }
  std::vector<float> tw;
  if (p->xform) {
    tw.resize(2 * size_t(kXformN));
    for (int k = 0; k < kXformN; ++k) {
      const double a = 2.0 * 3.14159265358979323846 * k / kXformN;
      tw[2 * size_t(k)] = float(std::cos(a));
      tw[2 * size_t(k) + 1] = float(std::sin(a));
    }
  }
  if ((p->xform && (e = cudaMemcpy(p->d_tw, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemcpy(p->d_table, tab_bytes.data(), tab_bytes.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_h, h_bytes.data(), h_bytes.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(p->counters, 0, kNumCounters * sizeof(int))) != cudaSuccess ||
      (p->model && (e = cudaMemset(p->model, 0, size_t(N) * size_t(N) * c2)) != cudaSuccess)) {
    free_plan(p);
    return cuda_error(e, "plan upload");
  }
  // Launch shapes: warps per CTA and table placement that fit shared memory; persistent
  // CTAs per SM from the occupancy calculator.
  const size_t kSmemLimit = 200 * 1024;
  int bps = 0;
  if (sweep_config(p->W, dtype, p->Ms, false, kSmemLimit, &p->tab_smem_grid, &p->warps_grid) ||
      sweep_config(p->W, dtype, p->Ms, true, kSmemLimit, &p->tab_smem_degrid, &p->warps_degrid)) {
    free_plan(p);
    return set_error(LMG_EUNSUPPORTED, "sweep shared memory does not fit for this W and dtype");
  }
  p->smem_grid = sweep_smem_bytes(p->W, dtype, p->Ms, p->tab_smem_grid, false, p->warps_grid);
  p->smem_degrid = sweep_smem_bytes(p->W, dtype, p->Ms, p->tab_smem_degrid, true, p->warps_degrid);
  for (int accum = 0; accum <= (dtype == LMG_C64 ? 1 : 0); ++accum) {
    if (sweep_set_smem_limits(p->W, dtype, accum, p->smem_grid, false, p->interp >= 2) ||
        sweep_occupancy(p->W, dtype, accum, p->smem_grid, false, p->interp >= 2, p->warps_grid, &bps)) {
      free_plan(p);
      return cuda_error(cudaGetLastError(), "sweep kernel attributes");
    }
    (accum ? p->blocks_grid_comp : p->blocks_grid) = p->sms * (bps > 0 ? bps : 1);
  }
  if (sweep_set_smem_limits(p->W, dtype, 0, p->smem_degrid, true, p->interp >= 2) ||
      sweep_occupancy(p->W, dtype, 0, p->smem_degrid, true, p->interp >= 2, p->warps_degrid, &bps)) {
    free_plan(p);
    return cuda_error(cudaGetLastError(), "sweep kernel attributes");
  }
  p->blocks_degrid = p->sms * (bps > 0 ? bps : 1);
  if (p->xform && xform_set_limits() != 0) {
    free_plan(p);
    return cuda_error(cudaGetLastError(), "transform kernel attributes");
  }
  if (opt.fft) {
    if (inject_fault("cufft_plan")) {
      free_plan(p);
      return set_error(LMG_ECUFFT, "cufftPlan2d failed: injected (LMG_INJECT_FAULT)");
    }
    const cufftResult fr = cufftPlan2d(&p->fft, int(N), int(N), dtype == LMG_C128 ? CUFFT_Z2Z : CUFFT_C2C);
    if (fr != CUFFT_SUCCESS) {
      free_plan(p);
      return set_error(fr == CUFFT_ALLOC_FAILED ? LMG_ENOMEM : LMG_ECUFFT,
                       "cufftPlan2d failed (code " + std::to_string(int(fr)) + ")");
    }
    p->fft_ok = true;
    // pruned 1-D batches for the imaging and prediction paths
    int n1 = int(N), half = int(n_image / 2);
    const cufftType ty = dtype == LMG_C128 ? CUFFT_Z2Z : CUFFT_C2C;
    cufftResult r1 = cufftPlanMany(&p->fft_rows_all, 1, &n1, nullptr, 1, n1, nullptr, 1, n1, ty, n1);
    cufftResult r2 = cufftPlanMany(&p->fft_rows_half, 1, &n1, nullptr, 1, n1, nullptr, 1, n1, ty, half);
    cufftResult r3 = cufftPlanMany(&p->fft_cols_all, 1, &n1, &n1, n1, 1, &n1, n1, 1, ty, n1);
    cufftResult r4 = cufftPlanMany(&p->fft_cols_half, 1, &n1, &n1, n1, 1, &n1, n1, 1, ty, half);
    if (r1 != CUFFT_SUCCESS || r2 != CUFFT_SUCCESS || r3 != CUFFT_SUCCESS || r4 != CUFFT_SUCCESS) {
      if (r1 == CUFFT_SUCCESS) cufftDestroy(p->fft_rows_all);
      if (r2 == CUFFT_SUCCESS) cufftDestroy(p->fft_rows_half);
      if (r3 == CUFFT_SUCCESS) cufftDestroy(p->fft_cols_all);
      if (r4 == CUFFT_SUCCESS) cufftDestroy(p->fft_cols_half);
      free_plan(p);
      return set_error(LMG_ECUFFT, "cufftPlanMany failed");
    }
    p->fft_pruned_ok = true;
  }
  *out = p;
  return LMG_OK;
}

int plan_bin(lmg_plan* p, const double* uv, int64_t nvis, cudaStream_t st, int64_t tracks) {
  BinArgs a{};
  a.uv = uv;
  a.tracks = tracks;
  a.nvis = nvis;
  a.scale2 = p->scale2;
  a.W = p->W;
  a.N = int(p->N);
  a.n_strips = p->n_strips;
  a.strip = p->strip;
  a.rows_per_block = p->rows_per_block;
  a.item_target = p->item_target;
  a.item_cap = p->item_cap;
  a.max_blocks = p->sms * 8;
  a.hist = p->hist;
  a.offsets = p->offsets;
  a.rank = p->rank;
  a.partial = p->partial;
  a.recs = p->recs;
  a.items = p->items;
  a.counters = p->counters;
  a.frac = p->frac;
  const int rc = launch_status(bin_launch(a, st), "binning");
  if (rc == LMG_OK) p->nvis = nvis;
  return rc;
}

}  // namespace lmg

extern "C" {

const char* lmg_last_error(void) { return g_error.c_str(); }
const char* lmg_version(void) { return kVersion; }

int lmg_kernel_table(int W, double x0, int oversample, int interp, int correction, lmg_table** out) {
  clear_error();
  if (!out) return set_error(LMG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!check_table_args(W, x0, oversample, interp, correction)) return LMG_EINVAL;
  lmg_table* t = inject_fault("host_alloc") ? nullptr : new (std::nothrow) lmg_table;
  if (!t) return set_error(LMG_ENOMEM, "host allocation of the table failed");
  t->W = W;
  t->x0 = x0;
  t->x0p = 0.5 * x0;
  t->Ms = oversample;
  t->interp = interp;
  t->correction = correction;
  int rc;
  try {
    rc = build_least_misfit(W, t->x0p, oversample, t);
  } catch (const std::bad_alloc&) {
    rc = set_error(LMG_ENOMEM, "host allocation failed");
  }
  if (rc != LMG_OK) {
    delete t;
    return rc;
  }
  *out = t;
  return LMG_OK;
}

int lmg_table_from_values(int W, double x0, int oversample, int interp, int correction, const double* C_host,
                          lmg_table** out) {
  clear_error();
  if (!out) return set_error(LMG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!C_host) return set_error(LMG_EINVAL, "C_host is NULL");
  if (!check_table_args(W, x0, oversample, interp, correction)) return LMG_EINVAL;
  if (interp == LMG_INTERP_DIRECT)
    return set_error(LMG_EINVAL, "LMG_INTERP_DIRECT needs a least-misfit table from lmg_kernel_table");
  lmg_table* t = inject_fault("host_alloc") ? nullptr : new (std::nothrow) lmg_table;
  if (!t) return set_error(LMG_ENOMEM, "host allocation of the table failed");
  t->W = W;
  t->x0 = x0;
  t->x0p = 0.5 * x0;
  t->Ms = oversample;
  t->interp = interp;
  t->correction = correction;
  t->E = std::nan("");
  t->h_nodes.assign(kNg + 1, 0.0);
  try {
    t->C.assign(C_host, C_host + size_t(oversample + 1) * W);
  } catch (const std::bad_alloc&) {
    delete t;
    return set_error(LMG_ENOMEM, "host allocation failed");
  }
  for (double v : t->C)
    if (!std::isfinite(v)) {
      delete t;
      return set_error(LMG_EINVAL, "table values must be finite");
    }
  *out = t;
  return LMG_OK;
}

int lmg_table_free(lmg_table* t) {
  delete t;
  return LMG_OK;
}

int lmg_table_export(const lmg_table* t, double* C_host, size_t nC, double* h_host, size_t nh, double* E,
                     int* info) {
  clear_error();
  if (!t) return set_error(LMG_EINVAL, "table is NULL");
  if (C_host) {
    if (nC < t->C.size()) return set_error(LMG_EINVAL, "C_host capacity too small");
    std::memcpy(C_host, t->C.data(), sizeof(double) * t->C.size());
  }
  if (h_host) {
    if (nh < t->h_nodes.size()) return set_error(LMG_EINVAL, "h_host capacity too small");
    std::memcpy(h_host, t->h_nodes.data(), sizeof(double) * t->h_nodes.size());
  }
  if (E) *E = t->E;
  if (info) {
    info[0] = t->W;
    info[1] = t->Ms;
    info[2] = kNg;
    info[3] = t->iterations;
  }
  return LMG_OK;
}

int lmg_correction_export(const lmg_table* t, int64_t n_image, int single_precision, double* h_host) {
  clear_error();
  if (!t || !h_host) return set_error(LMG_EINVAL, "NULL argument");
  if (n_image < 2 || (n_image & 1)) return set_error(LMG_EINVAL, "n_image must be even and >= 2");
  const double Nd = double(n_image) / t->x0;
  const int64_t N = int64_t(std::llround(Nd));
  if (std::fabs(Nd - double(N)) > 1e-9 * Nd || (N & 1))
    return set_error(LMG_EINVAL, "n_image / x0 must be an even integer");
  correction_factors(t, n_image, N, single_precision != 0, h_host);
  return LMG_OK;
}

int lmg_plan_create(const lmg_table* t, int64_t n_image, double pixel_scale, int64_t max_vis, int dtype,
                    lmg_plan** out) {
  clear_error();
  return plan_create(t, n_image, pixel_scale, max_vis, dtype, PlanOptions{}, out);
}

int lmg_plan_free(lmg_plan* p) {
  free_plan(p);
  return LMG_OK;
}

int lmg_plan_bin(lmg_plan* p, const double* uv, int64_t nvis, void* stream) {
  clear_error();
  if (!p) return set_error(LMG_EINVAL, "plan is NULL");
  if (nvis < 0 || nvis > p->max_vis) return set_error(LMG_EINVAL, "nvis must be in [0, max_vis]");
  if (nvis > 0 && !uv) return set_error(LMG_EINVAL, "uv is NULL");
  if (reinterpret_cast<uintptr_t>(uv) % 16 != 0) return set_error(LMG_EINVAL, "uv must be 16-byte aligned");
  return plan_bin(p, uv, nvis, static_cast<cudaStream_t>(stream));
}

int lmg_plan_bin_tracks(lmg_plan* p, const double* uv, int64_t nvis, int64_t tracks, void* stream) {
  clear_error();
  if (!p) return set_error(LMG_EINVAL, "plan is NULL");
  if (nvis < 0 || nvis > p->max_vis) return set_error(LMG_EINVAL, "nvis must be in [0, max_vis]");
  if (nvis > 0 && !uv) return set_error(LMG_EINVAL, "uv is NULL");
  if (tracks < 1) return set_error(LMG_EINVAL, "tracks must be >= 1");
  if (reinterpret_cast<uintptr_t>(uv) % 16 != 0) return set_error(LMG_EINVAL, "uv must be 16-byte aligned");
  return plan_bin(p, uv, nvis, static_cast<cudaStream_t>(stream), tracks);
}

int lmg_plan_dropped(lmg_plan* p, int64_t* dropped, void* stream) {
  clear_error();
  if (!p || !dropped) return set_error(LMG_EINVAL, "NULL argument");
  int c[8];
  cudaError_t e = cudaMemcpyAsync(c, p->counters, sizeof(c), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "reading counters");
  *dropped = c[kCntBad];
  return LMG_OK;
}

int lmg_plan_info(lmg_plan* p, int64_t* out, void* stream) {
  clear_error();
  if (!p || !out) return set_error(LMG_EINVAL, "NULL argument");
  int c[8];
  cudaError_t e = cudaMemcpyAsync(c, p->counters, sizeof(c), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "reading counters");
  int total = 0;
  if (p->nvis >= 0) {
    e = cudaMemcpy(&total, p->offsets + (long long)p->n_strips * p->N, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "reading offsets");
  }
  out[0] = p->N;
  out[1] = p->n_image;
  out[2] = p->W;
  out[3] = p->nvis;
  out[4] = total;
  out[5] = c[kCntItems] + c[kCntItemsBack];
  out[6] = p->dtype;
  return LMG_OK;
}

void* lmg_work_grid(lmg_plan* p) { return p ? p->work : nullptr; }

int lmg_grid(lmg_plan* p, const void* vis, const void* weights, int accum, void* grid, void* stream) {
  clear_error();
  if (!p || !grid) return set_error(LMG_EINVAL, "NULL argument");
  if (int rc = need_binned(p)) return rc;
  if (p->nvis > 0 && !vis) return set_error(LMG_EINVAL, "vis is NULL");
  if (accum != LMG_ACCUM_PLAIN && accum != LMG_ACCUM_COMPENSATED) return set_error(LMG_EINVAL, "bad accum");
  if (accum == LMG_ACCUM_COMPENSATED && p->dtype != LMG_C64)
    return set_error(LMG_EUNSUPPORTED, "compensated accumulation is for LMG_C64");
  if (int rc = need_aligned(grid, 16, "grid")) return rc;
  if (int rc = need_vis_aligned(p, vis, weights)) return rc;
  return do_grid(p, vis, weights, accum, grid, static_cast<cudaStream_t>(stream));
}

int lmg_degrid(lmg_plan* p, const void* grid, void* vis_out, void* stream) {
  clear_error();
  if (!p || !grid) return set_error(LMG_EINVAL, "NULL argument");
  if (int rc = need_binned(p)) return rc;
  if (p->nvis > 0 && !vis_out) return set_error(LMG_EINVAL, "vis_out is NULL");
  if (int rc = need_aligned(grid, 16, "grid")) return rc;
  if (int rc = need_vis_aligned(p, vis_out, nullptr)) return rc;
  return do_degrid(p, grid, vis_out, static_cast<cudaStream_t>(stream));
}

int lmg_degrid_add(lmg_plan* p, const void* grid, void* vis_inout, void* stream) {
  clear_error();
  if (!p || !grid) return set_error(LMG_EINVAL, "NULL argument");
  if (int rc = need_binned(p)) return rc;
  if (p->nvis > 0 && !vis_inout) return set_error(LMG_EINVAL, "vis_inout is NULL");
  if (int rc = need_aligned(grid, 16, "grid")) return rc;
  if (int rc = need_vis_aligned(p, vis_inout, nullptr)) return rc;
  return do_degrid(p, grid, vis_inout, static_cast<cudaStream_t>(stream), true);
}

int lmg_fft(lmg_plan* p, int direction, void* grid, void* stream) {
  clear_error();
  if (!p || !grid) return set_error(LMG_EINVAL, "NULL argument");
  if (direction != LMG_FFT_IMAGE && direction != LMG_FFT_MODEL) return set_error(LMG_EINVAL, "bad direction");
  if (int rc = need_aligned(grid, 16, "grid")) return rc;
  return do_fft(p, direction, grid, static_cast<cudaStream_t>(stream));
}

int lmg_fft_pruned(lmg_plan* p, int direction, void* grid, void* stream) {
  clear_error();
  if (!p || !grid) return set_error(LMG_EINVAL, "NULL argument");
  if (int rc = need_aligned(grid, 16, "grid")) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (direction == LMG_FFT_IMAGE) return fft_image_pruned(p, grid, st);
  if (direction == LMG_FFT_MODEL) return fft_model_pruned(p, grid, st);
  return set_error(LMG_EINVAL, "bad direction");
}

int lmg_grid_correct(lmg_plan* p, int direction, const void* in, void* out, void* stream) {
  clear_error();
  if (!p || !in || !out) return set_error(LMG_EINVAL, "NULL argument");
  if (int rc = need_aligned(in, elem_bytes(p->dtype), "in")) return rc;
  if (int rc = need_aligned(out, elem_bytes(p->dtype), "out")) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc;
  if (direction == LMG_CROP) rc = crop_correct_launch(in, out, p->d_h, int(p->n_image), int(p->N), p->dtype, st);
  else if (direction == LMG_PAD) rc = pad_correct_launch(in, out, p->d_h, int(p->n_image), int(p->N), p->dtype, st);
  else return set_error(LMG_EINVAL, "direction must be LMG_CROP or LMG_PAD");
  return launch_status(rc, "grid correction");
}

int lmg_dirty_image(lmg_plan* p, const void* vis, const void* weights, int accum, void* image_out, void* stream) {
  clear_error();
  if (!p || !image_out) return set_error(LMG_EINVAL, "NULL argument");
  if (int rc = need_binned(p)) return rc;
  if (!p->work) return set_error(LMG_EINVAL, "plan has no work grid (LMG_PLAN_NO_WORK_GRIDS): use lmg_dirty_image_ws");
  if (p->nvis > 0 && !vis) return set_error(LMG_EINVAL, "vis is NULL");
  if (accum != LMG_ACCUM_PLAIN && accum != LMG_ACCUM_COMPENSATED) return set_error(LMG_EINVAL, "bad accum");
  if (accum == LMG_ACCUM_COMPENSATED && p->dtype != LMG_C64)
    return set_error(LMG_EUNSUPPORTED, "compensated accumulation is for LMG_C64");
  if (int rc = need_aligned(image_out, p->xform ? 16 : elem_bytes(p->dtype), "image")) return rc;
  if (int rc = need_vis_aligned(p, vis, weights)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = do_grid(p, vis, weights, accum, p->work, st);
  if (rc == LMG_OK) rc = image_from_grid(p, p->work, image_out, p->xform_tmp, st);
  return rc;
}

int lmg_predict_vis(lmg_plan* p, const void* image, void* vis_out, void* stream) {
  clear_error();
  if (!p || !image) return set_error(LMG_EINVAL, "NULL argument");
  if (int rc = need_binned(p)) return rc;
  if (!p->work) return set_error(LMG_EINVAL, "plan has no work grids (LMG_PLAN_NO_WORK_GRIDS): use lmg_predict_vis_ws");
  if (p->nvis > 0 && !vis_out) return set_error(LMG_EINVAL, "vis_out is NULL");
  if (int rc = need_aligned(image, p->xform ? 16 : elem_bytes(p->dtype), "image")) return rc;
  if (int rc = need_vis_aligned(p, vis_out, nullptr)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc;
  if (p->xform) {
    rc = launch_status(xform_model_launch(image, p->work, p->xform_tmp, static_cast<const float*>(p->d_h), p->d_tw,
                                          int(p->n_image), st),
                       "model transform");
  } else {
    rc = launch_status(pad_rows_launch(image, p->model, p->d_h, int(p->n_image), int(p->N), p->dtype, st), "pad");
    if (rc == LMG_OK) rc = fft_model_to_work(p, st);
  }
  if (rc == LMG_OK) rc = do_degrid(p, p->work, vis_out, st);
  return rc;
}

int lmg_plan_create_ex(const lmg_table* t, int64_t n_image, double pixel_scale, int64_t max_vis, int dtype, int flags,
                       lmg_plan** out) {
  clear_error();
  if (flags & ~LMG_PLAN_NO_WORK_GRIDS) return set_error(LMG_EINVAL, "unknown plan flags");
  PlanOptions opt{};
  opt.work_grid = (flags & LMG_PLAN_NO_WORK_GRIDS) == 0;
  return plan_create(t, n_image, pixel_scale, max_vis, dtype, opt, out);
}

size_t lmg_workspace_bytes(const lmg_plan* p) {
  if (!p) return 0;
  return size_t(p->N) * size_t(p->N) * (p->dtype == LMG_C128 ? 16 : 8);
}

namespace {
int check_workspace(const lmg_plan* p, const void* ws, size_t ws_bytes) {
  if (!ws) return set_error(LMG_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return set_error(LMG_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < lmg_workspace_bytes(p))
    return set_error(LMG_EINVAL, "workspace too small: lmg_workspace_bytes gives " +
                                     std::to_string(lmg_workspace_bytes(p)) + " bytes");
  if (!p->fft_pruned_ok) return set_error(LMG_EUNSUPPORTED, "plan has no FFT plans");
  return LMG_OK;
}
}  // namespace

int lmg_dirty_image_ws(lmg_plan* p, const void* vis, const void* weights, int accum, void* image_out, void* workspace,
                       size_t ws_bytes, void* stream) {
  clear_error();
  if (!p || !image_out) return set_error(LMG_EINVAL, "NULL argument");
  if (int rc = need_binned(p)) return rc;
  if (int rc = check_workspace(p, workspace, ws_bytes)) return rc;
  if (p->nvis > 0 && !vis) return set_error(LMG_EINVAL, "vis is NULL");
  if (accum != LMG_ACCUM_PLAIN && accum != LMG_ACCUM_COMPENSATED) return set_error(LMG_EINVAL, "bad accum");
  if (accum == LMG_ACCUM_COMPENSATED && p->dtype != LMG_C64)
    return set_error(LMG_EUNSUPPORTED, "compensated accumulation is for LMG_C64");
  if (int rc = need_aligned(image_out, elem_bytes(p->dtype), "image")) return rc;
  if (int rc = need_vis_aligned(p, vis, weights)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = do_grid(p, vis, weights, accum, workspace, st);
  if (rc == LMG_OK) rc = fft_image_pruned(p, workspace, st);
  if (rc == LMG_OK)
    rc = launch_status(crop_correct_launch(workspace, image_out, p->d_h, int(p->n_image), int(p->N), p->dtype, st),
                       "crop");
  return rc;
}

int lmg_predict_vis_ws(lmg_plan* p, const void* image, void* vis_out, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  if (!p || !image) return set_error(LMG_EINVAL, "NULL argument");
  if (int rc = need_binned(p)) return rc;
  if (int rc = check_workspace(p, workspace, ws_bytes)) return rc;
  if (p->nvis > 0 && !vis_out) return set_error(LMG_EINVAL, "vis_out is NULL");
  if (int rc = need_aligned(image, elem_bytes(p->dtype), "image")) return rc;
  if (int rc = need_vis_aligned(p, vis_out, nullptr)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the whole workspace is written (zero outside the kept pixels), then transformed in place
  int rc = launch_status(pad_correct_launch(image, workspace, p->d_h, int(p->n_image), int(p->N), p->dtype, st), "pad");
  if (rc == LMG_OK) rc = fft_model_pruned(p, workspace, st);
  if (rc == LMG_OK) rc = do_degrid(p, workspace, vis_out, st);
  return rc;
}

int lmg_correct_factors(int direction, const void* in, void* out, const void* h, int64_t n_image, int64_t N, int dtype,
                        void* stream) {
  clear_error();
  if (!in || !out || !h) return set_error(LMG_EINVAL, "NULL argument");
  if (n_image < 2 || (n_image & 1) || N < n_image || (N & 1) || N > 65536)
    return set_error(LMG_EINVAL, "need even n_image >= 2 and even N in [n_image, 65536]");
  if (dtype != LMG_C64 && dtype != LMG_C128) return set_error(LMG_EINVAL, "dtype must be LMG_C64 or LMG_C128");
  if (int rc = need_aligned(in, elem_bytes(dtype), "in")) return rc;
  if (int rc = need_aligned(out, elem_bytes(dtype), "out")) return rc;
  if (int rc = need_aligned(h, dtype == LMG_C128 ? 8 : 4, "h")) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc;
  if (direction == LMG_CROP) rc = crop_correct_launch(in, out, h, int(n_image), int(N), dtype, st);
  else if (direction == LMG_PAD) rc = pad_correct_launch(in, out, h, int(n_image), int(N), dtype, st);
  else return set_error(LMG_EINVAL, "direction must be LMG_CROP or LMG_PAD");
  return launch_status(rc, "grid correction");
}

size_t lmg_transform_scratch_bytes(const lmg_plan* p) {
  if (!p || !p->xform) return 0;
  return xform_scratch_bytes(p->n_image);
}

namespace {
int check_transform_args(lmg_plan* p, const void* grid, const void* image, void* scratch) {
  if (!p || !grid || !image) return set_error(LMG_EINVAL, "NULL argument");
  if (!p->fft_pruned_ok) return set_error(LMG_EUNSUPPORTED, "plan has no FFT plans");
  if (int rc = need_aligned(grid, 16, "grid")) return rc;
  // the fused kernels move four pixels (32 bytes) at a time
  if (int rc = need_aligned(image, p->xform ? 16 : elem_bytes(p->dtype), "image")) return rc;
  if (p->xform) {
    if (!scratch && !p->xform_tmp)
      return set_error(LMG_EINVAL, "plan has no transform scratch (LMG_PLAN_NO_WORK_GRIDS): pass one of "
                                   "lmg_transform_scratch_bytes bytes");
    if (int rc = need_aligned(scratch, 16, "scratch")) return rc;
  }
  return LMG_OK;
}
}  // namespace

int lmg_image_from_grid(lmg_plan* p, void* grid, void* image_out, void* scratch, void* stream) {
  clear_error();
  if (int rc = check_transform_args(p, grid, image_out, scratch)) return rc;
  return image_from_grid(p, grid, image_out, scratch ? scratch : p->xform_tmp, static_cast<cudaStream_t>(stream));
}

int lmg_grid_from_image(lmg_plan* p, const void* image, void* grid_out, void* scratch, void* stream) {
  clear_error();
  if (int rc = check_transform_args(p, grid_out, image, scratch)) return rc;
  return grid_from_image(p, image, grid_out, scratch ? scratch : p->xform_tmp, static_cast<cudaStream_t>(stream));
}

int lmg_plan_status(lmg_plan* p, int* status_bits, void* stream) {
  clear_error();
  if (!p) return set_error(LMG_EINVAL, "plan is NULL");
  int c[kNumCounters];
  cudaError_t e = cudaMemcpyAsync(c, p->counters, sizeof(c), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "reading the device status");
  int bits = c[kCntStatus];
  if (static_cast<long long>(c[kCntItems]) + c[kCntItemsBack] > p->item_cap) bits |= kStatusItemOverflow;
  if (status_bits) *status_bits = bits;
  if (bits & kStatusItemOverflow)
    return set_error(LMG_EDEVICE, "binning produced more work items than the plan holds; the excess was dropped");
  if (bits) return set_error(LMG_EDEVICE, "device status " + std::to_string(bits));
  return LMG_OK;
}

}  // extern "C"

// Internal declarations shared by the translation units of liblmg.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cufft.h>

#include "kernels.h"
#include "lmg.h"

namespace lmg {

// Thread-local error message; set_error returns the status for `return set_error(...)`.
int set_error(int status, const std::string& msg);
void clear_error();
// Host-side fault injection (LMG_INJECT_FAULT; see api.cu): true when `point` is named.
bool inject_fault(const char* point);

// Table design parameters (Appendix A node counts).
constexpr int kNg = 32;
constexpr int kMg = 16;
constexpr int kMaxW = 16;

}  // namespace lmg

struct lmg_table {
  int W = 0;
  double x0 = 0.0;      // kept fraction (API convention)
  double x0p = 0.0;     // paper's x0 = x0 / 2
  int Ms = 0;           // oversample
  int interp = 1;
  int correction = 0;
  int iterations = 0;   // optimiser iterations for the final W
  double E = 0.0;       // integrated misfit at the optimum (NaN for caller tables)
  std::vector<double> h_nodes;  // Ng+1 values on [0, x0p]
  std::vector<double> C;        // (Ms+1) x W, row-major
};

namespace lmg {

// Table builder (host float64), table.cpp.
int build_least_misfit(int W, double x0p, int Ms, lmg_table* t);
// Correction factors h(x_p) at x_p = (p - n_image/2) / N from the (optionally
// float32-rounded) table function; table.cpp.
void correction_factors(const lmg_table* t, int64_t n_image, int64_t N, bool single_precision,
                        double* h_out);
// Coefficients of the direct calculation (LMG_INTERP_DIRECT), table.cpp: out[0] = phi =
// 2 pi x0 / Ng, out[1 + a (Ng+1) + k] = alpha[a][k], out[1 + (W + a)(Ng+1) + k] = beta[a][k]
// with C_a(s) = sum_k alpha[a][k] cos(k phi s) + beta[a][k] sin(k phi s).
int direct_coefficients(const lmg_table* t, std::vector<double>& out);
constexpr int kDirectMaxW = 11;

}  // namespace lmg

// Plan state: binned positions of one uv set for one (table, grid size, pixel scale, dtype).
struct lmg_plan {
  int W = 0, Ms = 0, interp = 1, dtype = 0, Wp = 0;
  int64_t n_image = 0, N = 0;
  double x0 = 0, pixel_scale = 0, scale2 = 0;
  // work items: blocks of 64 rows of a strip cut into items of ~512 records (measured best of
  // {64..512} x {256..2048} on the 4.1M-visibility tracks: better balance of the persistent sweeps)
  int n_strips = 0, strip = 64, rows_per_block = 64, item_target = 512, item_cap = 0, nchunks = 0;
  int64_t max_vis = 0, nvis = -1;
  int device = 0, sms = 0;
  int blocks_grid = 0, blocks_degrid = 0;
  bool tab_smem_grid = false, tab_smem_degrid = false;
  int warps_grid = 8, warps_degrid = 8;
  size_t smem_grid = 0, smem_degrid = 0;
  int blocks_grid_comp = 0;
  void* d_table = nullptr;
  void* d_h = nullptr;
  int* hist = nullptr;
  int* offsets = nullptr;
  int2* rank = nullptr;
  int* partial = nullptr;
  lmg::Rec* recs = nullptr;
  lmg::Item* items = nullptr;
  int* counters = nullptr;
  void* spill = nullptr;
  double2* frac = nullptr;   // float64 plans: quantisation residual of every position
  void* work = nullptr;      // N x N work grid (null in batch channels)
  void* model = nullptr;     // N x N model grid of lmg_predict_vis: zero outside the kept rows
  cufftHandle fft = 0;              // full 2-D transform (lmg_fft)
  bool fft_ok = false;
  // pruned transforms of lmg_dirty_image / lmg_predict_vis: 1-D batches over all rows,
  // the n_image / 2 rows at either end, all columns, the n_image / 2 columns at either end
  cufftHandle fft_rows_all = 0, fft_rows_half = 0, fft_cols_all = 0, fft_cols_half = 0;
  bool fft_pruned_ok = false;
  // fused kept-field transforms (complex64, N = 4096): twiddle table e(k / 4096) and the
  // plan's own scratch (N x n_image values; null without work grids)
  bool xform = false;
  void* d_tw = nullptr;
  void* xform_tmp = nullptr;
};

namespace lmg {

// Options of plan creation used by the multi-channel batch: capacities sized for the
// smallest bin parameters the tuner may choose, and no per-plan work grid or FFT plan.
struct PlanOptions {
  int min_rows_per_block = 64;
  int min_item_target = 512;
  bool work_grid = true;
  bool fft = true;
};

int plan_create(const lmg_table* t, int64_t n_image, double pixel_scale, int64_t max_vis, int dtype,
                const PlanOptions& opt, lmg_plan** out);
int plan_bin(lmg_plan* p, const double* uv, int64_t nvis, cudaStream_t st, int64_t tracks = 0);
void free_plan(lmg_plan* p);
SweepArgs sweep_args(const lmg_plan* p);
int cuda_error(cudaError_t e, const char* what);

}  // namespace lmg

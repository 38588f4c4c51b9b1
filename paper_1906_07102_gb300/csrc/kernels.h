// Launch interfaces of the device kernels (host-callable, defined in the .cu files).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lmg {

// Nodes k = 0..Ng of the direct calculation's folded sums (Ng = 32, Appendix A).
constexpr int kDirectNodes = 33;

// Strip width of the binning and the sweeps: one lane per two columns for complex64 (64),
// one lane per column for complex128 (32). dtype 0 = complex64, 1 = complex128.
__host__ __device__ constexpr int strip_width(int dtype) { return dtype ? 32 : 64; }

// Row stride (reals) of a device table: rows start on 16-byte boundaries and take an odd
// number of 16-byte units, so that 16-byte loads of random rows spread over the banks;
// entries W .. stride - 1 are zero.
__host__ __device__ constexpr int table_stride(int W, int dtype) {
  return ((((W * (dtype ? 8 : 4) + 15) / 16) | 1) * 16) / (dtype ? 8 : 4);
}

struct Rec;
struct Item;

// counters[] slots (device ints, reset by bin_launch)
enum {
  kCntBad = 0,         // dropped positions
  kCntItems = 1,       // items placed from the front (heavy)
  kCntStatus = 2,      // device status word: kStatus* bits set by the kernels' own checks
  kCntItemsBack = 3,   // items placed from the back (light)
  kCntGridWork = 4,    // work counter of the gridding sweep
  kCntDegridWork = 5,  // work counter of the degridding sweep
  kNumCounters = 8
};

// Device status bits (counters[kCntStatus]); the host reports them as LMG_EDEVICE.
enum {
  kStatusItemOverflow = 1,  // more work items than the plan's capacity: the excess was dropped
};

struct BinArgs {
  const double* uv;
  long long nvis;
  double scale2;  // N * pixel_scale * 2^32
  int W, N, n_strips, strip;  // strip: columns per strip (strip_width)
  int rows_per_block, item_target, item_cap;
  int max_blocks;
  int* hist;       // n_strips * N
  int* offsets;    // n_strips * N + 1
  int2* rank;      // max_vis: rank of the record(s) in their buckets
  int* partial;    // scan chunk sums
  Rec* recs;       // 2 * max_vis
  Item* items;     // item_cap
  int* counters;   // 8
  double2* frac;   // max_vis or NULL: per visibility (u_q - u, v_q - v) in cells, the residual
                   // of the 2^-32 quantisation (float64 plans: exact table fractions)
  long long tracks;  // > 0: positions ordered k = t * tracks + b (sample t of track b); the
                     // counting and placement passes then follow each track in runs of
                     // samples that share a bucket. 0: no order assumed.
};

// Fused kept-field transforms (fft.cu): complex64 plans with N = kXformN only.
constexpr int kXformN = 4096;
bool xform_supported(int dtype, long long N, long long n);
size_t xform_scratch_bytes(long long n);
int xform_set_limits();
int xform_image_launch(const void* grid, void* image, void* scratch, const float* h, const void* tw, int n,
                       cudaStream_t st);
int xform_model_launch(const void* image, void* grid, void* scratch, const float* h, const void* tw, int n,
                       cudaStream_t st);

int bin_launch(const BinArgs& a, cudaStream_t st);
int bin_scan_chunks(long long L);

struct SweepArgs {
  const Rec* recs;
  const int* offsets;
  const Item* items;
  int* counters;
  const void* table;  // device, (Ms+1) x Wp of the plan's real type
  int Wp, Ms, interp;
  int N, n_strips, strip;
  int W;
  int dtype;          // 0 float, 1 double
  int accum;          // 0 plain, 1 compensated (float only)
  int item_cap;
  int grid_blocks;    // persistent CTAs
  int warps;          // warps per CTA (1..8)
  int table_in_smem;
  // gridding
  const void* vis;
  const void* weights;
  void* grid;
  void* spill;        // item_cap * ring rows * strip complex
  // degridding
  const void* grid_in;
  void* vis_out;
  long long nvis;
  const double2* frac;  // float64 plans: quantisation residuals (BinArgs::frac), else NULL
};

int grid_launch(const SweepArgs& a, cudaStream_t st);
// Rows held in the sweep's rolling ring for support W (spill buffer rows per item).
int ring_slots(int W);
// zero_out: zero the outputs first (else the predictions are added to what is there)
int degrid_launch(const SweepArgs& a, cudaStream_t st, bool zero_out = true);
// Shared memory a sweep CTA needs (bytes) and CTAs per SM that fit; used to size launches.
size_t sweep_smem_bytes(int W, int dtype, int Ms, bool table_in_smem, bool degrid, int warps);
// ext: the kernels of the extended lookups (interp >= 2: Lagrange, direct calculation).
int sweep_set_smem_limits(int W, int dtype, int accum, size_t smem_bytes, bool degrid, bool ext);
int sweep_occupancy(int W, int dtype, int accum, size_t smem_bytes, bool degrid, bool ext, int warps,
                    int* blocks_per_sm);
// Kernel of the extended lookups (sweep_ext.cu).
void* sweep_kernel_ext(int W, int dtype, int accum, bool degrid);
// Warps per CTA and table placement so that a CTA's shared memory stays within `limit`.
int sweep_config(int W, int dtype, int Ms, bool degrid, size_t limit, bool* table_in_smem, int* warps);

// Grid correction (Eqs. 4, 15) and its adjoint.
int crop_correct_launch(const void* F, void* img, const void* h, int n_img, int N, int dtype, cudaStream_t st);
int pad_correct_launch(const void* img, void* P, const void* h, int n_img, int N, int dtype, cudaStream_t st);
// Pad + correct writing only the kept rows of P (the rest must already be zero).
int pad_rows_launch(const void* img, void* P, const void* h, int n_img, int N, int dtype, cudaStream_t st);

}  // namespace lmg

// Multi-channel batches (include/lmg.h, lmg_batch_*): many independent channels, each with
// its own table, grid size, pixel scale and uv set, gridded and degridded together.
//
// Each channel is binned like a single plan (same kernels). The sweeps then run as ONE
// persistent launch per support width W present in the batch (the sweep is specialised on
// W; channels of every grid size and visibility count share it): its warps take work
// indices from one counter, a work index maps through the per-channel prefix of item counts
// to (channel, item), and the item runs the same per-item code as the single-plan sweep.
// Spill rows and the zeroing of degridding outputs run as one launch per W class
// (blockIdx.y = channel); FFTs run as one batched cuFFT plan per distinct grid size. Each operation's launch sequence is
// captured once into a CUDA graph on the batch's own stream and replayed while the caller's
// buffers stay the same. Bin sizes, item sizes, warps per CTA and the table placement are
// chosen by a small autotuner that times the candidates on the caller's data.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "lmg_internal.h"
#include "sweep_body.cuh"

namespace lmg {
namespace {

// Per-channel descriptor of one batch operation (device memory).
struct BatchChan {
  SweepArgs a;
  int tab_off;  // offset (floats) of the channel's table in the shared-memory block, -1: global
  int pad[3];
};

// Per-channel descriptor of the crop / pad pass.
struct BatchImg {
  const float2* src;
  float2* dst;
  const float* h;
  int n_img, N;
};

// Binning results needed to count each channel's work items.
struct BatchMeta {
  const int* counters;
  int item_cap;
  int pad;
};

__device__ __forceinline__ int ring_slots_dev(int W) { return kD * ((W + kD - 1 + kD - 1) / kD); }

// prefix[c] = work items of channels 0 .. c-1 (heavy ones placed from the front, light ones
// from the back of each channel's item array).
__global__ void k_batch_prefix(const BatchMeta* __restrict__ meta, int n_chan, int* __restrict__ prefix) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int s = 0;
  prefix[0] = 0;
  for (int c = 0; c < n_chan; ++c) {
    int nfront;
    s += work_total(meta[c].counters, meta[c].item_cap, nfront);
    prefix[c + 1] = s;
  }
}

// Shared memory of the persistent batch kernels: prefix | tables (optional) | warp stages.
__host__ __device__ inline size_t batch_head_bytes(int n_chan, int tab_floats, int tab_in_smem) {
  return align16(sizeof(int) * size_t(n_chan + 1)) + (tab_in_smem ? align16(sizeof(float) * size_t(tab_floats)) : 0);
}

__device__ __forceinline__ int find_channel(const int* s_prefix, int n_chan, int w) {
  int lo = 0, hi = n_chan;  // s_prefix[lo] <= w < s_prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_prefix[mid] <= w) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Stages the prefix and (optionally) the tables; returns the warp's staging area.
__device__ __forceinline__ unsigned char* batch_stage(unsigned char* smem, const int* __restrict__ prefix, int n_chan,
                                                      const float* __restrict__ tables, int tab_floats, int tab_in_smem,
                                                      size_t warp_bytes) {
  int* s_prefix = reinterpret_cast<int*>(smem);
  for (int i = threadIdx.x; i <= n_chan; i += blockDim.x) s_prefix[i] = prefix[i];
  if (tab_in_smem) {
    float* s_tab = reinterpret_cast<float*>(smem + align16(sizeof(int) * size_t(n_chan + 1)));
    for (int i = threadIdx.x; i < tab_floats; i += blockDim.x) s_tab[i] = tables[i];
  }
  __syncthreads();
  return smem + batch_head_bytes(n_chan, tab_floats, tab_in_smem) + (threadIdx.x >> 5) * warp_bytes;
}

template <int W>
__global__ void __launch_bounds__(kThreads, min_blocks<W, float>())
    k_batch_grid(const BatchChan* __restrict__ ch, const int* __restrict__ prefix, int n_chan, int* work,
                 const float* __restrict__ tables, int tab_floats, int tab_in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  unsigned char* my = batch_stage(smem, prefix, n_chan, tables, tab_floats, tab_in_smem,
                                  Lay<W, float>::grid_bytes);
  const int* s_prefix = reinterpret_cast<const int*>(smem);
  const float* s_tab = reinterpret_cast<const float*>(smem + align16(sizeof(int) * size_t(n_chan + 1)));
  const int total = s_prefix[n_chan];
  for (int w = next_item(work, lane); w < total; w = next_item(work, lane)) {
    const int c = find_channel(s_prefix, n_chan, w);
    const SweepArgs a = ch[c].a;  // the fields the item uses, in registers
    const int toff = ch[c].tab_off;
    const int nfront = min(a.counters[kCntItems], a.item_cap);
    const int slot = item_slot(w - s_prefix[c], nfront, a.item_cap);
    const float* tab = (tab_in_smem && toff >= 0) ? s_tab + toff : static_cast<const float*>(a.table);
    grid_item<W, float, false>(a, tab, my, slot, lane);
  }
}

template <int W>
__global__ void __launch_bounds__(kThreads, min_blocks<W, float>())
    k_batch_degrid(const BatchChan* __restrict__ ch, const int* __restrict__ prefix, int n_chan, int* work,
                   const float* __restrict__ tables, int tab_floats, int tab_in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  unsigned char* my = batch_stage(smem, prefix, n_chan, tables, tab_floats, tab_in_smem,
                                  Lay<W, float>::degrid_bytes);
  const int* s_prefix = reinterpret_cast<const int*>(smem);
  const float* s_tab = reinterpret_cast<const float*>(smem + align16(sizeof(int) * size_t(n_chan + 1)));
  const int total = s_prefix[n_chan];
  for (int w = next_item(work, lane); w < total; w = next_item(work, lane)) {
    const int c = find_channel(s_prefix, n_chan, w);
    const SweepArgs a = ch[c].a;
    const int toff = ch[c].tab_off;
    const int nfront = min(a.counters[kCntItems], a.item_cap);
    const Item item = a.items[item_slot(w - s_prefix[c], nfront, a.item_cap)];
    const float* tab = (tab_in_smem && toff >= 0) ? s_tab + toff : static_cast<const float*>(a.table);
    degrid_item<W, float>(a, tab, my, item, lane);
  }
}

// Spill rows of every channel's items (blockIdx.y = channel).
__global__ void k_batch_spill(const BatchChan* __restrict__ ch) {
  const SweepArgs a = ch[blockIdx.y].a;
  int nfront;
  const int total = work_total(a.counters, a.item_cap, nfront);
  const int RS = ring_slots_dev(a.W);
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int w = gw; w < total; w += (gridDim.x * blockDim.x) >> 5)
    spill_item<float>(a.items, nfront, a.item_cap, a.W, RS, a.N, a.strip, static_cast<const float2*>(a.spill),
                      static_cast<float2*>(a.grid), w, lane);
}

// Zeroes every channel's degridding output before the sweep (blockIdx.y = channel): each
// record adds its partial sum, dropped positions stay zero.
__global__ void k_batch_zero(const BatchChan* __restrict__ ch) {
  const SweepArgs a = ch[blockIdx.y].a;
  float2* out = static_cast<float2*>(a.vis_out);
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < a.nvis; k += stride)
    out[k] = make_float2(0.f, 0.f);
}

// Crop + correct of every channel (blockIdx.y = channel); same arithmetic as the
// single-plan correction (checkerboard for the centring shift).
__global__ void k_batch_crop(const BatchImg* __restrict__ im) {
  const BatchImg d = im[blockIdx.y];
  for (int py = blockIdx.x; py < d.n_img; py += gridDim.x) {
    const int qy = py - d.n_img / 2, sy = qy < 0 ? qy + d.N : qy;
    const float2* src = d.src + static_cast<size_t>(sy) * d.N;
    float2* dst = d.dst + static_cast<size_t>(py) * d.n_img;
    for (int px = threadIdx.x; px < d.n_img; px += blockDim.x) {
      const int qx = px - d.n_img / 2, sx = qx < 0 ? qx + d.N : qx;
      const float2 v = src[sx];
      float f = d.h[px] * d.h[py];
      if ((qx + qy) & 1) f = -f;
      dst[px] = make_float2(f * v.x, f * v.y);
    }
  }
}

// Pad + correct of every channel (blockIdx.y = channel), one grid row per block iteration.
__global__ void k_batch_pad(const BatchImg* __restrict__ im) {
  const BatchImg d = im[blockIdx.y];
  const int half = d.n_img / 2;
  for (int iy = blockIdx.x; iy < d.N; iy += gridDim.x) {
    const int qy = iy < d.N / 2 ? iy : iy - d.N;
    const bool kept_row = qy >= -half && qy < d.n_img - half;
    const int py = qy + half;
    float2* dst = d.dst + static_cast<size_t>(iy) * d.N;
    for (int ix = threadIdx.x; ix < d.N; ix += blockDim.x) {
      const int qx = ix < d.N / 2 ? ix : ix - d.N;
      float2 o = make_float2(0.f, 0.f);
      if (kept_row && qx >= -half && qx < d.n_img - half) {
        const int px = qx + half;
        const float2 v = d.src[static_cast<size_t>(py) * d.n_img + px];
        float f = d.h[px] * d.h[py];
        if ((qx + qy) & 1) f = -f;
        o = make_float2(f * v.x, f * v.y);
      }
      dst[ix] = o;
    }
  }
}

template <int W> void* batch_kernel(bool degrid) {
  return degrid ? reinterpret_cast<void*>(&k_batch_degrid<W>) : reinterpret_cast<void*>(&k_batch_grid<W>);
}

void* batch_kernel_for(int W, bool degrid) {
  switch (W) {
    case 1: return batch_kernel<1>(degrid);
    case 2: return batch_kernel<2>(degrid);
    case 3: return batch_kernel<3>(degrid);
    case 4: return batch_kernel<4>(degrid);
    case 5: return batch_kernel<5>(degrid);
    case 6: return batch_kernel<6>(degrid);
    case 7: return batch_kernel<7>(degrid);
    case 8: return batch_kernel<8>(degrid);
    case 9: return batch_kernel<9>(degrid);
    case 10: return batch_kernel<10>(degrid);
    case 11: return batch_kernel<11>(degrid);
    case 12: return batch_kernel<12>(degrid);
    case 13: return batch_kernel<13>(degrid);
    case 14: return batch_kernel<14>(degrid);
    case 15: return batch_kernel<15>(degrid);
    case 16: return batch_kernel<16>(degrid);
    default: return nullptr;
  }
}

}  // namespace
}  // namespace lmg

// ----------------------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------------------
namespace lmg {
namespace {

enum { kOpGrid = 0, kOpDegrid = 1, kOpDirty = 2, kOpPredict = 3, kNumOps = 4 };

// Channels sharing one support width: one persistent sweep launch.
struct WClass {
  int W = 0;
  std::vector<int> chans;
  std::vector<int> tab_off;        // per member channel, offset of its table in d_tables
  int* d_prefix = nullptr;         // member channels + 1
  BatchMeta* d_meta = nullptr;     // per member channel
  BatchChan* d_desc[kNumOps] = {};  // per operation, per member channel
  float* d_tables = nullptr;       // distinct tables of the members, rows padded to Wp
  int tab_floats = 0;
  bool tab_fits = false;           // small enough to stage in shared memory
  size_t smem[2] = {0, 0};         // grid, degrid
  int blocks[2] = {0, 0};
};

// Channels sharing one grid size: contiguous work grids and the 1-D cuFFT plans of the
// pruned transforms (only the kept field of the image is needed, Eq. 4): every row and
// the kept columns for imaging, the kept rows and every column for prediction. h is half
// the largest kept width of the class's channels (a channel with a narrower field has
// zero rows there, or unused columns, so a wider pruning is still exact).
struct SizeClass {
  int64_t N = 0;
  int64_t h = 0;
  std::vector<int> chans;
  void* work = nullptr;
  cufftHandle rows_all = 0, cols_half = 0, rows_half = 0, cols_all = 0;
  bool fft_ok = false;
};

struct CachedGraph {
  std::vector<uintptr_t> key;
  cudaGraphExec_t exec = nullptr;
};

constexpr size_t kBatchSmemLimit = 200 * 1024;
constexpr size_t kTableSmemLimit = 64 * 1024;

}  // namespace
}  // namespace lmg

struct lmg_batch {
  int n_chan = 0, device = 0, sms = 0;
  std::vector<lmg_plan*> plans;
  std::vector<lmg::WClass> wcls;
  std::vector<lmg::SizeClass> scls;
  std::vector<void*> work;               // per channel work grid (inside its size class)
  lmg::BatchImg* d_img[2] = {nullptr, nullptr};  // crop (dirty image) and pad (predict)
  int* d_work = nullptr;                 // one work counter per W class
  int rows_per_block = 64, item_target = 512, warps = 8, tab_smem = 1;
  std::vector<const double*> uv;         // last binned uv sets (re-binned by the tuner)
  std::vector<int64_t> nvis;
  bool binned = false;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  lmg::CachedGraph graphs[lmg::kNumOps];
  int64_t captures = 0;
};

using namespace lmg;

namespace {

template <typename T> int balloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? LMG_ENOMEM : LMG_ECUDA,
                     std::string("batch: device allocation of ") + what + " failed: " + cudaGetErrorString(e));
  }
  return LMG_OK;
}

void drop_graphs(lmg_batch* b) {
  for (auto& g : b->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.key.clear();
  }
}

void free_batch(lmg_batch* b) {
  if (!b) return;
  if (b->cs) cudaStreamSynchronize(b->cs);
  drop_graphs(b);
  for (auto& k : b->wcls) {
    cudaFree(k.d_prefix);
    cudaFree(k.d_meta);
    cudaFree(k.d_tables);
    for (auto* d : k.d_desc) cudaFree(d);
  }
  for (auto& z : b->scls) {
    if (z.fft_ok) {
      cufftDestroy(z.rows_all);
      cufftDestroy(z.cols_half);
      cufftDestroy(z.rows_half);
      cufftDestroy(z.cols_all);
    }
    cudaFree(z.work);
  }
  cudaFree(b->d_img[0]);
  cudaFree(b->d_img[1]);
  cudaFree(b->d_work);
  for (auto* p : b->plans) free_plan(p);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->cs) cudaStreamDestroy(b->cs);
  delete b;
}

size_t class_smem(const WClass& k, bool degrid, int warps, bool tab_smem) {
  return batch_head_bytes(int(k.chans.size()), k.tab_floats, tab_smem && k.tab_fits) +
         size_t(warps) * stage_bytes(k.W, 0, degrid);
}

// Shared memory and persistent CTA counts of every W class for the current warps / table
// placement (kernel attributes are set here, outside any capture).
int configure(lmg_batch* b) {
  for (auto& k : b->wcls) {
    for (int d = 0; d < 2; ++d) {
      void* kern = batch_kernel_for(k.W, d == 1);
      if (!kern) return set_error(LMG_EUNSUPPORTED, "batch: no sweep kernel for this W");
      k.smem[d] = class_smem(k, d == 1, b->warps, b->tab_smem != 0);
      if (k.smem[d] > kBatchSmemLimit) return set_error(LMG_EUNSUPPORTED, "batch: sweep shared memory too large");
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(k.smem[d]));
      int bps = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 32 * b->warps, k.smem[d]);
      if (e != cudaSuccess) return cuda_error(e, "batch: sweep kernel attributes");
      k.blocks[d] = b->sms * (bps > 0 ? bps : 1);
    }
  }
  return LMG_OK;
}

// Per-channel sweep descriptors of one operation for every W class (synchronous upload).
int fill_sweeps(lmg_batch* b, int op, const void* const* in, const void* const* wts, void* const* out) {
  for (auto& k : b->wcls) {
    std::vector<BatchChan> h(k.chans.size());
    for (size_t j = 0; j < k.chans.size(); ++j) {
      const int c = k.chans[j];
      const lmg_plan* p = b->plans[size_t(c)];
      SweepArgs a = sweep_args(p);
      a.accum = 0;
      a.warps = b->warps;
      a.table_in_smem = (b->tab_smem && k.tab_fits) ? 1 : 0;
      if (op == kOpGrid || op == kOpDirty) {
        a.vis = in[c];
        a.weights = wts ? wts[c] : nullptr;
        a.grid = op == kOpGrid ? out[c] : b->work[size_t(c)];
        a.spill = p->spill;
      } else {
        a.grid_in = op == kOpDegrid ? in[c] : b->work[size_t(c)];
        a.vis_out = out[c];
      }
      h[j].a = a;
      h[j].tab_off = k.tab_off[j];
    }
    cudaError_t e = cudaMemcpy(k.d_desc[op], h.data(), sizeof(BatchChan) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "batch: descriptor upload");
  }
  return LMG_OK;
}

int fill_images(lmg_batch* b, int which, const void* const* src, void* const* dst) {
  std::vector<BatchImg> h(size_t(b->n_chan));
  for (int c = 0; c < b->n_chan; ++c) {
    const lmg_plan* p = b->plans[size_t(c)];
    BatchImg& d = h[size_t(c)];
    d.h = static_cast<const float*>(p->d_h);
    d.n_img = int(p->n_image);
    d.N = int(p->N);
    if (which == 0) {  // crop: work grid -> image
      d.src = static_cast<const float2*>(b->work[size_t(c)]);
      d.dst = static_cast<float2*>(dst[c]);
    } else {           // pad: image -> work grid
      d.src = static_cast<const float2*>(src[c]);
      d.dst = static_cast<float2*>(b->work[size_t(c)]);
    }
  }
  cudaError_t e = cudaMemcpy(b->d_img[which], h.data(), sizeof(BatchImg) * h.size(), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? LMG_OK : cuda_error(e, "batch: descriptor upload");
}

// Launch sequence of the sweeps of one operation: per W class, reset its work counter, the
// persistent sweep (degridding: after zeroing the outputs), then the spill pass (gridding).
int launch_sweeps(lmg_batch* b, int op, cudaStream_t s) {
  const bool degrid = op == kOpDegrid || op == kOpPredict;
  for (size_t i = 0; i < b->wcls.size(); ++i) {
    WClass& k = b->wcls[i];
    const int n = int(k.chans.size());
    const int d = degrid ? 1 : 0;
    cudaError_t e = cudaMemsetAsync(b->d_work + i, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_error(e, "batch: counter reset");
    const BatchChan* ch = k.d_desc[op];
    const int* prefix = k.d_prefix;
    int n_chan = n;
    int* work = b->d_work + i;
    const float* tables = k.d_tables;
    int tab_floats = k.tab_floats;
    int tab_in_smem = (b->tab_smem && k.tab_fits) ? 1 : 0;
    void* params[] = {&ch, &prefix, &n_chan, &work, &tables, &tab_floats, &tab_in_smem};
    if (degrid) k_batch_zero<<<dim3(2 * b->sms, n), 256, 0, s>>>(k.d_desc[op]);
    e = cudaLaunchKernel(batch_kernel_for(k.W, degrid), dim3(k.blocks[d]), dim3(32 * b->warps), params, k.smem[d], s);
    if (e != cudaSuccess) return cuda_error(e, "batch: sweep launch");
    if (!degrid) k_batch_spill<<<dim3(2 * b->sms, n), 256, 0, s>>>(k.d_desc[op]);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "batch: spill / zeroing launch");
  }
  return LMG_OK;
}

int exec_c2c(cufftHandle plan, cufftComplex* d, int dir, cudaStream_t s) {
  if (cufftSetStream(plan, s) != CUFFT_SUCCESS) return set_error(LMG_ECUFFT, "batch: cufftSetStream failed");
  const cufftResult r = cufftExecC2C(plan, d, d, dir);
  if (r != CUFFT_SUCCESS) return set_error(LMG_ECUFFT, "batch: cuFFT execution failed (code " + std::to_string(int(r)) + ")");
  return LMG_OK;
}

// The pruned 2-D transforms of every channel's work grid (in place). Imaging (inverse):
// every row of every channel in one call, then per channel the kept columns, which sit at
// [0, h) and [N - h, N) in the unshifted layout. Prediction (forward): per channel the kept
// rows (the padded model is zero elsewhere), then every column.
int launch_ffts(lmg_batch* b, int dir, cudaStream_t s) {
  for (auto& z : b->scls) {
    auto* w = static_cast<cufftComplex*>(z.work);
    const size_t N = size_t(z.N), h = size_t(z.h), cells = N * N;
    int rc = LMG_OK;
    if (dir == CUFFT_INVERSE) {
      rc = exec_c2c(z.rows_all, w, dir, s);
      for (size_t j = 0; rc == LMG_OK && j < z.chans.size(); ++j) {
        rc = exec_c2c(z.cols_half, w + j * cells, dir, s);
        if (rc == LMG_OK) rc = exec_c2c(z.cols_half, w + j * cells + (N - h), dir, s);
      }
    } else {
      for (size_t j = 0; rc == LMG_OK && j < z.chans.size(); ++j) {
        rc = exec_c2c(z.rows_half, w + j * cells, dir, s);
        if (rc == LMG_OK) rc = exec_c2c(z.rows_half, w + j * cells + (N - h) * N, dir, s);
        if (rc == LMG_OK) rc = exec_c2c(z.cols_all, w + j * cells, dir, s);
      }
    }
    if (rc != LMG_OK) return rc;
  }
  return LMG_OK;
}

// Replays the operation's graph, capturing it first when the caller's buffers changed.
int run_graph(lmg_batch* b, int op, const std::vector<uintptr_t>& key, cudaStream_t user,
              const std::function<int()>& fill, const std::function<int(cudaStream_t)>& record) {
  CachedGraph& g = b->graphs[op];
  cudaError_t e;
  if (!g.exec || g.key != key) {
    // the descriptors are rewritten: nothing of this batch may still be running
    if ((e = cudaStreamSynchronize(b->cs)) != cudaSuccess) return cuda_error(e, "batch: stream synchronisation");
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.key.clear();
    if (int rc = fill()) return rc;
    if ((e = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_error(e, "batch: begin capture");
    const int rc = record(b->cs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cs, &graph);
    if (rc != LMG_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc != LMG_OK ? rc : cuda_error(e, "batch: capturing the launch sequence");
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return cuda_error(e, "batch: graph instantiation");
    }
    g.key = key;
    ++b->captures;
  }
  if ((e = cudaEventRecord(b->ev_in, user)) != cudaSuccess || (e = cudaStreamWaitEvent(b->cs, b->ev_in, 0)) != cudaSuccess ||
      (e = cudaGraphLaunch(g.exec, b->cs)) != cudaSuccess || (e = cudaEventRecord(b->ev_out, b->cs)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(user, b->ev_out, 0)) != cudaSuccess)
    return cuda_error(e, "batch: graph launch");
  return LMG_OK;
}

std::vector<uintptr_t> make_key(int op, int n, std::initializer_list<const void* const*> arrays) {
  std::vector<uintptr_t> key{uintptr_t(op)};
  for (const void* const* arr : arrays)
    for (int c = 0; c < n; ++c) key.push_back(arr ? reinterpret_cast<uintptr_t>(arr[c]) : uintptr_t(1));
  return key;
}

// Pointer arrays of a batch call: non-NULL where needed, and aligned (visibilities and
// weights to their element, grids and images to 16 bytes: the kernels use vector accesses).
int check_ptrs(const lmg_batch* b, const void* const* arr, const char* what, bool need_nonnull_entries,
               size_t align = 8) {
  if (!arr) return set_error(LMG_EINVAL, std::string("batch: ") + what + " is NULL");
  for (int c = 0; c < b->n_chan; ++c) {
    if (need_nonnull_entries && !arr[c] && b->plans[size_t(c)]->nvis > 0)
      return set_error(LMG_EINVAL, std::string("batch: ") + what + "[" + std::to_string(c) + "] is NULL");
    if (arr[c] && reinterpret_cast<uintptr_t>(arr[c]) % align != 0)
      return set_error(LMG_EINVAL, std::string("batch: ") + what + "[" + std::to_string(c) + "] must be " +
                                       std::to_string(align) + "-byte aligned");
  }
  return LMG_OK;
}

int check_arrays(const lmg_batch* b, const void* const* arr, const char* what) {
  if (!arr) return set_error(LMG_EINVAL, std::string("batch: ") + what + " is NULL");
  for (int c = 0; c < b->n_chan; ++c)
    if (!arr[c]) return set_error(LMG_EINVAL, std::string("batch: ") + what + "[" + std::to_string(c) + "] is NULL");
  return check_ptrs(b, arr, what, true, 16);
}

int need_binned(const lmg_batch* b) {
  return b->binned ? LMG_OK : set_error(LMG_EINVAL, "batch: no binned positions (call lmg_batch_bin first)");
}

// Bins every channel with the batch's current bin parameters and counts the work items.
int bin_all(lmg_batch* b, cudaStream_t st) {
  for (int c = 0; c < b->n_chan; ++c) {
    lmg_plan* p = b->plans[size_t(c)];
    p->rows_per_block = b->rows_per_block;
    p->item_target = b->item_target;
    if (int rc = plan_bin(p, b->uv[size_t(c)], b->nvis[size_t(c)], st)) return rc;
  }
  for (auto& k : b->wcls) k_batch_prefix<<<1, 1, 0, st>>>(k.d_meta, int(k.chans.size()), k.d_prefix);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LMG_OK : cuda_error(e, "batch: item count launch");
}

}  // namespace

extern "C" {

int lmg_batch_create(int n_chan, const lmg_table* const* tables, const int64_t* n_image, const double* pixel_scale,
                     const int64_t* max_vis, lmg_batch** out) {
  clear_error();
  if (!out) return set_error(LMG_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_chan < 1 || n_chan > LMG_BATCH_MAX_CHANNELS)
    return set_error(LMG_EINVAL, "n_chan must be in [1, " + std::to_string(LMG_BATCH_MAX_CHANNELS) + "]");
  if (!tables || !n_image || !pixel_scale || !max_vis) return set_error(LMG_EINVAL, "NULL argument");
  for (int c = 0; c < n_chan; ++c) {
    if (!tables[c]) return set_error(LMG_EINVAL, "tables[" + std::to_string(c) + "] is NULL");
    if (tables[c]->interp > LMG_INTERP_LINEAR)
      return set_error(LMG_EUNSUPPORTED, "batches run nearest or linear tables (tables[" + std::to_string(c) + "])");
  }
  lmg_batch* b = new (std::nothrow) lmg_batch;
  if (!b) return set_error(LMG_ENOMEM, "host allocation failed");
  b->n_chan = n_chan;
  b->plans.assign(size_t(n_chan), nullptr);
  b->work.assign(size_t(n_chan), nullptr);
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_error(e, "batch: device query");
  }
  PlanOptions opt;
  opt.min_rows_per_block = 64;
  opt.min_item_target = 256;
  opt.work_grid = false;
  opt.fft = false;
  for (int c = 0; c < n_chan; ++c) {
    const int rc = plan_create(tables[c], n_image[c], pixel_scale[c], max_vis[c], LMG_C64, opt, &b->plans[size_t(c)]);
    if (rc != LMG_OK) {
      const std::string msg = lmg_last_error();
      free_batch(b);
      return set_error(rc, "batch channel " + std::to_string(c) + ": " + msg);
    }
  }
  // W classes: member channels, distinct tables (device copies of the plans' float32 tables)
  std::map<int, size_t> widx;
  for (int c = 0; c < n_chan; ++c) {
    const int W = b->plans[size_t(c)]->W;
    if (!widx.count(W)) {
      widx[W] = b->wcls.size();
      b->wcls.emplace_back();
      b->wcls.back().W = W;
    }
    b->wcls[widx[W]].chans.push_back(c);
  }
  int rc = LMG_OK;
  for (auto& k : b->wcls) {
    const size_t n = k.chans.size();
    std::map<const lmg_table*, int> toff;
    std::vector<int> first_chan;
    for (int c : k.chans) {
      if (!toff.count(tables[c])) {
        toff[tables[c]] = k.tab_floats;
        first_chan.push_back(c);
        const lmg_plan* p = b->plans[size_t(c)];
        k.tab_floats += (p->Ms + 1) * p->Wp;
      }
      k.tab_off.push_back(toff[tables[c]]);
    }
    k.tab_fits = sizeof(float) * size_t(k.tab_floats) <= kTableSmemLimit;
    if ((rc = balloc(&k.d_prefix, n + 1, "item prefix")) || (rc = balloc(&k.d_meta, n, "channel counters")) ||
        (rc = balloc(&k.d_tables, size_t(k.tab_floats), "tables")))
      break;
    for (auto& d : k.d_desc)
      if ((rc = balloc(&d, n, "descriptors"))) break;
    if (rc) break;
    std::vector<BatchMeta> meta(n);
    for (size_t j = 0; j < n; ++j) {
      const lmg_plan* p = b->plans[size_t(k.chans[j])];
      meta[j].counters = p->counters;
      meta[j].item_cap = p->item_cap;
    }
    e = cudaMemcpy(k.d_meta, meta.data(), sizeof(BatchMeta) * n, cudaMemcpyHostToDevice);
    for (size_t t = 0; e == cudaSuccess && t < first_chan.size(); ++t) {
      const lmg_plan* p = b->plans[size_t(first_chan[t])];
      e = cudaMemcpy(k.d_tables + toff[tables[first_chan[t]]], p->d_table, sizeof(float) * size_t(p->Ms + 1) * p->Wp,
                     cudaMemcpyDeviceToDevice);
    }
    if (e != cudaSuccess) {
      rc = cuda_error(e, "batch: table upload");
      break;
    }
  }
  // size classes: contiguous work grids and one batched FFT plan each
  if (rc == LMG_OK) {
    std::map<int64_t, size_t> sidx;
    for (int c = 0; c < n_chan; ++c) {
      const int64_t N = b->plans[size_t(c)]->N;
      if (!sidx.count(N)) {
        sidx[N] = b->scls.size();
        b->scls.emplace_back();
        b->scls.back().N = N;
      }
      b->scls[sidx[N]].chans.push_back(c);
      b->scls[sidx[N]].h = std::max<int64_t>(b->scls[sidx[N]].h, b->plans[size_t(c)]->n_image / 2);
    }
    for (auto& z : b->scls) {
      const size_t cells = size_t(z.N) * size_t(z.N);
      float2* w = nullptr;
      if ((rc = balloc(&w, cells * z.chans.size(), "work grids"))) break;
      z.work = w;
      for (size_t j = 0; j < z.chans.size(); ++j) b->work[size_t(z.chans[j])] = w + j * cells;
      int n1 = int(z.N);
      const int h = int(z.h);
      cufftResult fr = cufftPlanMany(&z.rows_all, 1, &n1, nullptr, 1, n1, nullptr, 1, n1, CUFFT_C2C,
                                     int(z.chans.size()) * n1);
      bool made[4] = {fr == CUFFT_SUCCESS, false, false, false};
      if (fr == CUFFT_SUCCESS) made[1] = (fr = cufftPlanMany(&z.cols_half, 1, &n1, &n1, n1, 1, &n1, n1, 1, CUFFT_C2C, h)) ==
                                         CUFFT_SUCCESS;
      if (fr == CUFFT_SUCCESS) made[2] = (fr = cufftPlanMany(&z.rows_half, 1, &n1, nullptr, 1, n1, nullptr, 1, n1, CUFFT_C2C,
                                                             h)) == CUFFT_SUCCESS;
      if (fr == CUFFT_SUCCESS) made[3] = (fr = cufftPlanMany(&z.cols_all, 1, &n1, &n1, n1, 1, &n1, n1, 1, CUFFT_C2C, n1)) ==
                                         CUFFT_SUCCESS;
      if (fr != CUFFT_SUCCESS) {
        cufftHandle* hs[4] = {&z.rows_all, &z.cols_half, &z.rows_half, &z.cols_all};
        for (int q = 0; q < 4; ++q)
          if (made[q]) cufftDestroy(*hs[q]);
        rc = set_error(fr == CUFFT_ALLOC_FAILED ? LMG_ENOMEM : LMG_ECUFFT,
                       "batch: cufftPlanMany failed (code " + std::to_string(int(fr)) + ")");
        break;
      }
      z.fft_ok = true;
    }
  }
  if (rc == LMG_OK && !((rc = balloc(&b->d_img[0], size_t(n_chan), "image descriptors")) ||
                        (rc = balloc(&b->d_img[1], size_t(n_chan), "image descriptors")) ||
                        (rc = balloc(&b->d_work, b->wcls.size(), "work counters")))) {
    if ((e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess)
      rc = cuda_error(e, "batch: stream / event creation");
  }
  if (rc == LMG_OK) rc = configure(b);
  if (rc != LMG_OK) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return LMG_OK;
}

int lmg_batch_free(lmg_batch* b) {
  free_batch(b);
  return LMG_OK;
}

int lmg_batch_bin(lmg_batch* b, const double* const* uv, const int64_t* nvis, void* stream) {
  clear_error();
  if (!b || !uv || !nvis) return set_error(LMG_EINVAL, "NULL argument");
  for (int c = 0; c < b->n_chan; ++c) {
    const lmg_plan* p = b->plans[size_t(c)];
    if (nvis[c] < 0 || nvis[c] > p->max_vis)
      return set_error(LMG_EINVAL, "batch: nvis[" + std::to_string(c) + "] must be in [0, max_vis]");
    if (nvis[c] > 0 && !uv[c]) return set_error(LMG_EINVAL, "batch: uv[" + std::to_string(c) + "] is NULL");
    if (reinterpret_cast<uintptr_t>(uv[c]) % 16 != 0)
      return set_error(LMG_EINVAL, "batch: uv[" + std::to_string(c) + "] must be 16-byte aligned");
  }
  b->uv.assign(uv, uv + b->n_chan);
  b->nvis.assign(nvis, nvis + b->n_chan);
  for (auto& g : b->graphs) g.key.clear();
  const int rc = bin_all(b, static_cast<cudaStream_t>(stream));
  b->binned = rc == LMG_OK;
  return rc;
}

int lmg_batch_grid(lmg_batch* b, const void* const* vis, const void* const* weights, void* const* grid, void* stream) {
  clear_error();
  if (!b) return set_error(LMG_EINVAL, "batch is NULL");
  if (int rc = need_binned(b)) return rc;
  if (int rc = check_ptrs(b, vis, "vis", true)) return rc;
  if (weights)
    if (int rc = check_ptrs(b, weights, "weights", false, 4)) return rc;
  if (int rc = check_arrays(b, const_cast<const void* const*>(grid), "grid")) return rc;
  const auto key = make_key(kOpGrid, b->n_chan, {vis, weights, const_cast<const void* const*>(grid)});
  return run_graph(
      b, kOpGrid, key, static_cast<cudaStream_t>(stream), [&] { return fill_sweeps(b, kOpGrid, vis, weights, grid); },
      [&](cudaStream_t s) { return launch_sweeps(b, kOpGrid, s); });
}

int lmg_batch_degrid(lmg_batch* b, const void* const* grid, void* const* vis_out, void* stream) {
  clear_error();
  if (!b) return set_error(LMG_EINVAL, "batch is NULL");
  if (int rc = need_binned(b)) return rc;
  if (int rc = check_arrays(b, grid, "grid")) return rc;
  if (int rc = check_ptrs(b, const_cast<const void* const*>(vis_out), "vis_out", true)) return rc;
  const auto key = make_key(kOpDegrid, b->n_chan, {grid, const_cast<const void* const*>(vis_out)});
  return run_graph(
      b, kOpDegrid, key, static_cast<cudaStream_t>(stream),
      [&] { return fill_sweeps(b, kOpDegrid, grid, nullptr, vis_out); },
      [&](cudaStream_t s) { return launch_sweeps(b, kOpDegrid, s); });
}

int lmg_batch_dirty_image(lmg_batch* b, const void* const* vis, const void* const* weights, void* const* image,
                          void* stream) {
  clear_error();
  if (!b) return set_error(LMG_EINVAL, "batch is NULL");
  if (int rc = need_binned(b)) return rc;
  if (int rc = check_ptrs(b, vis, "vis", true)) return rc;
  if (weights)
    if (int rc = check_ptrs(b, weights, "weights", false, 4)) return rc;
  if (int rc = check_arrays(b, const_cast<const void* const*>(image), "image")) return rc;
  const auto key = make_key(kOpDirty, b->n_chan, {vis, weights, const_cast<const void* const*>(image)});
  return run_graph(
      b, kOpDirty, key, static_cast<cudaStream_t>(stream),
      [&] {
        int rc = fill_sweeps(b, kOpDirty, vis, weights, nullptr);
        return rc ? rc : fill_images(b, 0, nullptr, image);
      },
      [&](cudaStream_t s) {
        int rc = launch_sweeps(b, kOpDirty, s);
        if (rc == LMG_OK) rc = launch_ffts(b, CUFFT_INVERSE, s);
        if (rc == LMG_OK) {
          k_batch_crop<<<dim3(256, b->n_chan), 256, 0, s>>>(b->d_img[0]);
          cudaError_t e = cudaGetLastError();
          if (e != cudaSuccess) rc = cuda_error(e, "batch: crop launch");
        }
        return rc;
      });
}

int lmg_batch_predict_vis(lmg_batch* b, const void* const* image, void* const* vis_out, void* stream) {
  clear_error();
  if (!b) return set_error(LMG_EINVAL, "batch is NULL");
  if (int rc = need_binned(b)) return rc;
  if (int rc = check_arrays(b, image, "image")) return rc;
  if (int rc = check_ptrs(b, const_cast<const void* const*>(vis_out), "vis_out", true)) return rc;
  const auto key = make_key(kOpPredict, b->n_chan, {image, const_cast<const void* const*>(vis_out)});
  return run_graph(
      b, kOpPredict, key, static_cast<cudaStream_t>(stream),
      [&] {
        int rc = fill_images(b, 1, image, nullptr);
        return rc ? rc : fill_sweeps(b, kOpPredict, nullptr, nullptr, vis_out);
      },
      [&](cudaStream_t s) {
        k_batch_pad<<<dim3(512, b->n_chan), 256, 0, s>>>(b->d_img[1]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "batch: pad launch");
        int rc = launch_ffts(b, CUFFT_FORWARD, s);
        return rc == LMG_OK ? launch_sweeps(b, kOpPredict, s) : rc;
      });
}

int lmg_batch_tune(lmg_batch* b, const void* const* vis, void* stream, int* chosen) {
  clear_error();
  if (!b) return set_error(LMG_EINVAL, "batch is NULL");
  if (int rc = need_binned(b)) return rc;
  if (int rc = check_ptrs(b, vis, "vis", true)) return rc;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->cs);
  if (e != cudaSuccess) return cuda_error(e, "batch: stream synchronisation");
  int64_t total = 0;
  for (int64_t n : b->nvis) total += n;
  float2* scratch = nullptr;
  if (int rc = balloc(&scratch, size_t(total), "tuning output")) return rc;
  std::vector<void*> outs(size_t(b->n_chan));
  int64_t off = 0;
  for (int c = 0; c < b->n_chan; ++c) {
    outs[size_t(c)] = scratch + off;
    off += b->nvis[size_t(c)];
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  bool any_fits = false;
  for (auto& k : b->wcls) any_fits = any_fits || k.tab_fits;

  // gridding + degridding time of one candidate (best of three after one warm-up)
  auto measure = [&](int rows, int target, int warps, int ts, float* ms) -> int {
    b->rows_per_block = rows;
    b->item_target = target;
    b->warps = warps;
    b->tab_smem = ts;
    int rc = bin_all(b, b->cs);
    if (rc == LMG_OK) rc = configure(b);
    if (rc == LMG_OK) rc = fill_sweeps(b, kOpDirty, vis, nullptr, nullptr);
    if (rc == LMG_OK) rc = fill_sweeps(b, kOpPredict, nullptr, nullptr, outs.data());
    *ms = 1e30f;
    for (int rep = 0; rc == LMG_OK && rep < 4; ++rep) {
      cudaEventRecord(t0, b->cs);
      rc = launch_sweeps(b, kOpDirty, b->cs);
      if (rc == LMG_OK) rc = launch_sweeps(b, kOpPredict, b->cs);
      cudaEventRecord(t1, b->cs);
      cudaError_t ee = cudaEventSynchronize(t1);
      if (ee != cudaSuccess) return cuda_error(ee, "batch: tuning run");
      float t = 0.f;
      cudaEventElapsedTime(&t, t0, t1);
      if (rep > 0) *ms = std::min(*ms, t);
    }
    return rc;
  };
  const int rows_c[] = {64, 128, 256, 512}, target_c[] = {256, 512, 1024, 2048};
  int best[4] = {256, 1024, 8, any_fits ? 1 : 0};
  float best_ms = 1e30f, ms = 0.f;
  int rc = LMG_OK;
  for (int r : rows_c)
    for (int tg : target_c) {
      if (rc != LMG_OK) break;
      rc = measure(r, tg, 8, best[3], &ms);
      if (rc == LMG_OK && ms < best_ms) {
        best_ms = ms;
        best[0] = r;
        best[1] = tg;
      }
    }
  for (int w : {4, 8})
    for (int ts = 0; ts <= (any_fits ? 1 : 0); ++ts) {
      if (rc != LMG_OK) break;
      rc = measure(best[0], best[1], w, ts, &ms);
      if (rc == LMG_OK && ms < best_ms) {
        best_ms = ms;
        best[2] = w;
        best[3] = ts;
      }
    }
  if (rc == LMG_OK) {
    b->rows_per_block = best[0];
    b->item_target = best[1];
    b->warps = best[2];
    b->tab_smem = best[3];
    rc = bin_all(b, b->cs);
    if (rc == LMG_OK) rc = configure(b);
  }
  e = cudaStreamSynchronize(b->cs);
  if (rc == LMG_OK && e != cudaSuccess) rc = cuda_error(e, "batch: tuning");
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(scratch);
  for (auto& g : b->graphs) g.key.clear();
  if (rc == LMG_OK && chosen)
    for (int i = 0; i < 4; ++i) chosen[i] = best[i];
  return rc;
}

int lmg_batch_info(lmg_batch* b, int64_t* out) {
  clear_error();
  if (!b || !out) return set_error(LMG_EINVAL, "NULL argument");
  int64_t total = 0;
  for (int64_t n : b->nvis) total += n;
  out[0] = b->n_chan;
  out[1] = int64_t(b->wcls.size());
  out[2] = int64_t(b->scls.size());
  out[3] = b->binned ? total : -1;
  out[4] = b->rows_per_block;
  out[5] = b->item_target;
  out[6] = b->warps;
  out[7] = b->captures;
  return LMG_OK;
}

}  // extern "C"

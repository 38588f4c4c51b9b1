// Gridding and degridding sweeps (Eqs. 5-6 and their transpose, Section 4).
//
// The grid is cut into 32-column strips; a warp owns one work item (a range of rows of
// one strip) and lane t owns column t of the strip. Records of the item are visited row
// by row (support-start row), in batches of 32:
//   1. lane l computes the 2W table weights of record l (Section 5.1 lookup) and stages
//      them in shared memory with the record's first column;
//   2. each lane builds the set of records whose support covers its column (32x32 bit
//      transpose of the per-record cover masks);
//   3. gridding: lane t adds Cv_j * (Cu_i w V) into W rolling row accumulators held in
//      registers (row r + j goes to slot (r - r0 + j) mod W, a compile-time index);
//      when the sweep leaves row r, that row is final and is stored with one coalesced
//      256-byte (complex64) store. Rows r1 .. r1+W-2 are written to a spill buffer and
//      added by k_grid_spill after all items have stored their rows.
//      degridding: lane t keeps the W grid rows r .. r+W-1 of its column in registers,
//      forms sum_j Cv_j G[r+j][t] times Cu_i for each covering record, stages it, and
//      lane l sums its record's W partials.
// Every grid cell is written exactly once by the gridding sweep (no pre-zeroing, no
// atomics except the spill rows).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace lmg {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <typename R> __host__ __device__ constexpr int wpad(int W) {
  return sizeof(R) == 4 ? ((W + 3) & ~3) : ((W + 1) & ~1);
}

template <int W, typename R> struct Stage {
  static constexpr int Wp = wpad<R>(W);
  // per warp: x0[32] | cv[32][Wp] | cu[32][Wp] (degrid) | a[32][W] complex
  static constexpr size_t x0_bytes = 32 * sizeof(int);
  static constexpr size_t cv_bytes = 32 * Wp * sizeof(R);
  static constexpr size_t a_bytes = 32 * W * 2 * sizeof(R);
  static constexpr size_t grid_bytes = x0_bytes + cv_bytes + a_bytes;
  static constexpr size_t degrid_bytes = x0_bytes + 2 * cv_bytes + a_bytes;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <int W, typename R>
__device__ __forceinline__ void load_row(const R* __restrict__ p, R (&v)[W]) {
  constexpr int Wp = wpad<R>(W);
  if constexpr (sizeof(R) == 4 && Wp % 4 == 0) {
    float tmp[Wp];
#pragma unroll
    for (int q = 0; q < Wp / 4; ++q) {
      const float4 f = reinterpret_cast<const float4*>(p)[q];
      tmp[4 * q] = f.x; tmp[4 * q + 1] = f.y; tmp[4 * q + 2] = f.z; tmp[4 * q + 3] = f.w;
    }
#pragma unroll
    for (int j = 0; j < W; ++j) v[j] = tmp[j];
  } else {
#pragma unroll
    for (int j = 0; j < W; ++j) v[j] = p[j];
  }
}

// Copy the table into shared memory (all threads of the CTA), or use it in place.
template <typename R>
__device__ __forceinline__ const R* stage_table(const SweepArgs& a, unsigned char* smem) {
  const R* g = static_cast<const R*>(a.table);
  if (!a.table_in_smem) return g;
  R* s = reinterpret_cast<R*>(smem);
  const int n = (a.Ms + 1) * a.Wp;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = g[i];
  __syncthreads();
  return s;
}

__device__ __forceinline__ int next_item(int* counter, int lane) {
  int it = 0;
  if (lane == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, it, 0);
}

// Window of 32 row offsets: lane l holds off[wbase + l] and off[wbase + l + 1].
struct RowWindow {
  int wbase, lo, hi;
  __device__ __forceinline__ void load(const int* __restrict__ off, int base, int N, int lane) {
    wbase = base;
    lo = off[min(base + lane, N)];
    hi = off[min(base + lane + 1, N)];
  }
  __device__ __forceinline__ void range(const int* __restrict__ off, int row, int N, int lane, int& beg, int& end) {
    if (row - wbase >= 32) load(off, row, N, lane);
    beg = __shfl_sync(0xffffffffu, lo, row - wbase);
    end = __shfl_sync(0xffffffffu, hi, row - wbase);
  }
};

template <typename R> struct Acc2 { R re, im; };

// Error-free addition s + e = a + b (Knuth TwoSum); a receives s, lo accumulates e.
__device__ __forceinline__ void two_sum_acc(float& a, float& lo, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  lo += __fsub_rn(a, ap) + __fsub_rn(b, bp);
  a = s;
}

template <int W, typename R, bool COMP>
__global__ void __launch_bounds__(kThreads) k_grid_sweep(const SweepArgs a) {
  using C2 = typename Cplx<R>::T;
  using St = Stage<W, R>;
  constexpr int Wp = St::Wp;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const R* tab = stage_table<R>(a, smem);
  const size_t tab_bytes = a.table_in_smem ? align16(size_t(a.Ms + 1) * a.Wp * sizeof(R)) : 0;
  unsigned char* my = smem + tab_bytes + warp * align16(St::grid_bytes);
  int* s_x0 = reinterpret_cast<int*>(my);
  R* s_cv = reinterpret_cast<R*>(my + St::x0_bytes);
  C2* s_a = reinterpret_cast<C2*>(my + St::x0_bytes + St::cv_bytes);

  const Rec* __restrict__ recs = a.recs;
  const C2* __restrict__ vis = static_cast<const C2*>(a.vis);
  const R* __restrict__ wts = static_cast<const R*>(a.weights);
  C2* __restrict__ grid = static_cast<C2*>(a.grid);
  C2* __restrict__ spill = static_cast<C2*>(a.spill);
  const int N = a.N;
  const int n_items = min(a.counters[kCntItems], a.item_cap);

  for (int it = next_item(a.counters + kCntGridWork, lane); it < n_items;
       it = next_item(a.counters + kCntGridWork, lane)) {
    const Item item = a.items[it];
    const int* __restrict__ off = a.offsets + static_cast<long long>(item.strip) * N;
    const int col = item.strip * kStrip + lane;
    R acc_re[W], acc_im[W], lo_re[W], lo_im[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc_re[q] = acc_im[q] = lo_re[q] = lo_im[q] = R(0);
    RowWindow win;
    win.load(off, item.r0, N, lane);
    for (int rbase = item.r0; rbase < item.r1; rbase += W) {
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int row = rbase + u;
        if (row < item.r1) {
          int beg, end;
          win.range(off, row, N, lane, beg, end);
          for (int b0 = beg; b0 < end; b0 += 32) {
            const int nrec = min(32, end - b0);
            unsigned cover = 0u;
            if (lane < nrec) {
              const Rec rc = recs[b0 + lane];
              R cu[W], cv[W];
              table_weights<W, R>(tab, Wp, a.Ms, a.interp, rc.su, cu);
              table_weights<W, R>(tab, Wp, a.Ms, a.interp, rc.sv, cv);
              C2 v = vis[rc.idx];
              if (wts != nullptr) {
                const R w = wts[rc.idx];
                v.x *= w;
                v.y *= w;
              }
              s_x0[lane] = rc.xrel;
#pragma unroll
              for (int j = 0; j < W; ++j) s_cv[lane * Wp + j] = cv[j];
#pragma unroll
              for (int i = 0; i < W; ++i) {
                C2 t;
                t.x = cu[i] * v.x;
                t.y = cu[i] * v.y;
                s_a[lane * W + i] = t;
              }
              cover = cover_mask(rc.xrel, W);
            }
            __syncwarp();
            unsigned M = transpose32(cover, lane);
            while (M) {
              const int l = __ffs(M) - 1;
              M &= M - 1u;
              const C2 ai = s_a[l * W + (lane - s_x0[l])];
              R cvl[W];
              load_row<W, R>(s_cv + l * Wp, cvl);
#pragma unroll
              for (int j = 0; j < W; ++j) {
                const int q = (u + j) % W;
                if constexpr (COMP) {
                  two_sum_acc(acc_re[q], lo_re[q], cvl[j] * ai.x);
                  two_sum_acc(acc_im[q], lo_im[q], cvl[j] * ai.y);
                } else {
                  acc_re[q] = fma(cvl[j], ai.x, acc_re[q]);
                  acc_im[q] = fma(cvl[j], ai.y, acc_im[q]);
                }
              }
            }
            __syncwarp();
          }
          // row `row` is complete: store it and recycle its slot
          C2 o;
          if constexpr (COMP) {
            o.x = acc_re[u] + lo_re[u];
            o.y = acc_im[u] + lo_im[u];
          } else {
            o.x = acc_re[u];
            o.y = acc_im[u];
          }
          grid[static_cast<size_t>(row) * N + col] = o;
          acc_re[u] = acc_im[u] = lo_re[u] = lo_im[u] = R(0);
        }
      }
    }
    // spill rows r1 .. r1+W-2 (slot q holds row r1 + ((q - (r1-r0)) mod W))
    C2* sp = spill + static_cast<size_t>(it) * W * kStrip;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      C2 o;
      if constexpr (COMP) {
        o.x = acc_re[q] + lo_re[q];
        o.y = acc_im[q] + lo_im[q];
      } else {
        o.x = acc_re[q];
        o.y = acc_im[q];
      }
      sp[q * kStrip + lane] = o;
    }
  }
}

// Adds each item's spill rows into the grid (after every item stored its own rows).
template <typename R>
__global__ void k_grid_spill(const Item* __restrict__ items, const int* __restrict__ counters, int item_cap,
                             int W, int N, const typename Cplx<R>::T* __restrict__ spill,
                             typename Cplx<R>::T* __restrict__ grid) {
  const int n_items = min(counters[kCntItems], item_cap);
  const long long gw = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long total = static_cast<long long>(n_items) * W;
  for (long long w = gw; w < total; w += (static_cast<long long>(gridDim.x) * blockDim.x) >> 5) {
    const int it = static_cast<int>(w / W), q = static_cast<int>(w % W);
    const Item item = items[it];
    if (item.r1 <= item.r0) continue;
    const int u_end = (item.r1 - item.r0) % W;
    const int j = (q - u_end + W) % W;
    if (j > W - 2) continue;
    const int row = (item.r1 + j) % N;
    const auto v = spill[(static_cast<size_t>(it) * W + q) * kStrip + lane];
    red_add(grid + static_cast<size_t>(row) * N + item.strip * kStrip + lane, v);
  }
}

template <int W, typename R>
__global__ void __launch_bounds__(kThreads) k_degrid_sweep(const SweepArgs a) {
  using C2 = typename Cplx<R>::T;
  using St = Stage<W, R>;
  constexpr int Wp = St::Wp;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const R* tab = stage_table<R>(a, smem);
  const size_t tab_bytes = a.table_in_smem ? align16(size_t(a.Ms + 1) * a.Wp * sizeof(R)) : 0;
  unsigned char* my = smem + tab_bytes + warp * align16(St::degrid_bytes);
  int* s_x0 = reinterpret_cast<int*>(my);
  R* s_cv = reinterpret_cast<R*>(my + St::x0_bytes);
  R* s_cu = reinterpret_cast<R*>(my + St::x0_bytes + St::cv_bytes);
  C2* s_p = reinterpret_cast<C2*>(my + St::x0_bytes + 2 * St::cv_bytes);

  const Rec* __restrict__ recs = a.recs;
  const C2* __restrict__ G = static_cast<const C2*>(a.grid_in);
  C2* __restrict__ out = static_cast<C2*>(a.vis_out);
  C2* __restrict__ dpart = static_cast<C2*>(a.dpart);
  const int N = a.N;
  const int n_items = min(a.counters[kCntItems], a.item_cap);

  for (int it = next_item(a.counters + kCntDegridWork, lane); it < n_items;
       it = next_item(a.counters + kCntDegridWork, lane)) {
    const Item item = a.items[it];
    const int* __restrict__ off = a.offsets + static_cast<long long>(item.strip) * N;
    if (item.r1 <= item.r0 || off[item.r0] == off[item.r1]) continue;
    const int col = item.strip * kStrip + lane;
    R g_re[W], g_im[W];
#pragma unroll
    for (int j = 0; j < W - 1; ++j) {
      const C2 v = G[static_cast<size_t>((item.r0 + j) % N) * N + col];
      g_re[j] = v.x;
      g_im[j] = v.y;
    }
    RowWindow win;
    win.load(off, item.r0, N, lane);
    for (int rbase = item.r0; rbase < item.r1; rbase += W) {
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int row = rbase + u;
        if (row < item.r1) {
          {
            const C2 v = G[static_cast<size_t>((row + W - 1) % N) * N + col];
            g_re[(u + W - 1) % W] = v.x;
            g_im[(u + W - 1) % W] = v.y;
          }
          int beg, end;
          win.range(off, row, N, lane, beg, end);
          for (int b0 = beg; b0 < end; b0 += 32) {
            const int nrec = min(32, end - b0);
            unsigned cover = 0u;
            Rec rc{0u, 0, 0u, 0u};
            if (lane < nrec) {
              rc = recs[b0 + lane];
              R cu[W], cv[W];
              table_weights<W, R>(tab, Wp, a.Ms, a.interp, rc.su, cu);
              table_weights<W, R>(tab, Wp, a.Ms, a.interp, rc.sv, cv);
              s_x0[lane] = rc.xrel;
#pragma unroll
              for (int j = 0; j < W; ++j) {
                s_cv[lane * Wp + j] = cv[j];
                s_cu[lane * Wp + j] = cu[j];
              }
              cover = cover_mask(rc.xrel, W);
            }
            __syncwarp();
            unsigned M = transpose32(cover, lane);
            while (M) {
              const int l = __ffs(M) - 1;
              M &= M - 1u;
              const int i = lane - s_x0[l];
              R cvl[W];
              load_row<W, R>(s_cv + l * Wp, cvl);
              R sr = R(0), si = R(0);
#pragma unroll
              for (int j = 0; j < W; ++j) {
                const int q = (u + j) % W;
                sr = fma(cvl[j], g_re[q], sr);
                si = fma(cvl[j], g_im[q], si);
              }
              const R c = s_cu[l * Wp + i];
              C2 p;
              p.x = c * sr;
              p.y = c * si;
              s_p[l * W + i] = p;
            }
            __syncwarp();
            if (lane < nrec) {
              const int i0 = max(0, -rc.xrel), i1 = min(W, kStrip - rc.xrel);
              R vr = R(0), vi = R(0);
              for (int i = i0; i < i1; ++i) {
                const C2 p = s_p[lane * W + i];
                vr += p.x;
                vi += p.y;
              }
              C2 o;
              o.x = vr;
              o.y = vi;
              if (rc.xrel >= 0) out[rc.idx] = o;
              else dpart[rc.idx] = o;
            }
            __syncwarp();
          }
        }
      }
    }
  }
}

// Adds the partial sums of secondary records (supports crossing a strip boundary) and
// zeroes the outputs of dropped positions.
template <typename R>
__global__ void k_degrid_fixup(const int* __restrict__ dup_list, const int* __restrict__ bad_list,
                               const int* __restrict__ counters, const typename Cplx<R>::T* __restrict__ dpart,
                               typename Cplx<R>::T* __restrict__ out) {
  const int n_dup = counters[kCntSecondary], n_bad = counters[kCntBad];
  const int stride = gridDim.x * blockDim.x;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_dup + n_bad; m += stride) {
    if (m < n_dup) {
      const int k = dup_list[m];
      auto v = out[k];
      const auto p = dpart[k];
      v.x += p.x;
      v.y += p.y;
      out[k] = v;
    } else {
      typename Cplx<R>::T z;
      z.x = 0;
      z.y = 0;
      out[bad_list[m - n_dup]] = z;
    }
  }
}

template <int W, typename R, bool COMP> void* grid_kernel_ptr() {
  return reinterpret_cast<void*>(&k_grid_sweep<W, R, COMP>);
}
template <int W, typename R> void* degrid_kernel_ptr() {
  return reinterpret_cast<void*>(&k_degrid_sweep<W, R>);
}

template <int W> void* pick_kernel(int dtype, int accum, bool degrid) {
  if (degrid) return dtype ? degrid_kernel_ptr<W, double>() : degrid_kernel_ptr<W, float>();
  if (dtype) return grid_kernel_ptr<W, double, false>();
  return accum ? grid_kernel_ptr<W, float, true>() : grid_kernel_ptr<W, float, false>();
}

void* kernel_for(int W, int dtype, int accum, bool degrid) {
  switch (W) {
    case 1: return pick_kernel<1>(dtype, accum, degrid);
    case 2: return pick_kernel<2>(dtype, accum, degrid);
    case 3: return pick_kernel<3>(dtype, accum, degrid);
    case 4: return pick_kernel<4>(dtype, accum, degrid);
    case 5: return pick_kernel<5>(dtype, accum, degrid);
    case 6: return pick_kernel<6>(dtype, accum, degrid);
    case 7: return pick_kernel<7>(dtype, accum, degrid);
    case 8: return pick_kernel<8>(dtype, accum, degrid);
    case 9: return pick_kernel<9>(dtype, accum, degrid);
    case 10: return pick_kernel<10>(dtype, accum, degrid);
    case 11: return pick_kernel<11>(dtype, accum, degrid);
    case 12: return pick_kernel<12>(dtype, accum, degrid);
    case 13: return pick_kernel<13>(dtype, accum, degrid);
    case 14: return pick_kernel<14>(dtype, accum, degrid);
    case 15: return pick_kernel<15>(dtype, accum, degrid);
    case 16: return pick_kernel<16>(dtype, accum, degrid);
    default: return nullptr;
  }
}

size_t stage_bytes(int W, int dtype, bool degrid) {
  const size_t rs = dtype ? 8 : 4;
  const int Wp = dtype ? ((W + 1) & ~1) : ((W + 3) & ~3);
  const size_t x0 = 32 * sizeof(int), cv = 32 * Wp * rs, ab = 32 * W * 2 * rs;
  return align16(x0 + (degrid ? 2 : 1) * cv + ab);
}

}  // namespace

size_t sweep_smem_bytes(int W, int dtype, int Ms, bool table_in_smem, bool degrid) {
  const size_t rs = dtype ? 8 : 4;
  const int Wp = dtype ? ((W + 1) & ~1) : ((W + 3) & ~3);
  const size_t tab = table_in_smem ? align16(size_t(Ms + 1) * Wp * rs) : 0;
  return tab + kWarps * stage_bytes(W, dtype, degrid);
}

int sweep_set_smem_limits(int W, int dtype, int accum, size_t smem_bytes, bool degrid) {
  void* k = kernel_for(W, dtype, accum, degrid);
  if (!k) return -1;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_bytes)) == cudaSuccess ? 0 : -1;
}

int sweep_occupancy(int W, int dtype, int accum, size_t smem_bytes, bool degrid, int* blocks_per_sm) {
  void* k = kernel_for(W, dtype, accum, degrid);
  if (!k) return -1;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kThreads, smem_bytes) == cudaSuccess ? 0
                                                                                                               : -1;
}

int grid_launch(const SweepArgs& a, cudaStream_t st) {
  void* k = kernel_for(a.W, a.dtype, a.accum, false);
  if (!k) return -1;
  const size_t smem = sweep_smem_bytes(a.W, a.dtype, a.Ms, a.table_in_smem != 0, false);
  cudaMemsetAsync(a.counters + kCntGridWork, 0, sizeof(int), st);
  SweepArgs args = a;
  void* params[] = {&args};
  if (cudaLaunchKernel(k, dim3(a.grid_blocks), dim3(kThreads), params, smem, st) != cudaSuccess) return -1;
  const int spill_blocks = 2 * 152;
  if (a.dtype) {
    k_grid_spill<double><<<spill_blocks, 256, 0, st>>>(a.items, a.counters, a.item_cap, a.W, a.N,
                                                       static_cast<const double2*>(a.spill),
                                                       static_cast<double2*>(a.grid));
  } else {
    k_grid_spill<float><<<spill_blocks, 256, 0, st>>>(a.items, a.counters, a.item_cap, a.W, a.N,
                                                      static_cast<const float2*>(a.spill),
                                                      static_cast<float2*>(a.grid));
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int degrid_launch(const SweepArgs& a, cudaStream_t st) {
  void* k = kernel_for(a.W, a.dtype, 0, true);
  if (!k) return -1;
  const size_t smem = sweep_smem_bytes(a.W, a.dtype, a.Ms, a.table_in_smem != 0, true);
  cudaMemsetAsync(a.counters + kCntDegridWork, 0, sizeof(int), st);
  SweepArgs args = a;
  void* params[] = {&args};
  if (cudaLaunchKernel(k, dim3(a.grid_blocks), dim3(kThreads), params, smem, st) != cudaSuccess) return -1;
  if (a.dtype) {
    k_degrid_fixup<double><<<2 * 152, 256, 0, st>>>(a.dup_list, a.bad_list, a.counters,
                                                    static_cast<const double2*>(a.dpart),
                                                    static_cast<double2*>(a.vis_out));
  } else {
    k_degrid_fixup<float><<<2 * 152, 256, 0, st>>>(a.dup_list, a.bad_list, a.counters,
                                                   static_cast<const float2*>(a.dpart),
                                                   static_cast<float2*>(a.vis_out));
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lmg

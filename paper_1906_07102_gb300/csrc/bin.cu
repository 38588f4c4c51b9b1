// Binning of visibility positions (support rule of Eq. 6) into strips of 64 (complex64) or
// 32 (complex128) columns sorted
// by pairs of support-start rows, and balanced work items for the sweep kernels.
//
// Pipeline (all on one stream, no host synchronisation):
//   1. k_bin_count   per visibility: float64 product to cells, exact fixed-point support
//                    rule, strip keys (one, or two when the support crosses into the next
//                    strip); the bucket counter's returned value is the record's rank.
//   2. scan          exclusive prefix sum of the bucket counts (strip-major, row-minor).
//   3. k_bin_scatter positions recomputed from (u, v) (cheaper than storing and reloading
//                    them), records of each pair of rows (2m, 2m+1) of a strip -- the row
//                    group the sweeps stage together -- to the pair's range, dealt so that
//                    any 32 consecutive records sample the whole pair (see dealt_position).
//   4. k_make_items  per strip and block of rows: items holding about item_target records,
//                    cut at even rows so that the sweeps' row groups are these pairs.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace lmg {
namespace {

// Support start (grid indices, wrapped to [0, N)) and table coordinates of position p =
// (u, v); false for a dropped position (product not finite or |u| N pixel_scale >= 2^30).
__device__ __forceinline__ bool vis_position(double2 p, double scale2, int W, int N, VisPos& vp,
                                             double2* delta = nullptr) {
  long long U, V;
  if (!fixed_position(p.x, scale2, U) || !fixed_position(p.y, scale2, V)) return false;
  if (delta) *delta = make_double2(quantisation_residual(p.x, scale2, U), quantisation_residual(p.y, scale2, V));
  long long n0, m0;
  support_start(U, W, n0, vp.su);
  support_start(V, W, m0, vp.sv);
  long long xi = (n0 + N / 2) % N;
  long long yi = (m0 + N / 2) % N;
  if (xi < 0) xi += N;
  if (yi < 0) yi += N;
  vp.x0 = static_cast<int>(xi);
  vp.y0 = static_cast<int>(yi);
  return true;
}

// Pass 1: positions to grid cells (support rule), bucket keys, and each record's rank in
// its bucket (the value returned by the bucket counter), so that pass 2 needs no atomics.
// Each thread takes kCountIlp positions per iteration so that their bucket atomics are in
// flight together.
constexpr int kCountIlp = 4;

__global__ void k_bin_count(const double* __restrict__ uv, long long nvis, double scale2, int W,
                            int N, int n_strips, int strip_w, int2* __restrict__ rank, int* __restrict__ hist,
                            int* __restrict__ counters, double2* __restrict__ frac) {
  const int lane = threadIdx.x & 31;  // for the dropped-position count
  const long long span = static_cast<long long>(blockDim.x) * kCountIlp;
  const long long stride = static_cast<long long>(gridDim.x) * span;
  for (long long base = static_cast<long long>(blockIdx.x) * span; base < nvis; base += stride) {
    VisPos vp[kCountIlp];
    int key1[kCountIlp], key2[kCountIlp];
    bool bad[kCountIlp];
#pragma unroll
    for (int u = 0; u < kCountIlp; ++u) {
      const long long k = base + u * blockDim.x + threadIdx.x;
      key1[u] = key2[u] = -1;
      bad[u] = false;
      vp[u] = VisPos{-1, 0, 0u, 0u};
      if (k < nvis) {
        double2 dl = make_double2(0.0, 0.0);
        const bool ok = vis_position(reinterpret_cast<const double2*>(uv)[k], scale2, W, N, vp[u],
                                     frac != nullptr ? &dl : nullptr);
        if (frac != nullptr) frac[k] = dl;
        if (ok) {
          const int strip = vp[u].x0 / strip_w;
          key1[u] = strip * N + vp[u].y0;
          if ((vp[u].x0 % strip_w) + W > strip_w) key2[u] = ((strip + 1) % n_strips) * N + vp[u].y0;
        } else {
          bad[u] = true;
        }
      }
    }
    int2 rk[kCountIlp];
#pragma unroll
    for (int u = 0; u < kCountIlp; ++u) {
      rk[u].x = key1[u] >= 0 ? atomicAdd(hist + key1[u], 1) : 0;
      rk[u].y = key2[u] >= 0 ? atomicAdd(hist + key2[u], 1) : 0;
    }
#pragma unroll
    for (int u = 0; u < kCountIlp; ++u) {
      const long long k = base + u * blockDim.x + threadIdx.x;
      if (k < nvis) rank[k] = rk[u];
      const unsigned nb = __popc(__ballot_sync(0xffffffffu, bad[u]));
      if (lane == 0 && nb) atomicAdd(counters + kCntBad, static_cast<int>(nb));
    }
  }
}

// Exclusive scan, stage 1: per-chunk sums.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanChunk = kScanThreads * kScanPer;

__global__ void k_scan_partials(const int* __restrict__ in, long long n, int* __restrict__ partial) {
  __shared__ int warp_sums[kScanThreads / 32];
  const long long base = static_cast<long long>(blockIdx.x) * kScanChunk + threadIdx.x * kScanPer;
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i)
    if (base + i < n) s += in[base + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += warp_sums[w];
    partial[blockIdx.x] = t;
  }
}

// Stage 2: exclusive scan of the chunk sums in one block (sequential over tiles of 1024).
__global__ void k_scan_top(int* __restrict__ partial, int nchunks) {
  __shared__ int carry;
  __shared__ int warp_sums[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nchunks; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nchunks ? partial[i] : 0;
    int x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
      int ws = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sums[lane] = ws;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? warp_sums[w - 1] : 0);
    if (i < nchunks) partial[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += incl;
    __syncthreads();
  }
}

// Stage 3: exclusive scan within each chunk plus the chunk offset; writes offsets[0..n].
__global__ void k_scan_final(const int* __restrict__ in, long long n, const int* __restrict__ partial,
                             int* __restrict__ offsets) {
  __shared__ int warp_sums[kScanThreads / 32];
  const long long base = static_cast<long long>(blockIdx.x) * kScanChunk + threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  int woff = 0;
  for (int k = 0; k < w; ++k) woff += warp_sums[k];
  int run = partial[blockIdx.x] + woff + x - s;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    if (base + i < n) offsets[base + i] = run;
    run += v[i];
  }
  if (base + kScanPer >= n && base < n) offsets[n] = run;  // thread holding the last element
}

// Pass 2: every record to offsets[bucket] + rank (no atomics).
// Position of the record of rank rho (0 .. n-1, in arrival order) inside its row pair of
// n records. Records of one baseline arrive in time order and land in nearby cells, so
// consecutive ranks cluster on a few columns; the sweeps give each lane the records that
// cover its column, so a chunk of clustered records leaves most lanes idle. The pair is
// dealt into nc = ceil(n / 32) runs, run j holding the ranks j, j + nc, j + 2 nc, ...
// (q or q + 1 of them, q = n / nc), so that any 32 consecutive positions hold ranks
// spread over the whole pair.
__device__ __forceinline__ int dealt_position(int rho, int n) {
  if (n <= 32) return rho;
  const int nc = (n + 31) >> 5, q = n / nc, r = n - q * nc;
  const int j = rho % nc;
  return j * q + min(j, r) + rho / nc;
}

__global__ void k_bin_scatter(const double* __restrict__ uv, double scale2, const int2* __restrict__ rank,
                              long long nvis, int W, int N, int n_strips, int strip_w,
                              const int* __restrict__ offsets, Rec* __restrict__ recs) {
  // kCountIlp visibilities per thread per iteration: their position, rank and offset loads
  // are in flight together (the pass is bound by its random L2 requests and their latency).
  // (u, v) and the ranks are read for the last time here: streaming loads (evict first)
  // leave the L2 to the offsets and the records being written.
  const long long span = static_cast<long long>(blockDim.x) * kCountIlp;
  const long long stride = static_cast<long long>(gridDim.x) * span;
  for (long long base = static_cast<long long>(blockIdx.x) * span; base < nvis; base += stride) {
    VisPos vp[kCountIlp];
    int2 rk[kCountIlp];
#pragma unroll
    for (int u = 0; u < kCountIlp; ++u) {
      const long long k = base + u * blockDim.x + threadIdx.x;
      vp[u] = VisPos{-1, 0, 0u, 0u};
      rk[u] = make_int2(0, 0);
      if (k < nvis) {
        rk[u] = __ldcs(rank + k);
        vis_position(__ldcs(reinterpret_cast<const double2*>(uv) + k), scale2, W, N, vp[u]);
      }
    }
    int g1[kCountIlp], g2[kCountIlp];  // bucket pair bases (-1: none)
#pragma unroll
    for (int u = 0; u < kCountIlp; ++u) {
      g1[u] = g2[u] = -1;
      if (vp[u].x0 >= 0) {
        const int strip = vp[u].x0 / strip_w, xr = vp[u].x0 % strip_w;
        const int pair_row = vp[u].y0 & ~1;
        g1[u] = strip * N + pair_row;
        if (xr + W > strip_w) g2[u] = ((strip + 1) % n_strips) * N + pair_row;
      }
    }
    // offsets of the pair's two rows and of the next pair (g is even: one 8-byte load and one
    // 4-byte load per record)
    int o1[kCountIlp][3], o2[kCountIlp][3];
#pragma unroll
    for (int u = 0; u < kCountIlp; ++u) {
      const int2 a1 = g1[u] >= 0 ? *reinterpret_cast<const int2*>(offsets + g1[u]) : make_int2(0, 0);
      const int2 a2 = g2[u] >= 0 ? *reinterpret_cast<const int2*>(offsets + g2[u]) : make_int2(0, 0);
      o1[u][0] = a1.x;
      o1[u][1] = a1.y;
      o1[u][2] = g1[u] >= 0 ? offsets[g1[u] + 2] : 0;
      o2[u][0] = a2.x;
      o2[u][1] = a2.y;
      o2[u][2] = g2[u] >= 0 ? offsets[g2[u] + 2] : 0;
    }
#pragma unroll
    for (int u = 0; u < kCountIlp; ++u) {
      if (g1[u] < 0) continue;
      const long long k = base + u * blockDim.x + threadIdx.x;
      const int odd = vp[u].y0 & 1, xr = vp[u].x0 % strip_w;
      // row pair (y0 & ~1, y0 | 1) of the strip: [offsets[g], offsets[g + 2])
      recs[o1[u][0] + dealt_position((odd ? o1[u][1] - o1[u][0] : 0) + rk[u].x, o1[u][2] - o1[u][0])] =
          Rec{static_cast<unsigned>(k), rec_pack(vp[u].y0, xr), vp[u].su, vp[u].sv};
      if (g2[u] >= 0)
        recs[o2[u][0] + dealt_position((odd ? o2[u][1] - o2[u][0] : 0) + rk[u].y, o2[u][2] - o2[u][0])] =
            Rec{static_cast<unsigned>(k), rec_pack(vp[u].y0, xr - strip_w), vp[u].su, vp[u].sv};
    }
  }
}

// One CTA per (strip, block of rows): the block's row offsets are staged in shared memory
// and the block is cut into items of about `target` records each (at least one item per
// block) by binary searches there, one item per thread. Items with more than target/2
// records are placed from the front of the array and the others from the back, so that
// the sweeps (which take items front to back, then back to front) start the heavy ones
// first.
constexpr int kMaxRowsPerBlock = 512;

__global__ void k_make_items(const int* __restrict__ offsets, int N, int n_strips, int rows_per_block,
                             int target, Item* __restrict__ items, int* __restrict__ counters, int cap) {
  __shared__ int s_off[kMaxRowsPerBlock + 1];
  const int nblk = (N + rows_per_block - 1) / rows_per_block;
  const int s = blockIdx.x / nblk, b = blockIdx.x % nblk;
  const int rb = b * rows_per_block, re = min(N, rb + rows_per_block);
  const int* off = offsets + static_cast<long long>(s) * N;
  for (int r = threadIdx.x; r <= re - rb; r += blockDim.x) s_off[r] = off[rb + r];
  __syncthreads();
  const int o0 = s_off[0], count = s_off[re - rb] - o0;
  const int m = max(1, (count + target - 1) / target);
  // first row (relative) whose offset reaches the k-th cut
  auto cut = [&](int k) {
    if (k <= 0) return 0;
    if (k >= m) return re - rb;
    const long long goal = o0 + (static_cast<long long>(count) * k) / m;
    int lo = 0, hi = re - rb;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s_off[mid] >= goal) hi = mid;
      else lo = mid + 1;
    }
    return lo & ~1;  // even rows: the sweeps' row groups are the binned row pairs
  };
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const int r0 = cut(k), r1 = cut(k + 1);
    const int n = s_off[r1] - s_off[r0];
    int slot;
    if (2 * n > target) slot = atomicAdd(counters + kCntItems, 1);
    else slot = cap - 1 - atomicAdd(counters + kCntItemsBack, 1);
    if (slot >= 0 && slot < cap) items[slot] = Item{s, rb + r0, rb + r1, n};
    else atomicOr(counters + kCntStatus, kStatusItemOverflow);
  }
}

}  // namespace

int bin_launch(const BinArgs& a, cudaStream_t st) {
  const long long L = static_cast<long long>(a.n_strips) * a.N;
  cudaMemsetAsync(a.hist, 0, sizeof(int) * L, st);
  cudaMemsetAsync(a.counters, 0, sizeof(int) * kNumCounters, st);
  const int threads = 256;
  const long long want_c = (a.nvis + threads * kCountIlp - 1) / (threads * kCountIlp);
  const int blocks_c = static_cast<int>(want_c < a.max_blocks ? (want_c > 0 ? want_c : 1) : a.max_blocks);
  k_bin_count<<<blocks_c, threads, 0, st>>>(a.uv, a.nvis, a.scale2, a.W, a.N, a.n_strips, a.strip, a.rank,
                                          a.hist, a.counters, a.frac);
  const int nchunks = static_cast<int>((L + kScanChunk - 1) / kScanChunk);
  k_scan_partials<<<nchunks, kScanThreads, 0, st>>>(a.hist, L, a.partial);
  k_scan_top<<<1, 1024, 0, st>>>(a.partial, nchunks);
  k_scan_final<<<nchunks, kScanThreads, 0, st>>>(a.hist, L, a.partial, a.offsets);
  k_bin_scatter<<<blocks_c, threads, 0, st>>>(a.uv, a.scale2, a.rank, a.nvis, a.W, a.N, a.n_strips, a.strip,
                                            a.offsets, a.recs);
  const int nblk = (a.N + a.rows_per_block - 1) / a.rows_per_block;
  const int ntask = a.n_strips * nblk;
  if (a.rows_per_block > kMaxRowsPerBlock) return -1;
  k_make_items<<<ntask, 128, 0, st>>>(a.offsets, a.N, a.n_strips, a.rows_per_block, a.item_target,
                                                   a.items, a.counters, a.item_cap);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int bin_scan_chunks(long long L) { return static_cast<int>((L + kScanChunk - 1) / kScanChunk); }

}  // namespace lmg

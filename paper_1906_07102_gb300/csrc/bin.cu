// Binning of visibility positions (support rule of Eq. 6) into 32-column strips sorted
// by support-start row, and balanced work items for the sweep kernels.
//
// Pipeline (all on one stream, no host synchronisation):
//   1. k_bin_count   per visibility: float64 product to cells, exact fixed-point support
//                    rule, strip keys (one, or two when the support crosses into the next
//                    strip); bucket counts with warp-aggregated atomics.
//   2. scan          exclusive prefix sum of the bucket counts (strip-major, row-minor).
//   3. k_bin_scatter records into their buckets (order inside a bucket is arbitrary).
//   4. k_make_items  per strip and block of rows: items holding about kItemRecs records.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace lmg {
namespace {

// Warp-aggregated atomicAdd of 1 to counter[key] for the lanes with key >= 0; returns
// the old value plus the lane's rank among lanes with the same key. All 32 lanes call.
__device__ __forceinline__ int agg_increment(int* counter, int key, int lane) {
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(peers) - 1;
  const int rank = __popc(peers & ((1u << lane) - 1u));
  int old = 0;
  if (lane == leader && key >= 0) old = atomicAdd(counter + key, __popc(peers));
  old = __shfl_sync(0xffffffffu, old, leader);
  return old + rank;
}

__global__ void k_bin_count(const double* __restrict__ uv, long long nvis, double scale2, int W,
                            int N, int n_strips, VisPos* __restrict__ pos, int* __restrict__ hist,
                            int* __restrict__ bad_list, int* __restrict__ counters) {
  const int lane = threadIdx.x & 31;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x; base < nvis; base += stride) {
    const long long k = base + threadIdx.x;
    int key1 = -1, key2 = -1, bad = -1;
    if (k < nvis) {
      long long U, V;
      const double2 p = reinterpret_cast<const double2*>(uv)[k];
      const bool ok = fixed_position(p.x, scale2, U) && fixed_position(p.y, scale2, V);
      VisPos vp;
      if (ok) {
        long long n0, m0;
        support_start(U, W, n0, vp.su);
        support_start(V, W, m0, vp.sv);
        long long xi = (n0 + N / 2) % N;
        long long yi = (m0 + N / 2) % N;
        if (xi < 0) xi += N;
        if (yi < 0) yi += N;
        vp.x0 = static_cast<int>(xi);
        vp.y0 = static_cast<int>(yi);
        const int strip = vp.x0 / kStrip;
        key1 = strip * N + vp.y0;
        if ((vp.x0 % kStrip) + W > kStrip) key2 = ((strip + 1) % n_strips) * N + vp.y0;
      } else {
        vp.x0 = -1;
        vp.y0 = 0;
        vp.su = vp.sv = 0u;
        bad = 0;
      }
      pos[k] = vp;
    }
    agg_increment(hist, key1, lane);
    agg_increment(hist, key2, lane);
    const int bslot = agg_increment(counters, bad < 0 ? -1 : 0, lane);
    if (bad >= 0) bad_list[bslot] = static_cast<int>(k);
    // counters[2] counts secondary records (for the degrid fix-up list)
    agg_increment(counters + 2, key2 >= 0 ? 0 : -1, lane);
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

// Stage 3: exclusive scan within each chunk plus the chunk offset; writes offsets[0..n]
// and a copy into cursor[0..n).
__global__ void k_scan_final(const int* __restrict__ in, long long n, const int* __restrict__ partial,
                             int* __restrict__ offsets, int* __restrict__ cursor) {
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
    if (base + i < n) {
      offsets[base + i] = run;
      cursor[base + i] = run;
    }
    run += v[i];
  }
  if (base + kScanPer >= n && base < n) offsets[n] = run;  // thread holding the last element
}

__global__ void k_bin_scatter(const VisPos* __restrict__ pos, long long nvis, int W, int N, int n_strips,
                              int* __restrict__ cursor, Rec* __restrict__ recs, int* __restrict__ dup_list,
                              int* __restrict__ counters) {
  const int lane = threadIdx.x & 31;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x; base < nvis; base += stride) {
    const long long k = base + threadIdx.x;
    int key1 = -1, key2 = -1;
    VisPos vp{-1, 0, 0u, 0u};
    if (k < nvis) {
      vp = pos[k];
      if (vp.x0 >= 0) {
        const int strip = vp.x0 / kStrip;
        key1 = strip * N + vp.y0;
        if ((vp.x0 % kStrip) + W > kStrip) key2 = ((strip + 1) % n_strips) * N + vp.y0;
      }
    }
    const int s1 = agg_increment(cursor, key1, lane);
    const int s2 = agg_increment(cursor, key2, lane);
    const int sd = agg_increment(counters + 3, key2 >= 0 ? 0 : -1, lane);
    if (key1 >= 0) recs[s1] = Rec{static_cast<unsigned>(k), vp.x0 % kStrip, vp.su, vp.sv};
    if (key2 >= 0) {
      recs[s2] = Rec{static_cast<unsigned>(k), (vp.x0 % kStrip) - kStrip, vp.su, vp.sv};
      dup_list[sd] = static_cast<int>(k);
    }
  }
}

// One thread per (strip, block of rows): cut the block into items of about `target`
// records each (at least one item per block), by binary search on the row offsets.
__global__ void k_make_items(const int* __restrict__ offsets, int N, int n_strips, int rows_per_block,
                             int target, Item* __restrict__ items, int* __restrict__ counters, int cap) {
  const int nblk = (N + rows_per_block - 1) / rows_per_block;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_strips * nblk) return;
  const int s = t / nblk, b = t % nblk;
  const int rb = b * rows_per_block, re = min(N, rb + rows_per_block);
  const int* off = offsets + static_cast<long long>(s) * N;
  const int o0 = off[rb], o1 = off[re];
  const int count = o1 - o0;
  const int m = max(1, (count + target - 1) / target);
  const int slot = atomicAdd(counters + 1, m);
  int prev = rb;
  for (int k = 0; k < m; ++k) {
    int next = re;
    if (k + 1 < m) {
      const long long goal = o0 + (static_cast<long long>(count) * (k + 1)) / m;
      int lo = prev, hi = re;  // first row r in [prev, re] with off[r] >= goal
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] >= goal) hi = mid;
        else lo = mid + 1;
      }
      next = lo;
    }
    if (slot + k < cap) items[slot + k] = Item{s, prev, next, 0};
    prev = next;
  }
}

}  // namespace

int bin_launch(const BinArgs& a, cudaStream_t st) {
  const long long L = static_cast<long long>(a.n_strips) * a.N;
  cudaMemsetAsync(a.hist, 0, sizeof(int) * L, st);
  cudaMemsetAsync(a.counters, 0, sizeof(int) * 8, st);
  const int threads = 256;
  const long long want = (a.nvis + threads - 1) / threads;
  const int blocks = static_cast<int>(want < a.max_blocks ? (want > 0 ? want : 1) : a.max_blocks);
  k_bin_count<<<blocks, threads, 0, st>>>(a.uv, a.nvis, a.scale2, a.W, a.N, a.n_strips, a.pos, a.hist,
                                          a.bad_list, a.counters);
  const int nchunks = static_cast<int>((L + kScanChunk - 1) / kScanChunk);
  k_scan_partials<<<nchunks, kScanThreads, 0, st>>>(a.hist, L, a.partial);
  k_scan_top<<<1, 1024, 0, st>>>(a.partial, nchunks);
  k_scan_final<<<nchunks, kScanThreads, 0, st>>>(a.hist, L, a.partial, a.offsets, a.cursor);
  k_bin_scatter<<<blocks, threads, 0, st>>>(a.pos, a.nvis, a.W, a.N, a.n_strips, a.cursor, a.recs, a.dup_list,
                                            a.counters);
  const int nblk = (a.N + a.rows_per_block - 1) / a.rows_per_block;
  const int ntask = a.n_strips * nblk;
  k_make_items<<<(ntask + 127) / 128, 128, 0, st>>>(a.offsets, a.N, a.n_strips, a.rows_per_block, a.item_target,
                                                   a.items, a.counters, a.item_cap);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int bin_scan_chunks(long long L) { return static_cast<int>((L + kScanChunk - 1) / kScanChunk); }

}  // namespace lmg

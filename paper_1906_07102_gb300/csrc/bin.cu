// Binning of visibility positions (support rule of Eq. 6) into strips of 64 (complex64) or
// 32 (complex128) columns sorted by pairs of support-start rows, and balanced work items for
// the sweep kernels.
//
// Pipeline (all on one stream, no host synchronisation):
//   1. k_bin_count   per visibility: float64 product to cells, exact fixed-point support
//                    rule, strip keys (one, or two when the support crosses into the next
//                    strip); the bucket counter's returned value is the record's rank.
//   2. scan          exclusive prefix sum of the bucket counts (strip-major, row-minor).
//   3. k_bin_scatter positions recomputed from (u, v) (measured cheaper than storing a
//                    decoded 16-byte position per visibility and reloading it), records
//                    of each pair of rows (2m, 2m+1) of a strip -- the row group
//                    the sweeps stage together -- to the pair's range, dealt so that any 32
//                    consecutive records sample the whole pair (see dealt_position).
//   4. k_make_items  per strip and block of rows: items holding about item_target records,
//                    cut at even rows so that the sweeps' row groups are these pairs.
// With a track layout (positions stored sample-major, k = t * tracks + b) passes 1 and 3
// follow each track instead (k_bin_count_tracks, k_bin_scatter_tracks).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace lmg {
namespace {

// i mod N in [0, N); positions inside the grid (the usual case) take no division.
__device__ __forceinline__ int wrap_index(long long i, int N) {
  if (static_cast<unsigned long long>(i) < static_cast<unsigned long long>(N)) return static_cast<int>(i);
  long long r = i % N;
  if (r < 0) r += N;
  return static_cast<int>(r);
}

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
  vp.x0 = wrap_index(n0 + N / 2, N);
  vp.y0 = wrap_index(m0 + N / 2, N);
  return true;
}

// Strip of a support-start column and the column inside it (strip_w is a power of two).
__device__ __forceinline__ int strip_of(int x0, int strip_w) { return x0 >> (__ffs(strip_w) - 1); }
__device__ __forceinline__ int col_in_strip(int x0, int strip_w) { return x0 & (strip_w - 1); }
__device__ __forceinline__ int next_strip(int strip, int n_strips) { return strip + 1 == n_strips ? 0 : strip + 1; }

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
          const int strip = strip_of(vp[u].x0, strip_w);
          key1[u] = strip * N + vp[u].y0;
          if (col_in_strip(vp[u].x0, strip_w) + W > strip_w) key2[u] = next_strip(strip, n_strips) * N + vp[u].y0;
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

// Stage 2: exclusive scan within each chunk plus the chunk's offset, the sum of the
// preceding chunks' totals (each CTA adds them up itself: a few thousand at most, cheaper
// than a separate launch); writes offsets[0..n].
__global__ void k_scan_final(const int* __restrict__ in, long long n, const int* __restrict__ partial,
                             int* __restrict__ offsets) {
  __shared__ int warp_sums[kScanThreads / 32];
  __shared__ int chunk_base;
  {
    int c = 0;
    for (int k = threadIdx.x; k < static_cast<int>(blockIdx.x); k += blockDim.x) c += partial[k];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < kScanThreads / 32; ++w) t += warp_sums[w];
      chunk_base = t;
    }
    __syncthreads();
  }
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
  int run = chunk_base + woff + x - s;
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
        const int strip = strip_of(vp[u].x0, strip_w), xr = col_in_strip(vp[u].x0, strip_w);
        const int pair_row = vp[u].y0 & ~1;
        g1[u] = strip * N + pair_row;
        if (xr + W > strip_w) g2[u] = next_strip(strip, n_strips) * N + pair_row;
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
      const int odd = vp[u].y0 & 1, xr = col_in_strip(vp[u].x0, strip_w);
      // row pair (y0 & ~1, y0 | 1) of the strip: [offsets[g], offsets[g + 2])
      recs[o1[u][0] + dealt_position((odd ? o1[u][1] - o1[u][0] : 0) + rk[u].x, o1[u][2] - o1[u][0])] =
          Rec{static_cast<unsigned>(k), rec_pack(vp[u].y0, xr), vp[u].su, vp[u].sv};
      if (g2[u] >= 0)
        recs[o2[u][0] + dealt_position((odd ? o2[u][1] - o2[u][0] : 0) + rk[u].y, o2[u][2] - o2[u][0])] =
            Rec{static_cast<unsigned>(k), rec_pack(vp[u].y0, xr - strip_w), vp[u].su, vp[u].sv};
    }
  }
}

// Track-ordered binning. With the positions stored sample-major (k = t * tracks + b: one
// sample of every track, then the next sample), thread g follows track b = g mod tracks over
// kTrackChunk consecutive samples (chunk g / tracks); the lanes of a warp read neighbouring
// tracks at the same sample, so the position loads stay coalesced. Along a track the support
// moves by at most a few cells per sample and consecutive samples fall in the same bucket
// (strip, row) in runs (5.9 samples on average on 6 h Earth-rotation tracks with 64-column
// strips). The counting pass takes one bucket atomic per run and stores the rank it returns
// (the rank of the run's first record) at the run's first visibility; the placement pass walks
// the same runs and gives record j of a run the rank + j, loading that rank and the bucket's
// offsets once per run. Runs end where the bucket changes (a dropped position ends one) and at
// the end of a chunk, identically in both passes. Results do not depend on `tracks`: any value
// bins correctly; it only sets the order of the records within a bucket and the cost.
constexpr int kTrackChunk = 32;

__device__ __forceinline__ void bucket_keys(const VisPos& vp, int W, int N, int n_strips, int strip_w, int& key1,
                                            int& key2) {
  const int strip = strip_of(vp.x0, strip_w);
  key1 = strip * N + vp.y0;
  key2 = col_in_strip(vp.x0, strip_w) + W > strip_w ? next_strip(strip, n_strips) * N + vp.y0 : -1;
}

__global__ void k_bin_count_tracks(const double* __restrict__ uv, long long nvis, long long tracks, double scale2,
                                   int W, int N, int n_strips, int strip_w, int2* __restrict__ rank,
                                   int* __restrict__ hist, int* __restrict__ counters, double2* __restrict__ frac) {
  const double2* uv2 = reinterpret_cast<const double2*>(uv);
  int* rank1 = reinterpret_cast<int*>(rank);  // rank[k].x = rank1[2 k], rank[k].y = rank1[2 k + 1]
  const long long n_t = (nvis + tracks - 1) / tracks;
  const long long n_threads = tracks * ((n_t + kTrackChunk - 1) / kTrackChunk);
  for (long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; g < n_threads;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long b = g % tracks, t0 = (g / tracks) * kTrackChunk;
    const long long k_end = min(nvis, min(n_t, t0 + kTrackChunk) * tracks);
    int cur1 = -1, len1 = 0, cur2 = -1, len2 = 0;
    long long start1 = 0, start2 = 0;
    // the rank of a run is stored at the next flush, so that the atomic's round trip overlaps
    // the samples between (a store of its value right away would wait for it)
    long long pend1 = -1, pend2 = -1;
    int pval1 = 0, pval2 = 0;
    for (long long k = t0 * tracks + b; k < k_end; k += tracks) {
      VisPos vp{0, 0, 0u, 0u};
      double2 dl = make_double2(0.0, 0.0);
      const bool ok = vis_position(uv2[k], scale2, W, N, vp, frac != nullptr ? &dl : nullptr);
      if (frac != nullptr) frac[k] = dl;
      int key1 = -1, key2 = -1;
      if (ok) bucket_keys(vp, W, N, n_strips, strip_w, key1, key2);
      else atomicAdd(counters + kCntBad, 1);
      if (key1 != cur1) {
        if (len1 > 0) {
          if (pend1 >= 0) rank1[2 * pend1] = pval1;
          pval1 = atomicAdd(hist + cur1, len1);
          pend1 = start1;
        }
        cur1 = key1;
        start1 = k;
        len1 = 0;
      }
      len1 += key1 >= 0;
      if (key2 != cur2) {
        if (len2 > 0) {
          if (pend2 >= 0) rank1[2 * pend2 + 1] = pval2;
          pval2 = atomicAdd(hist + cur2, len2);
          pend2 = start2;
        }
        cur2 = key2;
        start2 = k;
        len2 = 0;
      }
      len2 += key2 >= 0;
    }
    if (len1 > 0) {
      if (pend1 >= 0) rank1[2 * pend1] = pval1;
      pval1 = atomicAdd(hist + cur1, len1);
      pend1 = start1;
    }
    if (len2 > 0) {
      if (pend2 >= 0) rank1[2 * pend2 + 1] = pval2;
      pval2 = atomicAdd(hist + cur2, len2);
      pend2 = start2;
    }
    if (pend1 >= 0) rank1[2 * pend1] = pval1;
    if (pend2 >= 0) rank1[2 * pend2 + 1] = pval2;
  }
}

// Placement of the records of one run: the pair's base and the dealt position (see
// dealt_position) of rank rho = row offset + run rank + j, kept as rho = i nc + jj so that
// each further record of the run costs no division.
struct RunPlace {
  int base, nc, q, r, jj, i;
  __device__ __forceinline__ void start(const int* __restrict__ offsets, int key, int rank0) {
    const int g = key & ~1;  // N is even: the pair's first row has an even key
    const int2 a = *reinterpret_cast<const int2*>(offsets + g);
    const int n = offsets[g + 2] - a.x;
    const int rho = ((key & 1) ? a.y - a.x : 0) + rank0;
    base = a.x;
    nc = max(1, (n + 31) >> 5);
    q = n / nc;
    r = n - q * nc;
    i = rho / nc;
    jj = rho - i * nc;
  }
  __device__ __forceinline__ int next() {
    const int pos = base + jj * q + min(jj, r) + i;
    if (++jj == nc) {
      jj = 0;
      ++i;
    }
    return pos;
  }
};

__global__ void k_bin_scatter_tracks(const double* __restrict__ uv, double scale2, const int2* __restrict__ rank,
                                     long long nvis, long long tracks, int W, int N, int n_strips, int strip_w,
                                     const int* __restrict__ offsets, Rec* __restrict__ recs) {
  const double2* uv2 = reinterpret_cast<const double2*>(uv);
  const int* rank1 = reinterpret_cast<const int*>(rank);
  const long long n_t = (nvis + tracks - 1) / tracks;
  const long long n_threads = tracks * ((n_t + kTrackChunk - 1) / kTrackChunk);
  for (long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; g < n_threads;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long b = g % tracks, t0 = (g / tracks) * kTrackChunk;
    const long long k_end = min(nvis, min(n_t, t0 + kTrackChunk) * tracks);
    int cur1 = -1, cur2 = -1;
    RunPlace run1{}, run2{};
    for (long long k = t0 * tracks + b; k < k_end; k += tracks) {
      VisPos vp;
      const bool ok = vis_position(__ldcs(uv2 + k), scale2, W, N, vp);
      int key1 = -1, key2 = -1;
      if (ok) bucket_keys(vp, W, N, n_strips, strip_w, key1, key2);
      if (key1 != cur1) {
        cur1 = key1;
        if (key1 >= 0) run1.start(offsets, key1, __ldcs(rank1 + 2 * k));
      }
      if (key2 != cur2) {
        cur2 = key2;
        if (key2 >= 0) run2.start(offsets, key2, __ldcs(rank1 + 2 * k + 1));
      }
      if (key1 < 0) continue;
      const int xr = col_in_strip(vp.x0, strip_w);
      recs[run1.next()] = Rec{static_cast<unsigned>(k), rec_pack(vp.y0, xr), vp.su, vp.sv};
      if (key2 >= 0) recs[run2.next()] = Rec{static_cast<unsigned>(k), rec_pack(vp.y0, xr - strip_w), vp.su, vp.sv};
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
  long long n_tthreads = 0;
  if (a.tracks > 0) {
    const long long n_t = (a.nvis + a.tracks - 1) / a.tracks;
    n_tthreads = a.tracks * ((n_t + kTrackChunk - 1) / kTrackChunk);
  }
  const long long want_t = (n_tthreads + threads - 1) / threads;
  const int blocks_t = static_cast<int>(want_t < a.max_blocks ? (want_t > 0 ? want_t : 1) : a.max_blocks);
  if (a.tracks > 0)
    k_bin_count_tracks<<<blocks_t, threads, 0, st>>>(a.uv, a.nvis, a.tracks, a.scale2, a.W, a.N, a.n_strips,
                                                     a.strip, a.rank, a.hist, a.counters, a.frac);
  else
    k_bin_count<<<blocks_c, threads, 0, st>>>(a.uv, a.nvis, a.scale2, a.W, a.N, a.n_strips, a.strip, a.rank,
                                            a.hist, a.counters, a.frac);
  const int nchunks = static_cast<int>((L + kScanChunk - 1) / kScanChunk);
  k_scan_partials<<<nchunks, kScanThreads, 0, st>>>(a.hist, L, a.partial);
  k_scan_final<<<nchunks, kScanThreads, 0, st>>>(a.hist, L, a.partial, a.offsets);
  if (a.tracks > 0)
    k_bin_scatter_tracks<<<blocks_t, threads, 0, st>>>(a.uv, a.scale2, a.rank, a.nvis, a.tracks, a.W, a.N,
                                                       a.n_strips, a.strip, a.offsets, a.recs);
  else
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

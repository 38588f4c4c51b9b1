// Gridding and degridding sweeps (Eqs. 5-6 and their transpose, Section 4): the per-item
// device code shared by the single-plan kernels (sweep.cu) and the multi-channel
// persistent kernels (batch.cu).
//
// The grid is cut into 32-column strips; a warp owns one work item (a range of rows of
// one strip) and lane t owns column t of the strip. The item's records come grouped by
// pairs of support-start rows (dealt inside a pair by the binning, so that 32 consecutive
// records spread over the pair's columns) and are visited in groups of kD = 2 rows, in
// chunks of up to 32 records
// (the records and visibilities of the next two chunks are already in flight):
//   1. the chunk's 2W table weights per record (Section 5.1 lookup) are staged in shared
//      memory: Cu_i w V (gridding) or Cu_i (degridding), and Cv_j shifted by the record's
//      row offset d in the group, so that entry q of the staged vector weights target row
//      q of the group (q < T = W + kD - 1). G lanes share a record and look up one entry
//      each (a lane per record would read 32 random table rows per instruction, which
//      serialises on shared-memory banks). The shifted vectors are stored entry-major
//      with a row pitch of 32 + 32/G, so that lanes reading entry q of different records
//      hit distinct banks and so do the G lanes storing one record's entries;
//   2. each lane builds the set of records whose support covers its column (32x32 bit
//      transpose of the per-record cover masks) and visits them;
//   3. gridding: lane t holds a ring of RS >= T accumulators (rows of its column) in
//      registers and adds Cv'_q (Cu_i w V) to ring slot (base + q) -- a compile-time
//      index, the group loop being unrolled over one ring period. After a group its kD rows
//      are final and are stored as whole rows (256-byte coalesced stores for complex64).
//      The W-1 rows past the item go to a spill buffer and are added by k_grid_spill once
//      all items have stored their rows.
//      degridding: the ring holds grid rows of the lane's column; lane t forms
//      sum_q Cv'_q G[row0 + q][t] for each covering record and stages it; lane l sums
//      Cu_i times its record's W staged sums and adds the result to the zeroed output (a
//      visibility whose support crosses a strip has two records, one per strip).
// Every grid cell is written exactly once by the gridding sweep (no pre-zeroing, no
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "device_common.cuh"
#include "kernels.h"

namespace lmg {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <typename R> __host__ __device__ constexpr int wpad(int W) {
  return sizeof(R) == 4 ? (W | 1) : ((W + 1) & ~1);
}

// Rows per group and the register ring: RS >= T = W + kD - 1 slots, a multiple of kD, so
// that the group loop unrolled over P = RS / kD groups indexes every slot at compile time.
constexpr int kD = 2;  // the binning's row pairs (bin.cu) are these groups
template <int W> struct Ring {
  static constexpr int T = W + kD - 1;
  static constexpr int R = kD * ((T + kD - 1) / kD);
  static constexpr int P = R / kD;
};

// Cooperative table lookup while staging a chunk: G lanes share one record (each computes
// one table entry), P = 32 / G records per round.
template <int W> struct Coop {
  static constexpr int G = W <= 4 ? 4 : (W <= 8 ? 8 : 16);
  static constexpr int P = 32 / G;
  // Row pitch (elements) of the staged Cv: entry q of record l sits at q * pitch + l. The
  // extra P elements put the entries of the P records of one staging round in distinct
  // banks, while the sweep's reads (entry q of different records) stay conflict-free.
  static constexpr int pitch = 32 + P;
};
__host__ __device__ constexpr int coop_group(int W) { return W <= 4 ? 4 : (W <= 8 ? 8 : 16); }

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <int W, typename R> struct Stage {
  // per warp: x0[32] | cvs[T][pitch] (entry-major) | cu[32][W] (degrid) | a or p [32][W] complex
  static constexpr int T = Ring<W>::T;
  static constexpr size_t x0_bytes = 32 * sizeof(int);
  static constexpr size_t cv_bytes = align16(size_t(T) * Coop<W>::pitch * sizeof(R));
  static constexpr size_t cu_bytes = 32 * W * sizeof(R);
  static constexpr size_t a_bytes = 32 * W * 2 * sizeof(R);
  static constexpr size_t grid_bytes = x0_bytes + cv_bytes + a_bytes;
  static constexpr size_t degrid_bytes = x0_bytes + cv_bytes + cu_bytes + a_bytes;
};

// Table lookup (Section 5.1, Appendix F): row offset (elements) and interpolation fraction
// of coordinate S (units of 2^-32), from the exact integer product S Ms. Linear uses row
// k = floor(t) and fraction t - k with t = S Ms 2^-32; nearest uses row floor(t + 1/2). The
// table has Ms + 1 rows of stride Wp.
template <typename R, bool EXT>
__device__ __forceinline__ void table_coord(int Wp, int Ms, int interp, unsigned S, int& off, R& f) {
  const unsigned long long Pm = static_cast<unsigned long long>(S) * static_cast<unsigned>(Ms);
  if constexpr (!EXT) {
    if (interp) {
      off = static_cast<int>(Pm >> 32) * Wp;
      f = static_cast<R>(static_cast<unsigned>(Pm & 0xffffffffull)) * static_cast<R>(2.3283064365386962890625e-10);
    } else {
      off = static_cast<int>((Pm + 0x80000000ull) >> 32) * Wp;
      f = R(0);
    }
  } else if (interp == 4) {
    // direct calculation: the coefficients replace the rows; f = s
    off = 0;
    f = static_cast<R>(S) * static_cast<R>(2.3283064365386962890625e-10);
  } else {
    // degree d = interp: first stencil row k0 = floor(t - (d - 1) / 2), clamped to
    // [0, Ms - d], and f = t - k0 in [0, d] (t = S Ms 2^-32)
    const long long P = static_cast<long long>(Pm);
    long long k0 = (P - static_cast<long long>(interp - 1) * 0x80000000ll) >> 32;
    k0 = k0 < 0 ? 0 : (k0 > Ms - interp ? Ms - interp : k0);
    off = static_cast<int>(k0) * Wp;
    f = static_cast<R>(P - (k0 << 32)) * static_cast<R>(2.3283064365386962890625e-10);
  }
}

// Direct calculation (Section 5.2, float64 plans): C_a(s) = sum_k alpha[a][k] cos(k phi s) +
// beta[a][k] sin(k phi s), coef = {phi, alpha[W][33], beta[W][33]} (A^-1 and the node sums
// folded in on the host); cos/sin(k phi s) by rotation from one sincos.
template <typename R>
__device__ __forceinline__ R direct_entry(const R* __restrict__ coef, int W, int a, R s) {
  R sn, cs;
  if constexpr (sizeof(R) == 8) sincos(coef[0] * s, &sn, &cs);
  else sincosf(coef[0] * s, &sn, &cs);
  const R* al = coef + 1 + a * kDirectNodes;
  const R* be = coef + 1 + (W + a) * kDirectNodes;
  R ck = R(1), sk = R(0), acc = al[0];
  for (int k = 1; k < kDirectNodes; ++k) {
    const R c2 = ck * cs - sk * sn;
    sk = ck * sn + sk * cs;
    ck = c2;
    acc += al[k] * ck + be[k] * sk;
  }
  return acc;
}

// Lagrange interpolation of degree d (2 or 3) through the rows p[0], p[Wp], ..., p[d Wp]
// at local coordinate x in [0, d] (Appendix F for d > 1).
template <typename R>
__device__ __forceinline__ R lagrange_entry(const R* __restrict__ p, int Wp, int d, R x) {
  const R a = x, b = x - R(1), c = x - R(2);
  if (d == 2) return R(0.5) * b * c * p[0] - a * c * p[Wp] + R(0.5) * a * b * p[2 * Wp];
  const R e = x - R(3), sixth = R(1) / R(6);
  return -sixth * b * c * e * p[0] + R(0.5) * a * c * e * p[Wp] - R(0.5) * a * b * e * p[2 * Wp] +
         sixth * a * b * c * p[3 * Wp];
}

// Stages the weights of a chunk's records, held one per lane by lanes lo .. hi-1 (table
// row offsets and fractions for u and v, row offset d in the group, and for gridding
// w V): Cv shifted by d into s_cv (entry q of record l at q * pitch + l, zero for q
// outside [d, d + W)) and Cu, times w V when gridding, into s_u[l * W + i]. G lanes share
// a record and compute one table entry each (C = T[k] + f (T[k+1] - T[k]), or Lagrange
// through d + 1 rows), so a round's
// table reads touch P rows instead of 32 rows per instruction.
template <int W, typename R, bool GRID, bool EXT>
__device__ __forceinline__ void stage_chunk(const R* __restrict__ tab, int Wp, int interp, int lo, int hi, int ou,
                                            R fu, int ov, R fv, int d, R wx, R wy, R* __restrict__ s_cv,
                                            void* __restrict__ s_u, int lane) {
  using C2 = typename Cplx<R>::T;
  constexpr int G = Coop<W>::G, P = Coop<W>::P, pitch = Coop<W>::pitch, TT = Ring<W>::T;
  const int g = lane / G, i = lane % G;
  const int ovd = ov | (d << 28);  // row offsets stay below 2^28 (Ms <= 10^6, Wp <= 16)
  for (int r0 = lo; r0 < hi; r0 += P) {
    const int r = r0 + g, src = r & 31;
    const int ou_r = __shfl_sync(0xffffffffu, ou, src);
    const R fu_r = __shfl_sync(0xffffffffu, fu, src);
    const int ovd_r = __shfl_sync(0xffffffffu, ovd, src);
    const R fv_r = __shfl_sync(0xffffffffu, fv, src);
    const int ov_r = ovd_r & 0x0fffffff, d_r = ovd_r >> 28;
    R wx_r = R(0), wy_r = R(0);
    if constexpr (GRID) {
      wx_r = __shfl_sync(0xffffffffu, wx, src);
      wy_r = __shfl_sync(0xffffffffu, wy, src);
    }
    if (r < hi) {
      if (i < W) {
        R cu, cv;
        if constexpr (!EXT) {
          cu = tab[ou_r + i];
          cv = tab[ov_r + i];
          if (interp) {
            cu = cu + fu_r * (tab[ou_r + Wp + i] - cu);
            cv = cv + fv_r * (tab[ov_r + Wp + i] - cv);
          }
        } else {
          // direct calculation exists for float64 plans and W <= 11 only (plan creation)
          if constexpr (sizeof(R) == 8 && W <= 11) {
            if (interp == 4) {
              cu = direct_entry<R>(tab, W, i, fu_r);
              cv = direct_entry<R>(tab, W, i, fv_r);
            } else {
              cu = lagrange_entry<R>(tab + ou_r + i, Wp, interp, fu_r);
              cv = lagrange_entry<R>(tab + ov_r + i, Wp, interp, fv_r);
            }
          } else {
            cu = lagrange_entry<R>(tab + ou_r + i, Wp, interp, fu_r);
            cv = lagrange_entry<R>(tab + ov_r + i, Wp, interp, fv_r);
          }
        }
        if constexpr (GRID) {
          C2 t;
          t.x = cu * wx_r;
          t.y = cu * wy_r;
          static_cast<C2*>(s_u)[r * W + i] = t;
        } else {
          static_cast<R*>(s_u)[r * W + i] = cu;
        }
        s_cv[(i + d_r) * pitch + r] = cv;
      }
      // the kD - 1 zero entries, on the group's spare lanes where it has them
      for (int z = (i - W + G) % G; z < TT - W; z += G) s_cv[(z < d_r ? z : z + W) * pitch + r] = R(0);
    }
  }
}

// Gridding staging by the record's own lane (nearest / linear): the lane reads its rows
// with scalar loads. The float32 table rows have an odd stride (W | 1), so 32 random rows
// spread over the banks; measured faster for gridding than the cooperative staging, which
// degridding keeps (its staging is lighter).
template <int W, typename R>
__device__ __forceinline__ void stage_own(const R* __restrict__ tab, int Wp, int interp, bool mine, int ou, R fu,
                                          int ov, R fv, int d, R wx, R wy, R* __restrict__ s_cv,
                                          typename Cplx<R>::T* __restrict__ s_a, int lane) {
  using C2 = typename Cplx<R>::T;
  constexpr int pitch = Coop<W>::pitch, TT = Ring<W>::T;
  if (!mine) return;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    R cu = tab[ou + i], cv = tab[ov + i];
    if (interp) {
      cu = cu + fu * (tab[ou + Wp + i] - cu);
      cv = cv + fv * (tab[ov + Wp + i] - cv);
    }
    C2 t;
    t.x = cu * wx;
    t.y = cu * wy;
    s_a[lane * W + i] = t;
    s_cv[(i + d) * pitch + lane] = cv;
  }
#pragma unroll
  for (int z = 0; z < TT - W; ++z) s_cv[(z < d ? z : z + W) * pitch + lane] = R(0);
}

// Copy a table into shared memory (all threads of the CTA), or use it in place.
template <typename R>
__device__ __forceinline__ const R* stage_table(const void* table, int n, bool in_smem, unsigned char* smem) {
  const R* g = static_cast<const R*>(table);
  if (!in_smem) return g;
  R* s = reinterpret_cast<R*>(smem);
  for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = g[i];
  __syncthreads();
  return s;
}

__device__ __forceinline__ int next_item(int* counter, int lane) {
  int it = 0;
  if (lane == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, it, 0);
}

// Work index -> item: heavy items were placed from the front of the array, light ones
// from the back.
__device__ __forceinline__ int work_total(const int* counters, int cap, int& nfront) {
  nfront = min(counters[kCntItems], cap);
  return min(nfront + counters[kCntItemsBack], cap);
}
__device__ __forceinline__ int item_slot(int w, int nfront, int cap) { return w < nfront ? w : cap - 1 - (w - nfront); }

// Record prefetch for the software pipeline: one record and its visibility (and weight)
// per lane for a chunk starting at `start`.
template <typename R> struct Fetch {
  Rec rc;
  typename Cplx<R>::T v;
  R wt;
};

// Error-free addition s + e = a + b (Knuth TwoSum); a receives s, lo accumulates e.
__device__ __forceinline__ void two_sum_acc(float& a, float& lo, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  lo += __fsub_rn(a, ap) + __fsub_rn(b, bp);
  a = s;
}

// Resident CTAs per SM the register allocation must allow.
template <int W, typename R, bool COMP = false, bool EXT = false> constexpr int min_blocks() {
  // the extended lookups (Lagrange, direct) need more registers: fewer resident CTAs
  return COMP ? 2 : ((sizeof(R) == 4 && W <= 8) ? (EXT ? 2 : 3) : 1);
}


// One gridding work item (rows [r0, r1) of one strip), run by the 32 lanes of a warp;
// `my` is the warp's staging area in shared memory, `tab` the table (shared or global).
template <int W, typename R, bool COMP, bool EXT = false>
__device__ __forceinline__ void grid_item(const SweepArgs& a, const R* __restrict__ tab, unsigned char* my,
                                          int slot, int lane) {
  using C2 = typename Cplx<R>::T;
  using St = Stage<W, R>;
  constexpr int Wp = wpad<R>(W);
  constexpr int RS = Ring<W>::R, P = Ring<W>::P, TT = Ring<W>::T;
  int* s_x0 = reinterpret_cast<int*>(my);
  R* s_cv = reinterpret_cast<R*>(my + St::x0_bytes);
  C2* s_a = reinterpret_cast<C2*>(my + St::x0_bytes + St::cv_bytes);

  const Rec* __restrict__ recs = a.recs;
  const C2* __restrict__ vis = static_cast<const C2*>(a.vis);
  const R* __restrict__ wts = static_cast<const R*>(a.weights);
  C2* __restrict__ grid = static_cast<C2*>(a.grid);
  C2* __restrict__ spill = static_cast<C2*>(a.spill);
  const int N = a.N;

  auto fetch_rec = [&](int start, int end, Fetch<R>& f) {
    if (start + lane < end) f.rc = recs[start + lane];
  };
  auto fetch_vis = [&](int start, int end, Fetch<R>& f) {
    if (start + lane < end) {
      f.v = vis[f.rc.idx];
      f.wt = wts != nullptr ? wts[f.rc.idx] : R(1);
    }
  };

  const Item item = a.items[slot];
  const int* __restrict__ off = a.offsets + static_cast<long long>(item.strip) * N;
  const int col = item.strip * kStrip + lane;
  const int nrows = item.r1 - item.r0;
  // ring slot x % RS accumulates relative row x of column `col` (separate real and
  // imaginary arrays: two scalar FMAs measured faster here than one packed f32x2 FMA)
  R acc_re[RS], acc_im[RS], lo_re[RS], lo_im[RS];
#pragma unroll
  for (int q = 0; q < RS; ++q) {
    acc_re[q] = acc_im[q] = lo_re[q] = lo_im[q] = R(0);
  }
  // software pipeline over 32-record windows of the item (window k = records
  // rb + 32k .. rb + 32k + 31, lane l holding record rb + 32k + l): while window k is
  // processed, the visibilities of window k+1 and the records of window k+2 are in flight
  const int rb = off[item.r0], rend = off[item.r1];
  int wbase = rb, cstart = rb;
  Fetch<R> f0{}, f1{}, f2{};
  fetch_rec(rb, rend, f0);
  fetch_rec(rb + 32, rend, f1);
  fetch_vis(rb, rend, f0);
  fetch_vis(rb + 32, rend, f1);
  fetch_rec(rb + 64, rend, f2);
  for (int g0 = 0; g0 < nrows; g0 += RS) {
#pragma unroll
    for (int gp = 0; gp < P; ++gp) {
      const int gb = g0 + gp * kD;
      if (gb < nrows) {
        const int row0 = item.r0 + gb;
        const int re = off[min(row0 + kD, item.r1)];
        while (cstart < re) {
          // chunk: records [cstart, ce) of window wbase, staged by lanes cstart - wbase ..
          const int ce = min(re, wbase + 32);
          const int lo = cstart - wbase, hi = ce - wbase;
          const bool mine = lane >= lo && lane < hi;
          const int xrel = rec_xrel(f0.rc.rx);
          if (mine) s_x0[lane] = xrel;
          int ou, ov;
          R fu, fv;
          table_coord<R, EXT>(Wp, a.Ms, a.interp, f0.rc.su, ou, fu);
          table_coord<R, EXT>(Wp, a.Ms, a.interp, f0.rc.sv, ov, fv);
          if constexpr (EXT)
            stage_chunk<W, R, true, EXT>(tab, Wp, a.interp, lo, hi, ou, fu, ov, fv, rec_row(f0.rc.rx) - row0,
                                         f0.v.x * f0.wt, f0.v.y * f0.wt, s_cv, s_a, lane);
          else
            stage_own<W, R>(tab, Wp, a.interp, mine, ou, fu, ov, fv, rec_row(f0.rc.rx) - row0, f0.v.x * f0.wt,
                            f0.v.y * f0.wt, s_cv, s_a, lane);
          const unsigned cover = mine ? cover_mask(xrel, W) : 0u;
          __syncwarp();
          unsigned M = transpose32(cover, lane);
          if constexpr (!COMP) {
            while (M) {
              const int l1 = __ffs(M) - 1;
              M &= M - 1u;
              const bool two = M != 0u;
              const int l2 = two ? __ffs(M) - 1 : l1;
              if (two) M &= M - 1u;
              const C2 a1 = s_a[l1 * W + (lane - s_x0[l1])];
              C2 a2 = s_a[l2 * W + (lane - s_x0[l2])];
              if (!two) { a2.x = R(0); a2.y = R(0); }
#pragma unroll
              for (int q = 0; q < TT; ++q) {
                const R c1 = s_cv[q * Coop<W>::pitch + l1];
                const R c2 = s_cv[q * Coop<W>::pitch + l2];
                const int k = (gp * kD + q) % RS;
                acc_re[k] = fma(c1, a1.x, fma(c2, a2.x, acc_re[k]));
                acc_im[k] = fma(c1, a1.y, fma(c2, a2.y, acc_im[k]));
              }
            }
          }
          while (M) {
            const int l = __ffs(M) - 1;
            M &= M - 1u;
            const C2 ai = s_a[l * W + (lane - s_x0[l])];
#pragma unroll
            for (int q = 0; q < TT; ++q) {
              const R c = s_cv[q * Coop<W>::pitch + l];
              const int k = (gp * kD + q) % RS;
              if constexpr (COMP) {
                two_sum_acc(acc_re[k], lo_re[k], c * ai.x);
                two_sum_acc(acc_im[k], lo_im[k], c * ai.y);
              } else {
                acc_re[k] = fma(c, ai.x, acc_re[k]);
                acc_im[k] = fma(c, ai.y, acc_im[k]);
              }
            }
          }
          __syncwarp();
          cstart = ce;
          if (cstart == wbase + 32) {
            wbase += 32;
            f0 = f1;
            f1 = f2;
            fetch_vis(wbase + 32, rend, f1);
            fetch_rec(wbase + 64, rend, f2);
          }
        }
        // rows row0 .. row0 + kD - 1 are complete: store them and recycle their slots
#pragma unroll
        for (int d = 0; d < kD; ++d) {
          const int k = (gp * kD + d) % RS;
          if (gb + d < nrows) {
            C2 o;
            if constexpr (COMP) {
              o.x = acc_re[k] + lo_re[k];
              o.y = acc_im[k] + lo_im[k];
            } else {
              o.x = acc_re[k];
              o.y = acc_im[k];
            }
            grid[static_cast<size_t>(row0 + d) * N + col] = o;
            acc_re[k] = acc_im[k] = lo_re[k] = lo_im[k] = R(0);
          }
        }
      }
    }
  }
  // spill: slot q holds relative row nrows + ((q - nrows) mod RS); the W - 1 rows after
  // the item carry partial sums
  C2* sp = spill + static_cast<size_t>(slot) * RS * kStrip;
#pragma unroll
  for (int q = 0; q < RS; ++q) {
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

// Spill rows of work item w, run by the 32 lanes of a warp after every item stored its own
// rows: the W - 1 rows past the item (relative rows nrows + j, j < W - 1, held in ring slot
// (nrows + j) mod RS) are added into the grid. All of them are loaded before the first
// add, so that the warp waits for one round of loads.
template <typename R>
__device__ __forceinline__ void spill_item(const Item* __restrict__ items, int nfront, int item_cap, int W, int RS,
                                           int N, const typename Cplx<R>::T* __restrict__ spill,
                                           typename Cplx<R>::T* __restrict__ grid, int w, int lane) {
  constexpr int kMaxRows = 15;  // W - 1 for W <= 16
  const int slot = item_slot(w, nfront, item_cap);
  const Item item = items[slot];
  const int nrows = item.r1 - item.r0;
  if (nrows <= 0 || item.nrec == 0) return;
  const typename Cplx<R>::T* sp = spill + static_cast<size_t>(slot) * RS * kStrip + lane;
  typename Cplx<R>::T v[kMaxRows];
#pragma unroll
  for (int j = 0; j < kMaxRows; ++j)
    if (j < W - 1) v[j] = sp[((nrows + j) % RS) * kStrip];
  typename Cplx<R>::T* g = grid + item.strip * kStrip + lane;
#pragma unroll
  for (int j = 0; j < kMaxRows; ++j)
    if (j < W - 1) red_add(g + static_cast<size_t>((item.r1 + j) % N) * N, v[j]);
}

// One degridding work item, run by the 32 lanes of a warp (see grid_item).
template <int W, typename R, bool EXT = false>
__device__ __forceinline__ void degrid_item(const SweepArgs& a, const R* __restrict__ tab, unsigned char* my,
                                            const Item& item, int lane) {
  using C2 = typename Cplx<R>::T;
  using St = Stage<W, R>;
  constexpr int Wp = wpad<R>(W);
  constexpr int RS = Ring<W>::R, P = Ring<W>::P, TT = Ring<W>::T;
  constexpr bool kPk = sizeof(R) == 4;
  int* s_x0 = reinterpret_cast<int*>(my);
  R* s_cv = reinterpret_cast<R*>(my + St::x0_bytes);
  R* s_cu = reinterpret_cast<R*>(my + St::x0_bytes + St::cv_bytes);
  C2* s_p = reinterpret_cast<C2*>(my + St::x0_bytes + St::cv_bytes + St::cu_bytes);

  const Rec* __restrict__ recs = a.recs;
  const C2* __restrict__ G = static_cast<const C2*>(a.grid_in);
  C2* __restrict__ out = static_cast<C2*>(a.vis_out);
  const int N = a.N;

  if (item.nrec == 0) return;
  const int* __restrict__ off = a.offsets + static_cast<long long>(item.strip) * N;
  const int col = item.strip * kStrip + lane;
  const int nrows = item.r1 - item.r0;
  // ring slot x % RS holds grid row item.r0 + x of column `col`; rows 0 .. TT - kD - 1
  // are loaded up front, each group loads the kD rows that complete its window
  R g_re[RS], g_im[RS];
  unsigned long long g2[RS];
#pragma unroll
  for (int x = 0; x < TT - kD; ++x) {
    const C2 v = G[static_cast<size_t>((item.r0 + x) % N) * N + col];
    g_re[x] = v.x;
    g_im[x] = v.y;
    if constexpr (kPk) g2[x] = f2pack(float(v.x), float(v.y));
  }
  const int rb = off[item.r0], rend = off[item.r1];
  int wbase = rb, cstart = rb;
  Rec rc0{0u, 0, 0u, 0u}, rc1{0u, 0, 0u, 0u}, rc2{0u, 0, 0u, 0u};
  if (rb + lane < rend) rc0 = recs[rb + lane];
  if (rb + 32 + lane < rend) rc1 = recs[rb + 32 + lane];
  if (rb + 64 + lane < rend) rc2 = recs[rb + 64 + lane];
  for (int g0 = 0; g0 < nrows; g0 += RS) {
#pragma unroll
    for (int gp = 0; gp < P; ++gp) {
      const int gb = g0 + gp * kD;
      if (gb < nrows) {
        const int row0 = item.r0 + gb;
#pragma unroll
        for (int d = 0; d < kD; ++d) {
          const int x = gb + TT - kD + d;
          const C2 v = G[static_cast<size_t>((item.r0 + x) % N) * N + col];
          g_re[(gp * kD + TT - kD + d) % RS] = v.x;
          g_im[(gp * kD + TT - kD + d) % RS] = v.y;
          if constexpr (kPk) g2[(gp * kD + TT - kD + d) % RS] = f2pack(float(v.x), float(v.y));
        }
        const int re = off[min(row0 + kD, item.r1)];
        while (cstart < re) {
          const int ce = min(re, wbase + 32);
          const int lo = cstart - wbase, hi = ce - wbase;
          const bool mine = lane >= lo && lane < hi;
          const int xrel = rec_xrel(rc0.rx);
          if (mine) s_x0[lane] = xrel;
          int ou, ov;
          R fu, fv;
          table_coord<R, EXT>(Wp, a.Ms, a.interp, rc0.su, ou, fu);
          table_coord<R, EXT>(Wp, a.Ms, a.interp, rc0.sv, ov, fv);
          stage_chunk<W, R, false, EXT>(tab, Wp, a.interp, lo, hi, ou, fu, ov, fv, rec_row(rc0.rx) - row0, R(0), R(0),
                                   s_cv, s_cu, lane);
          const unsigned cover = mine ? cover_mask(xrel, W) : 0u;
          __syncwarp();
          unsigned M = transpose32(cover, lane);
          if constexpr (kPk) {
            while (M) {
              const int l1 = __ffs(M) - 1;
              M &= M - 1u;
              const bool two = M != 0u;
              const int l2 = two ? __ffs(M) - 1 : l1;
              if (two) M &= M - 1u;
              const int i1 = lane - s_x0[l1], i2 = lane - s_x0[l2];
              unsigned long long s1 = 0ull, s2 = 0ull;
#pragma unroll
              for (int q = 0; q < TT; ++q) {
                const R c1 = s_cv[q * Coop<W>::pitch + l1];
                const R c2 = s_cv[q * Coop<W>::pitch + l2];
                s1 = f2fma(f2pack(c1, c1), g2[(gp * kD + q) % RS], s1);
                s2 = f2fma(f2pack(c2, c2), g2[(gp * kD + q) % RS], s2);
              }
              s_p[l1 * W + i1] = f2unpack(s1);
              if (two) s_p[l2 * W + i2] = f2unpack(s2);
            }
          }
          while (M) {
            const int l = __ffs(M) - 1;
            M &= M - 1u;
            const int i = lane - s_x0[l];
            R sr = R(0), si = R(0);
            if constexpr (kPk) {
              unsigned long long s2 = 0ull;
#pragma unroll
              for (int q = 0; q < TT; ++q) {
                const R c = s_cv[q * Coop<W>::pitch + l];
                s2 = f2fma(f2pack(c, c), g2[(gp * kD + q) % RS], s2);
              }
              const float2 f = f2unpack(s2);
              sr = f.x;
              si = f.y;
            } else {
#pragma unroll
              for (int q = 0; q < TT; ++q) {
                const R c = s_cv[q * Coop<W>::pitch + l];
                sr = fma(c, g_re[(gp * kD + q) % RS], sr);
                si = fma(c, g_im[(gp * kD + q) % RS], si);
              }
            }
            C2 p;
            p.x = sr;
            p.y = si;
            s_p[l * W + i] = p;
          }
          __syncwarp();
          if (mine) {
            const int i0 = max(0, -xrel), i1 = min(W, kStrip - xrel);
            R vr = R(0), vi = R(0);
#pragma unroll
            for (int ii = 0; ii < W; ++ii) {
              if (ii < i0 || ii >= i1) continue;
              const C2 p = s_p[lane * W + ii];
              const R c = s_cu[lane * W + ii];
              vr = fma(c, p.x, vr);
              vi = fma(c, p.y, vi);
            }
            C2 o;
            o.x = vr;
            o.y = vi;
            // both records of a visibility crossing a strip add into the zeroed output
            // (two terms onto zero: the sum does not depend on their order)
            red_add(out + rc0.idx, o);
          }
          __syncwarp();
          cstart = ce;
          if (cstart == wbase + 32) {
            wbase += 32;
            rc0 = rc1;
            rc1 = rc2;
            if (wbase + 64 + lane < rend) rc2 = recs[wbase + 64 + lane];
          }
        }
      }
    }
  }
}

// Persistent single-plan sweep kernels: each warp takes work items from a counter and runs
// the per-item sweep. EXT selects the extended lookups (Lagrange, direct calculation),
// compiled separately so that the nearest / linear kernels keep their register budget.
template <int W, typename R, bool COMP, bool EXT>
__global__ void __launch_bounds__(kThreads, min_blocks<W, R, COMP, EXT>()) k_grid_sweep(const SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const R* tab = stage_table<R>(a.table, (a.Ms + 1) * a.Wp, a.table_in_smem != 0, smem);
  const size_t tab_bytes = a.table_in_smem ? align16(size_t(a.Ms + 1) * a.Wp * sizeof(R)) : 0;
  unsigned char* my = smem + tab_bytes + warp * align16(Stage<W, R>::grid_bytes);
  int nfront;
  const int total = work_total(a.counters, a.item_cap, nfront);
  for (int w = next_item(a.counters + kCntGridWork, lane); w < total; w = next_item(a.counters + kCntGridWork, lane))
    grid_item<W, R, COMP, EXT>(a, tab, my, item_slot(w, nfront, a.item_cap), lane);
}

template <int W, typename R, bool EXT>
__global__ void __launch_bounds__(kThreads, min_blocks<W, R, false, EXT>()) k_degrid_sweep(const SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const R* tab = stage_table<R>(a.table, (a.Ms + 1) * a.Wp, a.table_in_smem != 0, smem);
  const size_t tab_bytes = a.table_in_smem ? align16(size_t(a.Ms + 1) * a.Wp * sizeof(R)) : 0;
  unsigned char* my = smem + tab_bytes + warp * align16(Stage<W, R>::degrid_bytes);
  int nfront;
  const int total = work_total(a.counters, a.item_cap, nfront);
  for (int w = next_item(a.counters + kCntDegridWork, lane); w < total;
       w = next_item(a.counters + kCntDegridWork, lane)) {
    const Item item = a.items[item_slot(w, nfront, a.item_cap)];
    degrid_item<W, R, EXT>(a, tab, my, item, lane);
  }
}

template <bool EXT, int W> void* pick_sweep_kernel(int dtype, int accum, bool degrid) {
  if (degrid)
    return dtype ? reinterpret_cast<void*>(&k_degrid_sweep<W, double, EXT>)
                 : reinterpret_cast<void*>(&k_degrid_sweep<W, float, EXT>);
  if (dtype) return reinterpret_cast<void*>(&k_grid_sweep<W, double, false, EXT>);
  return accum ? reinterpret_cast<void*>(&k_grid_sweep<W, float, true, EXT>)
               : reinterpret_cast<void*>(&k_grid_sweep<W, float, false, EXT>);
}

template <bool EXT> void* sweep_kernel_pick(int W, int dtype, int accum, bool degrid) {
  switch (W) {
    case 1: return pick_sweep_kernel<EXT, 1>(dtype, accum, degrid);
    case 2: return pick_sweep_kernel<EXT, 2>(dtype, accum, degrid);
    case 3: return pick_sweep_kernel<EXT, 3>(dtype, accum, degrid);
    case 4: return pick_sweep_kernel<EXT, 4>(dtype, accum, degrid);
    case 5: return pick_sweep_kernel<EXT, 5>(dtype, accum, degrid);
    case 6: return pick_sweep_kernel<EXT, 6>(dtype, accum, degrid);
    case 7: return pick_sweep_kernel<EXT, 7>(dtype, accum, degrid);
    case 8: return pick_sweep_kernel<EXT, 8>(dtype, accum, degrid);
    case 9: return pick_sweep_kernel<EXT, 9>(dtype, accum, degrid);
    case 10: return pick_sweep_kernel<EXT, 10>(dtype, accum, degrid);
    case 11: return pick_sweep_kernel<EXT, 11>(dtype, accum, degrid);
    case 12: return pick_sweep_kernel<EXT, 12>(dtype, accum, degrid);
    case 13: return pick_sweep_kernel<EXT, 13>(dtype, accum, degrid);
    case 14: return pick_sweep_kernel<EXT, 14>(dtype, accum, degrid);
    case 15: return pick_sweep_kernel<EXT, 15>(dtype, accum, degrid);
    case 16: return pick_sweep_kernel<EXT, 16>(dtype, accum, degrid);
    default: return nullptr;
  }
}

// Staging bytes of one warp (runtime W).
inline size_t stage_bytes(int W, int dtype, bool degrid) {
  const size_t rs = dtype ? 8 : 4;
  const int T = W + kD - 1;
  const size_t x0 = 32 * sizeof(int), cv = align16(size_t(T) * (32 + 32 / coop_group(W)) * rs),
               cu = 32 * size_t(W) * rs, ab = 32 * W * 2 * rs;
  return align16(x0 + cv + (degrid ? cu : 0) + ab);
}

}  // namespace
}  // namespace lmg

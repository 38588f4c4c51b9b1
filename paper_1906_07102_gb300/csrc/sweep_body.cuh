// Gridding and degridding sweeps (Eqs. 5-6 and their transpose, Section 4): the per-item
// device code shared by the single-plan kernels (sweep.cu, sweep_ext.cu) and the
// multi-channel persistent kernels (batch.cu).
//
// The grid is cut into strips of S = 32 KC columns; a warp owns one work item (a range of
// rows of one strip) and lane t owns the KC adjacent columns KC t .. KC t + KC - 1 of the
// strip (KC = 2 for complex64, 1 for complex128). The item's records come grouped by pairs
// of support-start rows (dealt inside a pair by the binning, so that 32 consecutive records
// spread over the pair's columns) and are visited in groups of kD = 2 rows, in chunks of up
// to 32 records (the records and visibilities of the next two chunks already in flight):
//   1. each record's own lane looks up its 2W table weights (Section 5.1) and stages them:
//      Cv shifted by the record's row offset d in the group (entry q weights group row q,
//      q < TP, the window T = W + kD - 1 rounded up to even and zero-padded), record-major
//      so that a visiting lane reads it with 16-byte loads; and per covered lane one slot of
//      KC column weights: Cu_i w V (gridding) or Cu_i (degridding). Slot (lane mod PS) of a
//      record belongs to the lane that reads it, so no lane needs the record's start column;
//   2. each lane builds the set of records whose support covers one of its columns (32x32
//      bit transpose of the per-record lane masks) and visits them, two per iteration.
//      Degridding stages and transposes once per window of 32 consecutive records (lane l
//      holding record l, whatever row pair it belongs to; row pairs start at even rows, so
//      d = row & 1) and visits each chunk's part of the window's set: the same records in
//      the same order, with a window that spans several sparse row pairs staged once;
//   3. gridding: lane t holds a ring of RS >= TP accumulator rows for each of its columns in
//      registers, as pairs of rows (one f32x2 register per pair for complex64), and adds
//      (Cv'_q, Cv'_q+1) x (a, a) with one packed FMA per pair and per real/imaginary part --
//      the ring index is compile-time, the group loop being unrolled over one ring period.
//      After a group its kD rows are final and stored as whole rows (512-byte coalesced
//      stores for complex64). The W-1 rows past the item go to a spill buffer and are added
//      by k_grid_spill once all items have stored their rows.
//      degridding: the ring holds grid rows of the lane's columns; the lane forms
//      sum_q Cv'_q G[row0 + q][c] for its columns, weights them by its Cu slot and stages the
//      sum in the record's partial-sum slot; the record's lane adds its slots and adds the
//      result to the zeroed output (a visibility whose support crosses a strip has two
//      records, one per strip).
// Every grid cell is written exactly once by the gridding sweep (no pre-zeroing, no
// shared-memory atomics); only the spill rows are added with global vector atomics.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "device_common.cuh"
#include "kernels.h"

namespace lmg {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Rows per group and the register ring: RS >= TP slots, a multiple of kD, so that the
// group loop unrolled over P = RS / kD groups indexes every slot at compile time.
constexpr int kD = 2;  // the binning's row pairs (bin.cu) are these groups
template <int W> struct Ring {
  static constexpr int T = W + kD - 1;       // rows a group's records can touch
  static constexpr int TP = 2 * ((T + 1) / 2);  // staged entries: T rounded up to pairs
  static constexpr int R = kD * ((TP + kD - 1) / kD);
  static constexpr int P = R / kD;
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Columns per lane: 2 for complex64 (64-column strips), 1 for complex128 (32 columns).
template <typename R> __host__ __device__ constexpr int cols_per_lane() { return sizeof(R) == 4 ? 2 : 1; }

// Staging layout of one warp.
template <int W, typename R> struct Lay {
  static constexpr int KC = cols_per_lane<R>();
  static constexpr int TP = Ring<W>::TP;
  // Cv' record-major, CVS reals per record (an odd number of 16-byte units)
  static constexpr int CVS = ((((TP * int(sizeof(R)) + 15) / 16) | 1) * 16) / int(sizeof(R));
  // lanes one record can cover, and the slots per record (a power of two >= NL)
  static constexpr int NL = (W - 1 + KC - 1) / KC + 1;
  static constexpr int PS = NL <= 2 ? 2 : (NL <= 4 ? 4 : (NL <= 8 ? 8 : 16));
  // slot sizes: the KC complex column weights a = Cu w V of gridding, KC reals Cu
  // (degridding), one complex (degridding partial sum). A record's slots are followed by 16 bytes of padding,
  // an odd number of 16-byte units per record (or of 8-byte words for 8-byte slots), which
  // spreads the records over the banks.
  static constexpr int SA = KC * 2 * int(sizeof(R));
  static constexpr int SU = KC * int(sizeof(R));
  static constexpr int SP = 2 * int(sizeof(R));
  static constexpr int AP = PS * SA + 16;
  static constexpr int UP = (PS + 1) * SU;
  static constexpr int PP = (PS + 1) * SP;
  // 33 records per chunk area: record 32 stays zero and stands in for a missing second
  // record of an inner-loop iteration
  static constexpr int NREC = 33;
  static constexpr size_t cv_bytes = size_t(NREC) * CVS * sizeof(R);
  static constexpr size_t a_bytes = size_t(NREC) * AP;
  static constexpr size_t u_bytes = size_t(NREC) * UP;
  static constexpr size_t p_bytes = size_t(NREC) * PP;
  static constexpr size_t grid_bytes = align16(cv_bytes + a_bytes);
  static constexpr size_t degrid_bytes = align16(cv_bytes + align16(u_bytes) + p_bytes);
};

// Pairs of rows in one register: f32x2 for float (Blackwell's packed FMA), two doubles.
template <typename R> struct PairOf;
template <> struct PairOf<float> { using T = unsigned long long; };
template <> struct PairOf<double> { using T = double2; };

__device__ __forceinline__ unsigned long long pfma(unsigned long long a, unsigned long long b, unsigned long long c) {
  return f2fma(a, b, c);
}
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ unsigned long long pdup(float x) { return f2pack(x, x); }
__device__ __forceinline__ double2 pdup(double x) { return make_double2(x, x); }
template <typename P> __device__ __forceinline__ P pzero();
template <> __device__ __forceinline__ unsigned long long pzero<unsigned long long>() { return 0ull; }
template <> __device__ __forceinline__ double2 pzero<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float plo(unsigned long long p) { return f2unpack(p).x; }
__device__ __forceinline__ float phi(unsigned long long p) { return f2unpack(p).y; }
__device__ __forceinline__ double plo(double2 p) { return p.x; }
__device__ __forceinline__ double phi(double2 p) { return p.y; }
__device__ __forceinline__ float psum(unsigned long long p) {
  const float2 v = f2unpack(p);
  return v.x + v.y;
}
__device__ __forceinline__ double psum(double2 p) { return p.x + p.y; }

// Packed error-free addition (Knuth TwoSum on both halves): a receives the rounded sum,
// lo accumulates the rounding errors (compensated accumulation, complex64 only).
__device__ __forceinline__ void two_sum_pair(unsigned long long& a, unsigned long long& lo, unsigned long long b) {
  unsigned long long s, bp, ap, ea, eb;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s) : "l"(a), "l"(b));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(bp) : "l"(s), "l"(a));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ap) : "l"(s), "l"(bp));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ea) : "l"(a), "l"(ap));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(eb) : "l"(b), "l"(bp));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(ea) : "l"(ea), "l"(eb));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(lo) : "l"(lo), "l"(ea));
  a = s;
}
__device__ __forceinline__ unsigned long long pmul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

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

// The same for float64 plans from the exact coordinate s = fl(S 2^-32 + delta), delta the
// quantisation residual u_q - u of the binning: rows as above from the integer product
// S Ms, fraction f = fl(s Ms) - k (and f = s for the direct calculation), so that the
// weights keep the full float64 precision of the position.
template <bool EXT>
__device__ __forceinline__ void table_coord_exact(int Wp, int Ms, int interp, unsigned S, double delta, int& off,
                                                  double& f) {
  const double s = __dadd_rn(static_cast<double>(S) * 2.3283064365386962890625e-10, delta);
  const double t = __dmul_rn(s, static_cast<double>(Ms));
  const unsigned long long Pm = static_cast<unsigned long long>(S) * static_cast<unsigned>(Ms);
  if constexpr (!EXT) {
    if (interp) {
      const long long k = static_cast<long long>(Pm >> 32);
      off = static_cast<int>(k) * Wp;
      f = __dsub_rn(t, static_cast<double>(k));
    } else {
      off = static_cast<int>((Pm + 0x80000000ull) >> 32) * Wp;
      f = 0.0;
    }
  } else if (interp == 4) {
    off = 0;
    f = s;
  } else {
    const long long P = static_cast<long long>(Pm);
    long long k0 = (P - static_cast<long long>(interp - 1) * 0x80000000ll) >> 32;
    k0 = k0 < 0 ? 0 : (k0 > Ms - interp ? Ms - interp : k0);
    off = static_cast<int>(k0) * Wp;
    f = __dsub_rn(t, static_cast<double>(k0));
  }
}

// Row offsets and fractions of a record for both axes (exact coordinates for float64 plans
// that carry quantisation residuals).
template <typename R, bool EXT>
__device__ __forceinline__ void record_coords(const SweepArgs& a, const Rec& rc, int& ou, R& fu, int& ov, R& fv) {
  if constexpr (sizeof(R) == 8) {
    if (a.frac != nullptr) {
      const double2 dl = a.frac[rc.idx];
      table_coord_exact<EXT>(a.Wp, a.Ms, a.interp, rc.su, dl.x, ou, fu);
      table_coord_exact<EXT>(a.Wp, a.Ms, a.interp, rc.sv, dl.y, ov, fv);
      return;
    }
  }
  table_coord<R, EXT>(a.Wp, a.Ms, a.interp, rc.su, ou, fu);
  table_coord<R, EXT>(a.Wp, a.Ms, a.interp, rc.sv, ov, fv);
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

// 16-byte vector of reals.
template <typename R> struct Vec16;
template <> struct Vec16<float> {
  using T = float4;
  static constexpr int N = 4;
};
template <> struct Vec16<double> {
  using T = double2;
  static constexpr int N = 2;
};
template <typename R> __device__ __forceinline__ R vget(const typename Vec16<R>::T& v, int k);
template <> __device__ __forceinline__ float vget<float>(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
template <> __device__ __forceinline__ double vget<double>(const double2& v, int k) { return k == 0 ? v.x : v.y; }

// The W table weights at one coordinate (row offset `off`, fraction f): nearest / linear
// rows read with 16-byte loads, or the extended lookups (Lagrange, direct calculation).
template <int W, typename R, bool EXT>
__device__ __forceinline__ void lookup(const R* __restrict__ tab, int Wp, int interp, int off, R f, R (&c)[W]) {
  if constexpr (!EXT) {
    using V = typename Vec16<R>::T;
    constexpr int VE = Vec16<R>::N, NV = (W + VE - 1) / VE;
    const V* p0 = reinterpret_cast<const V*>(tab + off);
    V r0[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) r0[v] = p0[v];
    if (interp) {
      const V* p1 = reinterpret_cast<const V*>(tab + off + Wp);
      V r1[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) r1[v] = p1[v];
#pragma unroll
      for (int i = 0; i < W; ++i) {
        const R a = vget<R>(r0[i / VE], i % VE);
        c[i] = a + f * (vget<R>(r1[i / VE], i % VE) - a);
      }
    } else {
#pragma unroll
      for (int i = 0; i < W; ++i) c[i] = vget<R>(r0[i / VE], i % VE);
    }
  } else {
    // direct calculation exists for float64 plans and W <= 11 only (plan creation)
    if constexpr (sizeof(R) == 8 && W <= 11) {
      if (interp == 4) {
#pragma unroll 1
        for (int i = 0; i < W; ++i) c[i] = direct_entry<R>(tab, W, i, f);
        return;
      }
    }
#pragma unroll
    for (int i = 0; i < W; ++i) c[i] = lagrange_entry<R>(tab + off + i, Wp, interp, f);
  }
}

// Stages Cv' (Cv shifted by the row offset d in {0, 1}, zero outside) record-major at dst
// (TP reals, 16-byte aligned), with 16-byte stores.
template <int W, typename R>
__device__ __forceinline__ void stage_cv(const R (&cv)[W], int d, R* __restrict__ dst) {
  using V = typename Vec16<R>::T;
  constexpr int TP = Ring<W>::TP, VE = Vec16<R>::N, NV = (TP + VE - 1) / VE;
  R e[NV * VE];
#pragma unroll
  for (int q = 0; q < NV * VE; ++q) {
    const R c0 = q < W ? cv[q] : R(0);            // d = 0: entry q is Cv_q
    const R c1 = (q >= 1 && q <= W) ? cv[q - 1] : R(0);  // d = 1: entry q is Cv_{q-1}
    e[q] = d ? c1 : c0;
  }
  V* out = reinterpret_cast<V*>(dst);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    V x;
    if constexpr (sizeof(R) == 4) x = make_float4(e[4 * v], e[4 * v + 1], e[4 * v + 2], e[4 * v + 3]);
    else x = make_double2(e[2 * v], e[2 * v + 1]);
    out[v] = x;
  }
}

// Column weights of record xrel (support start column relative to the strip) for covered
// lane L0 + m: entry j < KC is the weight of column KC (L0 + m) + j, i.e. of support index
// i = KC m + j - (xrel mod KC); zero outside [0, W).
template <int W, int KC> __device__ __forceinline__ int slot_index(int m, int j, int par) { return KC * m + j - par; }

// Gridding stage of a record by its own lane: Cv' and the slots a = Cu w V.
template <int W, typename R, bool EXT>
__device__ __forceinline__ void stage_grid(const R* __restrict__ tab, int Wp, int interp, int ou, R fu, int ov, R fv,
                                           int d, int xrel, R wx, R wy, unsigned char* __restrict__ s_cv,
                                           unsigned char* __restrict__ s_a, int lane) {
  using L = Lay<W, R>;
  constexpr int KC = L::KC;
  R cu[W], cv[W];
  lookup<W, R, EXT>(tab, Wp, interp, ou, fu, cu);
  lookup<W, R, EXT>(tab, Wp, interp, ov, fv, cv);
  stage_cv<W, R>(cv, d, reinterpret_cast<R*>(s_cv) + lane * L::CVS);
  unsigned char* rec = s_a + lane * L::AP;
  const int L0 = xrel >> (KC - 1), par = xrel & (KC - 1);
#pragma unroll
  for (int m = 0; m < L::NL; ++m) {
    R v[2 * KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      R re = R(0), im = R(0);
#pragma unroll
      for (int pp = 0; pp < KC; ++pp) {  // par is runtime: pick the support index by parity
        const int i = slot_index<W, KC>(m, j, pp);
        if (pp == par && i >= 0 && i < W) {
          re = cu[i] * wx;
          im = cu[i] * wy;
        }
      }
      v[2 * j] = re;
      v[2 * j + 1] = im;
    }
    unsigned char* dst = rec + ((L0 + m) & (L::PS - 1)) * L::SA;
    if constexpr (sizeof(R) == 4) {
      static_assert(KC == 2, "complex64 lanes own two columns");
      *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int j = 0; j < KC; ++j) reinterpret_cast<double2*>(dst)[j] = make_double2(v[2 * j], v[2 * j + 1]);
    }
  }
}

// Degridding stage of a record by its own lane: Cv' and the slots of Cu.
template <int W, typename R, bool EXT>
__device__ __forceinline__ void stage_degrid(const R* __restrict__ tab, int Wp, int interp, int ou, R fu, int ov, R fv,
                                             int d, int xrel, unsigned char* __restrict__ s_cv,
                                             unsigned char* __restrict__ s_u, int lane) {
  using L = Lay<W, R>;
  constexpr int KC = L::KC;
  R cu[W], cv[W];
  lookup<W, R, EXT>(tab, Wp, interp, ou, fu, cu);
  lookup<W, R, EXT>(tab, Wp, interp, ov, fv, cv);
  stage_cv<W, R>(cv, d, reinterpret_cast<R*>(s_cv) + lane * L::CVS);
  unsigned char* rec = s_u + lane * L::UP;
  const int L0 = xrel >> (KC - 1), par = xrel & (KC - 1);
#pragma unroll
  for (int m = 0; m < L::NL; ++m) {
    R v[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      R c = R(0);
#pragma unroll
      for (int pp = 0; pp < KC; ++pp) {
        const int i = slot_index<W, KC>(m, j, pp);
        if (pp == par && i >= 0 && i < W) c = cu[i];
      }
      v[j] = c;
    }
    unsigned char* dst = rec + ((L0 + m) & (L::PS - 1)) * L::SU;
    if constexpr (sizeof(R) == 4 && KC == 2) *reinterpret_cast<float2*>(dst) = make_float2(v[0], v[1]);
    else *reinterpret_cast<R*>(dst) = v[0];
  }
}

// Zeroes the stand-in record 32 of a warp's staging area (its Cv' and its slots).
__device__ __forceinline__ void zero_bytes(unsigned char* p, int bytes, int lane) {
  for (int i = 4 * lane; i < bytes; i += 128) *reinterpret_cast<int*>(p + i) = 0;
}

// Support-start row offsets of an item's row pairs, 32 pairs per block: lane t holds the
// end offset of pair 32 b + t (the offset of row min(r0 + 2 (32 b + t + 1), r1)).
__device__ __forceinline__ int pair_ends(const int* __restrict__ off, const Item& item, int b, int lane) {
  return off[min(item.r0 + 2 * (32 * b + lane + 1), item.r1)];
}

// Lanes L0 .. L1 (inclusive) intersected with [0, 32).
__device__ __forceinline__ unsigned lane_range_mask(int L0, int L1) {
  const int a = L0 < 0 ? 0 : L0, b = L1 > 31 ? 31 : L1;
  if (a > b) return 0u;
  return (0xffffffffu >> (31 - b)) & (0xffffffffu << a);
}
// Bits a .. b - 1 of a window's record mask (0 <= a < b <= 32).
__device__ __forceinline__ unsigned record_range(int a, int b) {
  return (b >= 32 ? 0xffffffffu : ((1u << b) - 1u)) & ~((1u << a) - 1u);
}
template <int W, int KC> __device__ __forceinline__ unsigned cover_lanes(int xrel) {
  return lane_range_mask(xrel >> (KC - 1), (xrel + W - 1) >> (KC - 1));
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

// Resident CTAs per SM the register allocation must allow.
template <int W, typename R, bool COMP = false, bool EXT = false> constexpr int min_blocks() {
  return (sizeof(R) == 4 && W <= 8 && !COMP) ? 2 : 1;
}

// KC complex values of one row of a lane's columns: 16-byte store / load.
template <typename R, int KC>
__device__ __forceinline__ void store_cols(typename Cplx<R>::T* dst, const R (&re)[KC], const R (&im)[KC]) {
  if constexpr (sizeof(R) == 4 && KC == 2) {
    *reinterpret_cast<float4*>(dst) = make_float4(re[0], im[0], re[1], im[1]);
  } else {
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      typename Cplx<R>::T o;
      o.x = re[j];
      o.y = im[j];
      dst[j] = o;
    }
  }
}
template <typename R, int KC>
__device__ __forceinline__ void load_cols(const typename Cplx<R>::T* src, R (&re)[KC], R (&im)[KC]) {
  if constexpr (sizeof(R) == 4 && KC == 2) {
    const float4 v = *reinterpret_cast<const float4*>(src);
    re[0] = v.x;
    im[0] = v.y;
    re[1] = v.z;
    im[1] = v.w;
  } else {
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      const typename Cplx<R>::T v = src[j];
      re[j] = v.x;
      im[j] = v.y;
    }
  }
}

// Loads one gridding slot (KC complex a = Cu w V) as (a_re, a_re) and (a_im, a_im) per column,
// ready for the packed FMA (measured faster than staging the pairs duplicated, which doubles
// the slot loads).
template <typename R, int KC>
__device__ __forceinline__ void load_slot(const unsigned char* p, typename PairOf<R>::T (&a)[KC][2]) {
  if constexpr (sizeof(R) == 4) {
    static_assert(KC == 2, "complex64 lanes own two columns");
    const float4 x = *reinterpret_cast<const float4*>(p);
    a[0][0] = pdup(x.x);
    a[0][1] = pdup(x.y);
    a[1][0] = pdup(x.z);
    a[1][1] = pdup(x.w);
  } else {
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      const double2 x = reinterpret_cast<const double2*>(p)[j];
      a[j][0] = pdup(x.x);
      a[j][1] = pdup(x.y);
    }
  }
}

// Loads the Cv' pairs of record l.
template <int W, typename R>
__device__ __forceinline__ void load_cv_pairs(const unsigned char* s_cv, int l,
                                              typename PairOf<R>::T (&c)[Ring<W>::TP / 2]) {
  using L = Lay<W, R>;
  constexpr int NPR = Ring<W>::TP / 2;
  const R* p = reinterpret_cast<const R*>(s_cv) + l * L::CVS;
  if constexpr (sizeof(R) == 4) {
    const ulonglong2* v = reinterpret_cast<const ulonglong2*>(p);
#pragma unroll
    for (int m = 0; m < NPR / 2; ++m) {
      const ulonglong2 x = v[m];
      c[2 * m] = x.x;
      c[2 * m + 1] = x.y;
    }
    if constexpr (NPR % 2) c[NPR - 1] = reinterpret_cast<const unsigned long long*>(p)[NPR - 1];
  } else {
    const double2* v = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int m = 0; m < NPR; ++m) c[m] = v[m];
  }
}

// One gridding work item (rows [r0, r1) of one strip), run by the 32 lanes of a warp;
// `my` is the warp's staging area in shared memory, `tab` the table (shared or global).
template <int W, typename R, bool COMP, bool EXT = false>
__device__ __forceinline__ void grid_item(const SweepArgs& a, const R* __restrict__ tab, unsigned char* my,
                                          int slot, int lane) {
  using C2 = typename Cplx<R>::T;
  using P = typename PairOf<R>::T;
  using L = Lay<W, R>;
  constexpr int KC = L::KC, S = 32 * KC;
  constexpr int RS = Ring<W>::R, NP = Ring<W>::P, NPR = Ring<W>::TP / 2, RH = RS / 2;
  static_assert(!COMP || sizeof(R) == 4, "compensated accumulation is for complex64");
  unsigned char* s_cv = my;
  unsigned char* s_a = my + L::cv_bytes;

  const Rec* __restrict__ recs = a.recs;
  const C2* __restrict__ vis = static_cast<const C2*>(a.vis);
  const R* __restrict__ wts = static_cast<const R*>(a.weights);
  C2* __restrict__ grid = static_cast<C2*>(a.grid);
  C2* __restrict__ spill = static_cast<C2*>(a.spill);
  const int N = a.N, Wp = a.Wp;

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
  const int col0 = item.strip * S + KC * lane;
  const int nrows = item.r1 - item.r0;
  // ring pair h holds relative rows 2h' and 2h' + 1 (h' = h mod RH) of the lane's columns
  P accR[KC][RH], accI[KC][RH];
  P loR[COMP ? KC : 1][COMP ? RH : 1], loI[COMP ? KC : 1][COMP ? RH : 1];
#pragma unroll
  for (int j = 0; j < KC; ++j)
#pragma unroll
    for (int h = 0; h < RH; ++h) accR[j][h] = accI[j][h] = pzero<P>();
  if constexpr (COMP) {
#pragma unroll
    for (int j = 0; j < KC; ++j)
#pragma unroll
      for (int h = 0; h < RH; ++h) loR[j][h] = loI[j][h] = pzero<P>();
  }
  const int myslot = lane & (L::PS - 1);
  zero_bytes(s_cv + 32 * L::CVS * sizeof(R), L::CVS * sizeof(R), lane);
  zero_bytes(s_a + 32 * L::AP, L::AP, lane);
  // software pipeline over 32-record windows of the item (window k = records
  // rb + 32k .. rb + 32k + 31, lane l holding record rb + 32k + l): while window k is
  // processed, the visibilities of window k+1 and the records of window k+2 are in flight
  const int rb = off[item.r0], rend = off[item.r1];
  int pend = pair_ends(off, item, 0, lane);
  int wbase = rb, cstart = rb;
  Fetch<R> f0{}, f1{}, f2{};
  fetch_rec(rb, rend, f0);
  fetch_rec(rb + 32, rend, f1);
  fetch_vis(rb, rend, f0);
  fetch_vis(rb + 32, rend, f1);
  fetch_rec(rb + 64, rend, f2);
  for (int g0 = 0; g0 < nrows; g0 += RS) {
#pragma unroll
    for (int gp = 0; gp < NP; ++gp) {
      const int gb = g0 + gp * kD;
      if (gb < nrows) {
        const int row0 = item.r0 + gb;
        if (gb > 0 && (gb & 63) == 0) pend = pair_ends(off, item, gb >> 6, lane);
        const int re = __shfl_sync(0xffffffffu, pend, (gb & 63) >> 1);
        while (cstart < re) {
          // chunk: records [cstart, ce) of window wbase, staged by lanes cstart - wbase ..
          const int ce = min(re, wbase + 32);
          const bool mine = lane >= cstart - wbase && lane < ce - wbase;
          const int xrel = rec_xrel(f0.rc.rx);
          if (mine) {
            int ou, ov;
            R fu, fv;
            record_coords<R, EXT>(a, f0.rc, ou, fu, ov, fv);
            stage_grid<W, R, EXT>(tab, Wp, a.interp, ou, fu, ov, fv, rec_row(f0.rc.rx) - row0, xrel,
                                  f0.v.x * f0.wt, f0.v.y * f0.wt, s_cv, s_a, lane);
          }
          const unsigned cover = mine ? cover_lanes<W, KC>(xrel) : 0u;
          __syncwarp();
          unsigned M = transpose32(cover, lane);
          while (M) {
            const int l1 = __ffs(M) - 1;
            M &= M - 1u;
            const int l2 = M ? __ffs(M) - 1 : 32;  // record 32 is zero
            M &= M - 1u;
            P c1[NPR], c2[NPR];
            load_cv_pairs<W, R>(s_cv, l1, c1);
            load_cv_pairs<W, R>(s_cv, l2, c2);
            P a1[KC][2], a2[KC][2];
            load_slot<R, KC>(s_a + l1 * L::AP + myslot * L::SA, a1);
            load_slot<R, KC>(s_a + l2 * L::AP + myslot * L::SA, a2);
#pragma unroll
            for (int j = 0; j < KC; ++j) {
              const P d1r = a1[j][0], d1i = a1[j][1], d2r = a2[j][0], d2i = a2[j][1];
#pragma unroll
              for (int m = 0; m < NPR; ++m) {
                const int h = (gp + m) % RH;
                if constexpr (COMP) {
                  two_sum_pair(accR[j][h], loR[j][h], pmul(c1[m], d1r));
                  two_sum_pair(accI[j][h], loI[j][h], pmul(c1[m], d1i));
                  two_sum_pair(accR[j][h], loR[j][h], pmul(c2[m], d2r));
                  two_sum_pair(accI[j][h], loI[j][h], pmul(c2[m], d2i));
                } else {
                  accR[j][h] = pfma(c2[m], d2r, pfma(c1[m], d1r, accR[j][h]));
                  accI[j][h] = pfma(c2[m], d2i, pfma(c1[m], d1i, accI[j][h]));
                }
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
        // rows row0 and row0 + 1 (ring pair gp mod RH) are complete: store them, recycle
        const int h = gp % RH;
#pragma unroll
        for (int d = 0; d < kD; ++d) {
          if (gb + d < nrows) {
            R orr[KC], oi[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) {
              if constexpr (COMP) {
                orr[j] = (d ? phi(accR[j][h]) : plo(accR[j][h])) + (d ? phi(loR[j][h]) : plo(loR[j][h]));
                oi[j] = (d ? phi(accI[j][h]) : plo(accI[j][h])) + (d ? phi(loI[j][h]) : plo(loI[j][h]));
              } else {
                orr[j] = d ? phi(accR[j][h]) : plo(accR[j][h]);
                oi[j] = d ? phi(accI[j][h]) : plo(accI[j][h]);
              }
            }
            store_cols<R, KC>(grid + static_cast<size_t>(row0 + d) * N + col0, orr, oi);
          }
        }
#pragma unroll
        for (int j = 0; j < KC; ++j) {
          accR[j][h] = accI[j][h] = pzero<P>();
          if constexpr (COMP) loR[j][h] = loI[j][h] = pzero<P>();
        }
      }
    }
  }
  // spill: ring pair h holds relative rows nrows + ((2h - nrows) mod RS) (and the next);
  // the W - 1 rows after the item carry partial sums
  C2* sp = spill + static_cast<size_t>(slot) * RS * S + KC * lane;
#pragma unroll
  for (int h = 0; h < RH; ++h) {
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      R orr[KC], oi[KC];
#pragma unroll
      for (int j = 0; j < KC; ++j) {
        if constexpr (COMP) {
          orr[j] = (d ? phi(accR[j][h]) : plo(accR[j][h])) + (d ? phi(loR[j][h]) : plo(loR[j][h]));
          oi[j] = (d ? phi(accI[j][h]) : plo(accI[j][h])) + (d ? phi(loI[j][h]) : plo(loI[j][h]));
        } else {
          orr[j] = d ? phi(accR[j][h]) : plo(accR[j][h]);
          oi[j] = d ? phi(accI[j][h]) : plo(accI[j][h]);
        }
      }
      store_cols<R, KC>(sp + static_cast<size_t>(2 * h + d) * S, orr, oi);
    }
  }
}

// Spill rows of work item w, run by the 32 lanes of a warp after every item stored its own
// rows: the W - 1 rows past the item (relative rows nrows + j, j < W - 1, held in ring slot
// (nrows + j) mod RS) are added into the grid. All of them are loaded before the first
// add, so that the warp waits for one round of loads. S = 32 KC columns, KC per lane.
template <typename R>
__device__ __forceinline__ void spill_item(const Item* __restrict__ items, int nfront, int item_cap, int W, int RS,
                                           int N, int S, const typename Cplx<R>::T* __restrict__ spill,
                                           typename Cplx<R>::T* __restrict__ grid, int w, int lane) {
  constexpr int kMaxRows = 15;  // W - 1 for W <= 16
  constexpr int KC = cols_per_lane<R>();
  const int slot = item_slot(w, nfront, item_cap);
  const Item item = items[slot];
  const int nrows = item.r1 - item.r0;
  if (nrows <= 0 || item.nrec == 0) return;
  const typename Cplx<R>::T* sp = spill + static_cast<size_t>(slot) * RS * S + KC * lane;
  R vr[kMaxRows][KC], vi[kMaxRows][KC];
#pragma unroll
  for (int j = 0; j < kMaxRows; ++j)
    if (j < W - 1) load_cols<R, KC>(sp + static_cast<size_t>((nrows + j) % RS) * S, vr[j], vi[j]);
  typename Cplx<R>::T* g = grid + static_cast<size_t>(item.strip) * S + KC * lane;
#pragma unroll
  for (int j = 0; j < kMaxRows; ++j)
    if (j < W - 1) {
      typename Cplx<R>::T* dst = g + static_cast<size_t>((item.r1 + j) % N) * N;
      if constexpr (sizeof(R) == 4 && KC == 2) {
        red_add2(dst, make_float2(vr[j][0], vi[j][0]), make_float2(vr[j][1], vi[j][1]));
      } else {
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          typename Cplx<R>::T v;
          v.x = vr[j][c];
          v.y = vi[j][c];
          red_add(dst + c, v);
        }
      }
    }
}

// One degridding work item, run by the 32 lanes of a warp (see grid_item).
template <int W, typename R, bool EXT = false>
__device__ __forceinline__ void degrid_item(const SweepArgs& a, const R* __restrict__ tab, unsigned char* my,
                                            const Item& item, int lane) {
  using C2 = typename Cplx<R>::T;
  using P = typename PairOf<R>::T;
  using L = Lay<W, R>;
  constexpr int KC = L::KC, S = 32 * KC;
  constexpr int RS = Ring<W>::R, NP = Ring<W>::P, NPR = Ring<W>::TP / 2, RH = RS / 2;
  unsigned char* s_cv = my;
  unsigned char* s_u = my + L::cv_bytes;
  unsigned char* s_p = my + L::cv_bytes + align16(L::u_bytes);

  const Rec* __restrict__ recs = a.recs;
  const C2* __restrict__ G = static_cast<const C2*>(a.grid_in);
  C2* __restrict__ out = static_cast<C2*>(a.vis_out);
  const int N = a.N, Wp = a.Wp;

  if (item.nrec == 0) return;
  const int* __restrict__ off = a.offsets + static_cast<long long>(item.strip) * N;
  const int col0 = item.strip * S + KC * lane;
  const int nrows = item.r1 - item.r0;
  // ring pair h holds grid rows item.r0 + 2h' and + 1 (h' = h mod RH) of the lane's columns;
  // rows 0 .. TP - 3 are loaded up front; each group moves the pair that completes its
  // window into the ring (loaded during the previous group) and loads the next group's
  P gR[KC][RH], gI[KC][RH];
  R nr0[KC], ni0[KC], nr1[KC], ni1[KC];  // the next window-completing pair, in flight
  auto fetch_pair = [&](int x) {  // relative rows x, x + 1
    load_cols<R, KC>(G + static_cast<size_t>((item.r0 + x) % N) * N + col0, nr0, ni0);
    load_cols<R, KC>(G + static_cast<size_t>((item.r0 + x + 1) % N) * N + col0, nr1, ni1);
  };
  auto put_pair = [&](int h) {
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      if constexpr (sizeof(R) == 4) {
        gR[j][h] = f2pack(nr0[j], nr1[j]);
        gI[j][h] = f2pack(ni0[j], ni1[j]);
      } else {
        gR[j][h] = make_double2(nr0[j], nr1[j]);
        gI[j][h] = make_double2(ni0[j], ni1[j]);
      }
    }
  };
#pragma unroll
  for (int h = 0; h < NPR - 1; ++h) {
    fetch_pair(2 * h);
    put_pair(h);
  }
  fetch_pair(2 * (NPR - 1));
  const int myslot = lane & (L::PS - 1);
  zero_bytes(s_cv + 32 * L::CVS * sizeof(R), L::CVS * sizeof(R), lane);
  zero_bytes(s_u + 32 * L::UP, L::UP, lane);
  const int rb = off[item.r0], rend = off[item.r1];
  int pend = pair_ends(off, item, 0, lane);
  int wbase = rb, cstart = rb;
  int staged = -1;    // window whose records are staged
  unsigned MW = 0u;   // records of that window covering this lane's columns
  Rec rc0{0u, 0, 0u, 0u}, rc1{0u, 0, 0u, 0u}, rc2{0u, 0, 0u, 0u};
  if (rb + lane < rend) rc0 = recs[rb + lane];
  if (rb + 32 + lane < rend) rc1 = recs[rb + 32 + lane];
  if (rb + 64 + lane < rend) rc2 = recs[rb + 64 + lane];
  for (int g0 = 0; g0 < nrows; g0 += RS) {
#pragma unroll
    for (int gp = 0; gp < NP; ++gp) {
      const int gb = g0 + gp * kD;
      if (gb < nrows) {
        put_pair((gp + NPR - 1) % RH);
        fetch_pair(gb + 2 * NPR);
        if (gb > 0 && (gb & 63) == 0) pend = pair_ends(off, item, gb >> 6, lane);
        const int re = __shfl_sync(0xffffffffu, pend, (gb & 63) >> 1);
        while (cstart < re) {
          const int ce = min(re, wbase + 32);
          const int xrel = rec_xrel(rc0.rx);
          if (staged != wbase) {
            // every record of the window is staged once, by its own lane, whatever row pair
            // it belongs to: row pairs start at even rows, so its Cv' shift is row & 1
            __syncwarp();  // the previous window's staging and partial sums have been read
            const bool valid = wbase + lane < rend;
            if (valid) {
              int ou, ov;
              R fu, fv;
              record_coords<R, EXT>(a, rc0, ou, fu, ov, fv);
              stage_degrid<W, R, EXT>(tab, Wp, a.interp, ou, fu, ov, fv, rec_row(rc0.rx) & 1, xrel, s_cv, s_u,
                                      lane);
            }
            MW = transpose32(valid ? cover_lanes<W, KC>(xrel) : 0u, lane);
            staged = wbase;
            __syncwarp();
          }
          const bool mine = lane >= cstart - wbase && lane < ce - wbase;
          unsigned M = MW & record_range(cstart - wbase, ce - wbase);
          while (M) {
            const int l1 = __ffs(M) - 1;
            M &= M - 1u;
            const bool two = M != 0u;
            const int l2 = two ? __ffs(M) - 1 : 32;  // record 32 is zero
            M &= M - 1u;
            P c1[NPR], c2[NPR];
            load_cv_pairs<W, R>(s_cv, l1, c1);
            load_cv_pairs<W, R>(s_cv, l2, c2);
            R u1[KC], u2[KC];
            {
              const unsigned char* p1 = s_u + l1 * L::UP + myslot * L::SU;
              const unsigned char* p2 = s_u + l2 * L::UP + myslot * L::SU;
              if constexpr (sizeof(R) == 4 && KC == 2) {
                const float2 x1 = *reinterpret_cast<const float2*>(p1), x2 = *reinterpret_cast<const float2*>(p2);
                u1[0] = x1.x;
                u1[1] = x1.y;
                u2[0] = x2.x;
                u2[1] = x2.y;
              } else {
                u1[0] = *reinterpret_cast<const R*>(p1);
                u2[0] = *reinterpret_cast<const R*>(p2);
              }
            }
            R p1r = R(0), p1i = R(0), p2r = R(0), p2i = R(0);
#pragma unroll
            for (int j = 0; j < KC; ++j) {
              P s1r = pzero<P>(), s1i = pzero<P>(), s2r = pzero<P>(), s2i = pzero<P>();
#pragma unroll
              for (int m = 0; m < NPR; ++m) {
                const int h = (gp + m) % RH;
                s1r = pfma(c1[m], gR[j][h], s1r);
                s1i = pfma(c1[m], gI[j][h], s1i);
                s2r = pfma(c2[m], gR[j][h], s2r);
                s2i = pfma(c2[m], gI[j][h], s2i);
              }
              p1r = fma(u1[j], psum(s1r), p1r);
              p1i = fma(u1[j], psum(s1i), p1i);
              p2r = fma(u2[j], psum(s2r), p2r);
              p2i = fma(u2[j], psum(s2i), p2i);
            }
            C2 o1, o2;
            o1.x = p1r;
            o1.y = p1i;
            o2.x = p2r;
            o2.y = p2i;
            *reinterpret_cast<C2*>(s_p + l1 * L::PP + myslot * L::SP) = o1;
            if (two) *reinterpret_cast<C2*>(s_p + l2 * L::PP + myslot * L::SP) = o2;
          }
          __syncwarp();
          if (mine) {
            // the record's lane adds the partial sums of the lanes its support covers
            const int L0 = xrel >> (KC - 1), L1 = (xrel + W - 1) >> (KC - 1);
            R vr = R(0), vi = R(0);
#pragma unroll
            for (int m = 0; m < L::NL; ++m) {
              const int Ln = L0 + m;
              if (Ln >= 0 && Ln <= 31 && Ln <= L1) {
                const C2 p = *reinterpret_cast<const C2*>(s_p + lane * L::PP + (Ln & (L::PS - 1)) * L::SP);
                vr += p.x;
                vi += p.y;
              }
            }
            C2 o;
            o.x = vr;
            o.y = vi;
            // both records of a visibility crossing a strip add into the zeroed output
            // (two terms onto zero: the sum does not depend on their order)
            red_add(out + rc0.idx, o);
          }
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
  unsigned char* my = smem + tab_bytes + warp * Lay<W, R>::grid_bytes;
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
  unsigned char* my = smem + tab_bytes + warp * Lay<W, R>::degrid_bytes;
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
template <int W> size_t stage_bytes_w(int dtype, bool degrid) {
  if (dtype) return degrid ? Lay<W, double>::degrid_bytes : Lay<W, double>::grid_bytes;
  return degrid ? Lay<W, float>::degrid_bytes : Lay<W, float>::grid_bytes;
}
inline size_t stage_bytes(int W, int dtype, bool degrid) {
  switch (W) {
    case 1: return stage_bytes_w<1>(dtype, degrid);
    case 2: return stage_bytes_w<2>(dtype, degrid);
    case 3: return stage_bytes_w<3>(dtype, degrid);
    case 4: return stage_bytes_w<4>(dtype, degrid);
    case 5: return stage_bytes_w<5>(dtype, degrid);
    case 6: return stage_bytes_w<6>(dtype, degrid);
    case 7: return stage_bytes_w<7>(dtype, degrid);
    case 8: return stage_bytes_w<8>(dtype, degrid);
    case 9: return stage_bytes_w<9>(dtype, degrid);
    case 10: return stage_bytes_w<10>(dtype, degrid);
    case 11: return stage_bytes_w<11>(dtype, degrid);
    case 12: return stage_bytes_w<12>(dtype, degrid);
    case 13: return stage_bytes_w<13>(dtype, degrid);
    case 14: return stage_bytes_w<14>(dtype, degrid);
    case 15: return stage_bytes_w<15>(dtype, degrid);
    case 16: return stage_bytes_w<16>(dtype, degrid);
    default: return 0;
  }
}

}  // namespace
}  // namespace lmg

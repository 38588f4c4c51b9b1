// Device-side types and helpers shared by the binning, gridding and degridding kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lmg {

constexpr int kFracBits = 32;

// Support start (grid indices, wrapped to [0, N)) and fixed-point table coordinate of
// one visibility; x0 < 0 marks a dropped position.
struct VisPos {
  int x0, y0;
  unsigned su, sv;
};

// One binned record: a visibility as seen from one strip (strip_width columns). rx packs
// the support-start row (bits 8..31) and xrel (bits 0..7, signed), the support start
// column relative to the strip's first column (negative when the support started in the
// previous strip, i.e. for the strip's secondary copy).
struct alignas(16) Rec {  // one 16-byte load or store
  unsigned idx;
  int rx;
  unsigned su, sv;
};
__host__ __device__ __forceinline__ int rec_pack(int row, int xrel) { return (row << 8) | (xrel & 0xff); }
__host__ __device__ __forceinline__ int rec_xrel(int rx) { return static_cast<int>(static_cast<signed char>(rx & 0xff)); }
__host__ __device__ __forceinline__ int rec_row(int rx) { return static_cast<int>(static_cast<unsigned>(rx) >> 8); }

// Work item: rows [r0, r1) of one strip holding nrec records.
struct Item {
  int strip, r0, r1, nrec;
};

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

// Fixed point of the float64 product u * scale2, with scale2 = N * pixel_scale * 2^32:
// U = round-half-even(fl64(u * scale2)) computed exactly with integer operations.
// Returns false when the product is not finite or |U| >= 2^62 (|u_cells| >= 2^30).
__device__ __forceinline__ bool fixed_position(double u, double scale2, long long& U) {
  const double p = __dmul_rn(u, scale2);
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(p));
  const int e = int((bits >> 52) & 0x7ff);
  if (e >= 1023 + 62) return false;  // too large, infinite or NaN
  const bool neg = (bits >> 63) != 0;
  unsigned long long q;
  if (e == 0) {
    q = 0;  // zero or subnormal: rounds to 0
  } else {
    const unsigned long long m = (bits & 0xfffffffffffffull) | (1ull << 52);
    const int sh = e - 1075;
    if (sh >= 0) {
      q = m << sh;
    } else {
      const int k = -sh;
      if (k > 54) {
        q = 0;
      } else {
        q = m >> k;
        const unsigned long long rem = m & ((1ull << k) - 1ull);
        const unsigned long long half = 1ull << (k - 1);
        if (rem > half || (rem == half && (q & 1ull))) ++q;
      }
    }
  }
  U = neg ? -static_cast<long long>(q) : static_cast<long long>(q);
  return true;
}

// Residual u_q - u (cells) of the quantisation U = round(u scale2), scale2 = N pixel_scale
// 2^32: (U - fl(u scale2)) 2^-32, exact (U and the product differ by at most 1/2, and U
// converts to double exactly wherever the product has a fraction).
__device__ __forceinline__ double quantisation_residual(double u, double scale2, long long U) {
  const double p = __dmul_rn(u, scale2);
  return __dmul_rn(__dsub_rn(static_cast<double>(U), p), 2.3283064365386962890625e-10);
}

// Support rule (Eq. 6): n_start = ceil(u - W/2) and S = (n_start - (u - W/2)) 2^32.
__device__ __forceinline__ void support_start(long long U, int W, long long& n_start, unsigned& S) {
  const long long Y = U - (W & 1) * (1ll << (kFracBits - 1));
  const long long c = -((-Y) >> kFracBits);
  n_start = c - (W >> 1);
  S = static_cast<unsigned>((c << kFracBits) - Y);
}

// Lane t of the result holds bit l = bit t of lane l's input (32 x 32 bit transpose).
__device__ __forceinline__ unsigned transpose32(unsigned x, int lane) {
  const unsigned masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int j = 16 >> k;
    const unsigned m = masks[k];
    const unsigned y = __shfl_xor_sync(0xffffffffu, x, j);
    if (lane & j) x = (x & ~m) | ((y & ~m) >> j);
    else          x = (x & m) | ((y & m) << j);
  }
  return x;
}

// Packed single-precision pairs (re, im) in one 64-bit register: Blackwell's f32x2 FMA
// does a complex-by-real multiply-add in one instruction.
__device__ __forceinline__ unsigned long long f2pack(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 f2unpack(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
// a * b + c, elementwise on the two halves
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ void red_add(float2* p, float2 v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}
// two complex64 values (16 bytes, 16-byte aligned) in one vector reduction
__device__ __forceinline__ void red_add2(float2* p, float2 a, float2 b) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y)
               : "memory");
}
__device__ __forceinline__ void red_add(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

}  // namespace lmg

// Fused transforms of the kept field for complex64 plans with a 4096^2 grid: the imaging
// transform (Eq. 4) with its correction and crop (Eq. 15), and its adjoint, pad and
// correction followed by the transform of Eq. 2 -- each as two kernels over a scratch array
// of N x n values instead of the 1-D library transforms plus a separate correction pass.
//
// One 4096-point transform is run by 256 threads as three radix-16 passes
// (4096 = 16 x 16 x 16): with n = n0 + 16 n1 + 256 n2 and k = k0 + 16 k1 + 256 k2,
//   X[k] = sum_n0 e(n0 k2 / 16) [W^{16 n0 k1} W^{n0 k0}] sum_n1 e(n1 k1 / 16) W^{16 n1 k0}
//          sum_n2 e(n2 k0 / 16) x[n],          e(a) = exp(S 2 pi i a), W = e(1 / 4096),
// so thread t first takes the 16-point DFT over n2 of x[t + 256 n2], multiplies by
// W^{t k0} (t = n0 + 16 n1), then (through shared memory) the DFT over n1 for (n0, k0)
// and the factor W^{16 n0 k1}, then the DFT over n0 for (k0, k1): thread t ends with
// X[t + 256 k2]. The twiddles W^m come from a table of e(m / 4096) built on the host in
// float64 and rounded once: each CTA keeps its 64 entries W^b and 64 entries W^{64 a} in
// shared memory and forms W^{64 a + b} as one product (a load per lane from the whole
// table would touch a sector per lane: lanes t need W^{t k0}, k0 apart).
//
// Layouts: grids are [N][N] (row = v, index n + N/2); the scratch holds the kept columns
// q' (0 <= q' < n) of every row in blocks of kBW columns, element (row, q') at
// ((q' / kBW) N + row) kBW + q' % kBW, so that a block is one contiguous kBW x 4096 array
// (a column CTA reads or writes it whole) and a row's kept values are kBW x 8-byte pieces
// (the row kernels read and write them). A kept pixel offset q = p - n/2 is stored at
// q mod N.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace lmg {
namespace {

constexpr int kN = kXformN;        // 4096
constexpr int kT = 256;            // threads per transform
constexpr int kPitchA = 264;       // first exchange: 16 rows of 256 values (+8: the two
                                   // half-warps of a read fall on different banks)
constexpr int kPitchB = 17;        // second exchange: 256 rows of 16 values (+1)
constexpr int kBuf = 256 * kPitchB;  // elements of one transform's exchange buffer (>= 16 kPitchA)
static_assert(kBuf >= 16 * kPitchA, "exchange buffer");
constexpr int kBW = 4;             // columns per scratch block = transforms per column CTA
constexpr int kColThreads = kBW * kT;
constexpr int kColMinBlocks = kBW == 4 ? 1 : (kBW == 2 ? 2 : 3);  // resident CTAs per SM

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// 4-point DFT with exponent sign S, in place: (a, b, c, d) -> (X0, X1, X2, X3).
template <int S> __device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
  const float2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = csub(b, d);
  const float2 j3 = S > 0 ? make_float2(-s3.y, s3.x) : make_float2(s3.y, -s3.x);  // S i s3
  a = cadd(s0, s2);
  b = cadd(s1, j3);
  c = csub(s0, s2);
  d = csub(s1, j3);
}

// e(m / 16) for m = 0 .. 9 (cos and sin of m pi / 8), the internal twiddles of dft16.
__device__ __forceinline__ float2 e16(int m, int S) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, c2 = 0.70710678118654752f;
  float c = 1.f, s = 0.f;
  switch (m) {
    case 1: c = c1; s = s1; break;
    case 2: c = c2; s = c2; break;
    case 3: c = s1; s = c1; break;
    case 4: c = 0.f; s = 1.f; break;
    case 6: c = -c2; s = c2; break;
    case 9: c = -c1; s = -s1; break;
    default: break;
  }
  return make_float2(c, S > 0 ? s : -s);
}

// 16-point DFT with exponent sign S, in place in natural order (4 x 4: DFTs over n / 4 for
// each n mod 4, twiddles e(na kb / 16), DFTs over n mod 4).
template <int S> __device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
  for (int na = 0; na < 4; ++na) dft4<S>(v[na], v[na + 4], v[na + 8], v[na + 12]);  // z[na][kb] at v[na + 4 kb]
#pragma unroll
  for (int na = 1; na < 4; ++na)
#pragma unroll
    for (int kb = 1; kb < 4; ++kb) v[na + 4 * kb] = cmul(v[na + 4 * kb], e16(na * kb, S));
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) dft4<S>(v[4 * kb], v[4 * kb + 1], v[4 * kb + 2], v[4 * kb + 3]);
  // v[4 kb + ka] now holds y[kb + 4 ka]
  float2 y[16];
#pragma unroll
  for (int kb = 0; kb < 4; ++kb)
#pragma unroll
    for (int ka = 0; ka < 4; ++ka) y[kb + 4 * ka] = v[4 * kb + ka];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = y[k];
}

// stw: the CTA's shared copy, stw[b] = W^b and stw[64 + a] = W^{64 a} (a, b < 64).
template <int S> __device__ __forceinline__ float2 twiddle(const float2* stw, int m) {
  const float2 w = cmul(stw[64 + (m >> 6)], stw[m & 63]);
  return S > 0 ? w : make_float2(w.x, -w.y);
}

// v[k] *= W^{base k} for k = 1 .. 15 (base < 512). W^{base}, W^{2 base}, W^{4 base} and
// W^{8 base} come from the table, the others as products of at most four of them (by the
// bits of k): 8 shared loads instead of 30, at most three more roundings per factor.
template <int S> __device__ __forceinline__ void apply_twiddles(float2 (&v)[16], const float2* stw, int base) {
  const float2 w1 = twiddle<S>(stw, base), w2 = twiddle<S>(stw, 2 * base), w4 = twiddle<S>(stw, 4 * base),
               w8 = twiddle<S>(stw, 8 * base);
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    float2 w = (k & 1) ? w1 : ((k & 2) ? w2 : ((k & 4) ? w4 : w8));
    if ((k & 1) && (k & 2)) w = cmul(w, w2);
    if ((k & 3) && (k & 4)) w = cmul(w, w4);
    if ((k & 7) && (k & 8)) w = cmul(w, w8);
    v[k] = cmul(v[k], w);
  }
}

__device__ __forceinline__ void load_twiddles(const float2* __restrict__ tw, float2* stw) {
  if (threadIdx.x < 128) stw[threadIdx.x] = __ldg(tw + (threadIdx.x < 64 ? threadIdx.x : 64 * (threadIdx.x - 64)));
}

// One 4096-point transform (sign S) by threads t = 0 .. 255 of a group whose shared buffer
// is buf (kBuf values); v[j] = x[t + 256 j] on entry, X[t + 256 k] in v[k] on exit; tw is
// the CTA's shared twiddle copy (load_twiddles, made visible by a sync before the call).
// sync() must synchronise at least the group; the buffer is free again after the next sync.
template <int S, typename Sync>
__device__ __forceinline__ void fft4096(float2 (&v)[16], float2* buf, const float2* tw, int t, Sync sync) {
  dft16<S>(v);
  apply_twiddles<S>(v, tw, t);  // W^{t k0}
#pragma unroll
  for (int k0 = 0; k0 < 16; ++k0) buf[k0 * kPitchA + t] = v[k0];
  sync();
  const int n0 = t & 15, k0 = t >> 4;
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) v[n1] = buf[k0 * kPitchA + n0 + 16 * n1];
  dft16<S>(v);
  apply_twiddles<S>(v, tw, 16 * n0);  // W^{16 n0 k1}
  sync();
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) buf[(k0 + 16 * k1) * kPitchB + n0] = v[k1];
  sync();
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = buf[t * kPitchB + m];
  dft16<S>(v);
}

struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Kept output index k of a transform -> kept offset q' in [0, n), or -1.
__device__ __forceinline__ int kept_slot(int k, int half) {
  if (k < half) return k + half;
  if (k >= kN - half) return k - (kN - half);
  return -1;
}

__device__ __forceinline__ size_t scratch_index(int row, int q) {
  return (static_cast<size_t>(q / kBW) * kN + row) * kBW + q % kBW;
}

// Imaging, rows: every grid row transformed (+i), its kept columns to the scratch.
__global__ void __launch_bounds__(kT) k_image_rows(const float2* __restrict__ G, float2* __restrict__ T,
                                                   const float2* __restrict__ tw, int n) {
  __shared__ float2 buf[kBuf];
  __shared__ float2 stw[128];
  load_twiddles(tw, stw);
  const int row = blockIdx.x, t = threadIdx.x, half = n / 2;
  const float2* src = G + static_cast<size_t>(row) * kN;
  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __ldcs(src + t + 256 * j);
  __syncthreads();
  fft4096<1>(v, buf, stw, t, BlockSync{});
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const int q = kept_slot(t + 256 * k2, half);
    if (q >= 0) T[scratch_index(row, q)] = v[k2];
  }
}

// Imaging, columns: kBW kept columns per CTA (256 threads each) transformed (+i), their
// kept rows corrected (h(x) h(y) and the centring sign (-1)^(qx + qy)) into the image.
__global__ void __launch_bounds__(kColThreads, kColMinBlocks)
    k_image_cols(const float2* __restrict__ T, float2* __restrict__ img, const float* __restrict__ h,
                 const float2* __restrict__ tw, int n) {
  extern __shared__ __align__(16) float2 sm[];
  __shared__ float2 stw[128];
  load_twiddles(tw, stw);
  const int b = blockIdx.x, g = threadIdx.x >> 8, t = threadIdx.x & (kT - 1), half = n / 2;
  float2* buf = sm + g * kBuf;
  // the block (4096 rows x kBW columns, contiguous) into kBW column buffers, two values per load
  const float4* blk = reinterpret_cast<const float4*>(T + static_cast<size_t>(b) * kN * kBW);
  for (int c = threadIdx.x; c < kN * kBW / 2; c += kColThreads) {
    const float4 x = __ldcs(blk + c);
    const int e = 2 * c;
    sm[(e % kBW) * kBuf + e / kBW] = make_float2(x.x, x.y);
    sm[((e + 1) % kBW) * kBuf + (e + 1) / kBW] = make_float2(x.z, x.w);
  }
  __syncthreads();
  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = buf[t + 256 * j];
  __syncthreads();
  fft4096<1>(v, buf, stw, t, BlockSync{});
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const int r = kept_slot(t + 256 * k2, half);
    if (r >= 0) buf[r] = v[k2];
  }
  __syncthreads();
  // kept rows r of the columns kBW b .. kBW b + kBW - 1: one kBW x 8-byte piece per row
  const int q0 = kBW * b;
  for (int r = threadIdx.x; r < n; r += kColThreads) {
    const int qy = r - half;
    const float hy = h[r];
    float2 o[kBW];
#pragma unroll
    for (int c = 0; c < kBW; ++c) {
      const int qx = q0 + c - half;
      float f = h[q0 + c] * hy;
      if ((qx + qy) & 1) f = -f;
      const float2 x = sm[c * kBuf + r];
      o[c] = make_float2(f * x.x, f * x.y);
    }
    float2* dst = img + static_cast<size_t>(r) * n + q0;
    if constexpr (kBW == 1) {
      dst[0] = o[0];
    } else {
#pragma unroll
      for (int c = 0; c < kBW; c += 2)
        *reinterpret_cast<float4*>(dst + c) = make_float4(o[c].x, o[c].y, o[c + 1].x, o[c + 1].y);
    }
  }
}

// Prediction, columns: kBW image columns per CTA corrected, placed at their kept rows of
// a zero column of 4096 and transformed (-i) into the scratch (all 4096 rows).
__global__ void __launch_bounds__(kColThreads, kColMinBlocks)
    k_model_cols(const float2* __restrict__ img, float2* __restrict__ T, const float* __restrict__ h,
                 const float2* __restrict__ tw, int n) {
  extern __shared__ __align__(16) float2 sm[];
  __shared__ float2 stw[128];
  load_twiddles(tw, stw);
  const int b = blockIdx.x, g = threadIdx.x >> 8, t = threadIdx.x & (kT - 1), half = n / 2;
  float2* buf = sm + g * kBuf;
  const int q0 = kBW * b;
  for (int i = threadIdx.x; i < kBW * kN; i += kColThreads) sm[(i >> 12) * kBuf + (i & (kN - 1))] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += kColThreads) {
    const int qy = r - half, iy = qy < 0 ? qy + kN : qy;
    const float hy = h[r];
    const float2* src = img + static_cast<size_t>(r) * n + q0;
    float2 x[kBW];
    if constexpr (kBW == 1) {
      x[0] = src[0];
    } else {
#pragma unroll
      for (int c = 0; c < kBW; c += 2) {
        const float4 a = *reinterpret_cast<const float4*>(src + c);
        x[c] = make_float2(a.x, a.y);
        x[c + 1] = make_float2(a.z, a.w);
      }
    }
#pragma unroll
    for (int c = 0; c < kBW; ++c) {
      const int qx = q0 + c - half;
      float f = h[q0 + c] * hy;
      if ((qx + qy) & 1) f = -f;
      sm[c * kBuf + iy] = make_float2(f * x[c].x, f * x[c].y);
    }
  }
  __syncthreads();
  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = buf[t + 256 * j];
  __syncthreads();
  fft4096<-1>(v, buf, stw, t, BlockSync{});
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) buf[t + 256 * k2] = v[k2];
  __syncthreads();
  // the block, contiguous, two values per store
  float4* blk = reinterpret_cast<float4*>(T + static_cast<size_t>(b) * kN * kBW);
  for (int c = threadIdx.x; c < kN * kBW / 2; c += kColThreads) {
    const int e = 2 * c;
    const float2 x0 = sm[(e % kBW) * kBuf + e / kBW], x1 = sm[((e + 1) % kBW) * kBuf + (e + 1) / kBW];
    blk[c] = make_float4(x0.x, x0.y, x1.x, x1.y);
  }
}

// Prediction, rows: each row's kept columns from the scratch (zero elsewhere) transformed
// (-i) into the grid row.
__global__ void __launch_bounds__(kT) k_model_rows(const float2* __restrict__ T, float2* __restrict__ G,
                                                   const float2* __restrict__ tw, int n) {
  __shared__ float2 buf[kBuf];
  __shared__ float2 stw[128];
  load_twiddles(tw, stw);
  const int row = blockIdx.x, t = threadIdx.x, half = n / 2;
  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int q = kept_slot(t + 256 * j, half);
    v[j] = q >= 0 ? __ldcs(T + scratch_index(row, q)) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft4096<-1>(v, buf, stw, t, BlockSync{});
  float2* dst = G + static_cast<size_t>(row) * kN;
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) dst[t + 256 * k2] = v[k2];
}

constexpr size_t kColSmem = size_t(kBW) * kBuf * sizeof(float2);

}  // namespace

bool xform_supported(int dtype, long long N, long long n) {
  return dtype == 0 && N == kN && n >= 8 && n <= kN && n % 8 == 0;
}

size_t xform_scratch_bytes(long long n) { return static_cast<size_t>(kN) * static_cast<size_t>(n) * sizeof(float2); }

int xform_set_limits() {
  if (cudaFuncSetAttribute(k_image_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kColSmem)) != cudaSuccess ||
      cudaFuncSetAttribute(k_model_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kColSmem)) != cudaSuccess)
    return -1;
  return 0;
}

int xform_image_launch(const void* grid, void* image, void* scratch, const float* h, const void* tw, int n,
                       cudaStream_t st) {
  const float2* w = static_cast<const float2*>(tw);
  k_image_rows<<<kN, kT, 0, st>>>(static_cast<const float2*>(grid), static_cast<float2*>(scratch), w, n);
  k_image_cols<<<n / kBW, kColThreads, kColSmem, st>>>(static_cast<const float2*>(scratch), static_cast<float2*>(image), h, w,
                                               n);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int xform_model_launch(const void* image, void* grid, void* scratch, const float* h, const void* tw, int n,
                       cudaStream_t st) {
  const float2* w = static_cast<const float2*>(tw);
  k_model_cols<<<n / kBW, kColThreads, kColSmem, st>>>(static_cast<const float2*>(image), static_cast<float2*>(scratch), h, w,
                                               n);
  k_model_rows<<<kN, kT, 0, st>>>(static_cast<const float2*>(scratch), static_cast<float2*>(grid), w, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lmg

// Grid correction with crop (Eqs. 4, 15) and its adjoint, pad with correction.
//
// The grids are held in index order i = n + N/2. An unnormalised FFT of that array gives
// sum_i G[i] e^{+i 2 pi i q / N} = (-1)^q sum_n G_n e^{+i 2 pi n q / N}, so the centring
// shift is the checkerboard (-1)^(qx + qy) applied here, with q = p - n_image/2 the pixel
// offset from the image centre (stored at q mod N).
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "kernels.h"

namespace lmg {
namespace {

template <typename R>
__global__ void k_crop_correct(const typename Cplx<R>::T* __restrict__ F, typename Cplx<R>::T* __restrict__ img,
                               const R* __restrict__ h, int n_img, int N) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y;
  if (px >= n_img) return;
  const int qx = px - n_img / 2, qy = py - n_img / 2;
  const int sx = qx < 0 ? qx + N : qx, sy = qy < 0 ? qy + N : qy;
  const auto v = F[static_cast<size_t>(sy) * N + sx];
  R f = h[px] * h[py];
  if ((qx + qy) & 1) f = -f;
  typename Cplx<R>::T o;
  o.x = f * v.x;
  o.y = f * v.y;
  img[static_cast<size_t>(py) * n_img + px] = o;
}

template <typename R>
__global__ void k_pad_correct(const typename Cplx<R>::T* __restrict__ img, typename Cplx<R>::T* __restrict__ P,
                              const R* __restrict__ h, int n_img, int N) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  const int iy = blockIdx.y;
  if (ix >= N) return;
  const int qx = ix < N / 2 ? ix : ix - N, qy = iy < N / 2 ? iy : iy - N;
  typename Cplx<R>::T o;
  o.x = 0;
  o.y = 0;
  const int half = n_img / 2;
  if (qx >= -half && qx < n_img - half && qy >= -half && qy < n_img - half) {
    const int px = qx + half, py = qy + half;
    const auto v = img[static_cast<size_t>(py) * n_img + px];
    R f = h[px] * h[py];
    if ((qx + qy) & 1) f = -f;
    o.x = f * v.x;
    o.y = f * v.y;
  }
  P[static_cast<size_t>(iy) * N + ix] = o;
}

// The kept rows only of the padded, corrected model grid (row py of the image at grid row
// qy mod N, every column of it); the other rows are left as they are (zero in the plan's
// model buffer, which nothing else writes).
template <typename R>
__global__ void k_pad_rows(const typename Cplx<R>::T* __restrict__ img, typename Cplx<R>::T* __restrict__ P,
                           const R* __restrict__ h, int n_img, int N) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y;
  if (ix >= N) return;
  const int half = n_img / 2;
  const int qy = py - half, iy = qy < 0 ? qy + N : qy;
  const int qx = ix < N / 2 ? ix : ix - N;
  typename Cplx<R>::T o;
  o.x = 0;
  o.y = 0;
  if (qx >= -half && qx < n_img - half) {
    const int px = qx + half;
    const auto v = img[static_cast<size_t>(py) * n_img + px];
    R f = h[px] * h[py];
    if ((qx + qy) & 1) f = -f;
    o.x = f * v.x;
    o.y = f * v.y;
  }
  P[static_cast<size_t>(iy) * N + ix] = o;
}

// complex64 with two pixels per thread: with n_img / 2 and N / 2 even, a pixel pair
// (px, px + 1) from an even px never straddles the wrap of the grid index nor the edge of
// the kept field, so both of its loads and stores are 16-byte vectors. The pair's signs
// (-1)^(qx + qy) alternate; the factors are the scalar kernels' products, bit for bit.
__global__ void k_crop_correct_v2(const float4* __restrict__ F, float4* __restrict__ img, const float* __restrict__ h,
                                  int n_img, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y, px = 2 * t;
  if (px >= n_img) return;
  const int qx = px - n_img / 2, qy = py - n_img / 2;
  const int sx = qx < 0 ? qx + N : qx, sy = qy < 0 ? qy + N : qy;
  const float4 v = F[(static_cast<size_t>(sy) * N + sx) >> 1];
  const float2 hx = reinterpret_cast<const float2*>(h)[t];
  const float hy = ((qx + qy) & 1) ? -h[py] : h[py];
  const float f0 = hx.x * hy, f1 = -(hx.y * hy);
  img[(static_cast<size_t>(py) * n_img + px) >> 1] = make_float4(f0 * v.x, f0 * v.y, f1 * v.z, f1 * v.w);
}

// Pad + correct of one grid row iy (image row py, or zeros when py < 0), two columns per
// thread as in k_crop_correct_v2.
__device__ __forceinline__ void pad_pair_v2(const float4* __restrict__ img, float4* __restrict__ P,
                                            const float* __restrict__ h, int n_img, int N, int iy, int py, int qy,
                                            int t) {
  const int ix = 2 * t;
  const int half = n_img / 2;
  const int qx = ix < N / 2 ? ix : ix - N;
  float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
  if (py >= 0 && qx >= -half && qx < n_img - half) {
    const int px = qx + half;
    const float4 v = img[(static_cast<size_t>(py) * n_img + px) >> 1];
    const float2 hx = reinterpret_cast<const float2*>(h)[px >> 1];
    const float hy = ((qx + qy) & 1) ? -h[py] : h[py];
    const float f0 = hx.x * hy, f1 = -(hx.y * hy);
    o = make_float4(f0 * v.x, f0 * v.y, f1 * v.z, f1 * v.w);
  }
  P[(static_cast<size_t>(iy) * N + ix) >> 1] = o;
}

__global__ void k_pad_correct_v2(const float4* __restrict__ img, float4* __restrict__ P, const float* __restrict__ h,
                                 int n_img, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * t >= N) return;
  const int iy = blockIdx.y, half = n_img / 2;
  const int qy = iy < N / 2 ? iy : iy - N;
  const int py = (qy >= -half && qy < n_img - half) ? qy + half : -1;
  pad_pair_v2(img, P, h, n_img, N, iy, py, qy, t);
}

__global__ void k_pad_rows_v2(const float4* __restrict__ img, float4* __restrict__ P, const float* __restrict__ h,
                              int n_img, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * t >= N) return;
  const int py = blockIdx.y, qy = py - n_img / 2;
  pad_pair_v2(img, P, h, n_img, N, qy < 0 ? qy + N : qy, py, qy, t);
}

// The two-pixel kernels apply: complex64, n_img and N multiples of 4, 16-byte aligned
// arrays (h 8-byte aligned).
bool pairs_ok(const void* a, const void* b, const void* h, int n_img, int N, int dtype) {
  return dtype == 0 && n_img % 4 == 0 && N % 4 == 0 && reinterpret_cast<uintptr_t>(a) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(b) % 16 == 0 && reinterpret_cast<uintptr_t>(h) % 8 == 0;
}

}  // namespace

int pad_rows_launch(const void* img, void* P, const void* h, int n_img, int N, int dtype, cudaStream_t st) {
  dim3 block(256), grid((N + 255) / 256, n_img);
  if (pairs_ok(img, P, h, n_img, N, dtype))
    k_pad_rows_v2<<<dim3((N / 2 + 255) / 256, n_img), block, 0, st>>>(
        static_cast<const float4*>(img), static_cast<float4*>(P), static_cast<const float*>(h), n_img, N);
  else if (dtype)
    k_pad_rows<double><<<grid, block, 0, st>>>(static_cast<const double2*>(img), static_cast<double2*>(P),
                                               static_cast<const double*>(h), n_img, N);
  else
    k_pad_rows<float><<<grid, block, 0, st>>>(static_cast<const float2*>(img), static_cast<float2*>(P),
                                              static_cast<const float*>(h), n_img, N);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int crop_correct_launch(const void* F, void* img, const void* h, int n_img, int N, int dtype, cudaStream_t st) {
  dim3 block(256), grid((n_img + 255) / 256, n_img);
  if (pairs_ok(F, img, h, n_img, N, dtype))
    k_crop_correct_v2<<<dim3((n_img / 2 + 255) / 256, n_img), block, 0, st>>>(
        static_cast<const float4*>(F), static_cast<float4*>(img), static_cast<const float*>(h), n_img, N);
  else if (dtype)
    k_crop_correct<double><<<grid, block, 0, st>>>(static_cast<const double2*>(F), static_cast<double2*>(img),
                                                   static_cast<const double*>(h), n_img, N);
  else
    k_crop_correct<float><<<grid, block, 0, st>>>(static_cast<const float2*>(F), static_cast<float2*>(img),
                                                  static_cast<const float*>(h), n_img, N);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int pad_correct_launch(const void* img, void* P, const void* h, int n_img, int N, int dtype, cudaStream_t st) {
  dim3 block(256), grid((N + 255) / 256, N);
  if (pairs_ok(img, P, h, n_img, N, dtype))
    k_pad_correct_v2<<<dim3((N / 2 + 255) / 256, N), block, 0, st>>>(
        static_cast<const float4*>(img), static_cast<float4*>(P), static_cast<const float*>(h), n_img, N);
  else if (dtype)
    k_pad_correct<double><<<grid, block, 0, st>>>(static_cast<const double2*>(img), static_cast<double2*>(P),
                                                  static_cast<const double*>(h), n_img, N);
  else
    k_pad_correct<float><<<grid, block, 0, st>>>(static_cast<const float2*>(img), static_cast<float2*>(P),
                                                 static_cast<const float*>(h), n_img, N);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lmg

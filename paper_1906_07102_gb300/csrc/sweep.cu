// Single-plan gridding and degridding: the nearest / linear table kernels (the extended
// lookups are compiled in sweep_ext.cu), the spill pass, launch configuration.
#include "sweep_body.cuh"

namespace lmg {
namespace {

template <typename R>
__global__ void k_grid_spill(const Item* __restrict__ items, const int* __restrict__ counters, int item_cap,
                             int W, int RS, int N, const typename Cplx<R>::T* __restrict__ spill,
                             typename Cplx<R>::T* __restrict__ grid) {
  // one warp per item slot (the launch covers item_cap slots)
  int nfront;
  const int total = work_total(counters, item_cap, nfront);
  const int w = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  if (w < total)
    spill_item<R>(items, nfront, item_cap, W, RS, N, 32 * cols_per_lane<R>(), spill, grid, w, threadIdx.x & 31);
}

void* kernel_for(int W, int dtype, int accum, bool degrid, bool ext) {
  return ext ? sweep_kernel_ext(W, dtype, accum, degrid) : sweep_kernel_pick<false>(W, dtype, accum, degrid);
}

}  // namespace

int ring_slots(int W) { return kD * ((W + kD - 1 + kD - 1) / kD); }

size_t sweep_smem_bytes(int W, int dtype, int Ms, bool table_in_smem, bool degrid, int warps) {
  const size_t rs = dtype ? 8 : 4;
  const int Wp = table_stride(W, dtype);
  const size_t tab = table_in_smem ? align16(size_t(Ms + 1) * Wp * rs) : 0;
  return tab + size_t(warps) * stage_bytes(W, dtype, degrid);
}

int sweep_set_smem_limits(int W, int dtype, int accum, size_t smem_bytes, bool degrid, bool ext) {
  void* k = kernel_for(W, dtype, accum, degrid, ext);
  if (!k) return -1;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_bytes)) == cudaSuccess ? 0 : -1;
}

int sweep_occupancy(int W, int dtype, int accum, size_t smem_bytes, bool degrid, bool ext, int warps,
                    int* blocks_per_sm) {
  void* k = kernel_for(W, dtype, accum, degrid, ext);
  if (!k) return -1;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 32 * warps, smem_bytes) == cudaSuccess ? 0
                                                                                                                : -1;
}

int sweep_config(int W, int dtype, int Ms, bool degrid, size_t limit, bool* table_in_smem, int* warps) {
  const size_t rs = dtype ? 8 : 4;
  const int Wp = table_stride(W, dtype);
  *table_in_smem = align16(size_t(Ms + 1) * Wp * rs) <= 96 * 1024;
  for (int pass = 0; pass < 2; ++pass) {
    for (int w = kWarps; w >= 1; w >>= 1) {
      if (sweep_smem_bytes(W, dtype, Ms, *table_in_smem, degrid, w) <= limit) {
        *warps = w;
        return 0;
      }
    }
    *table_in_smem = false;
  }
  return -1;
}

int grid_launch(const SweepArgs& a, cudaStream_t st) {
  void* k = kernel_for(a.W, a.dtype, a.accum, false, a.interp >= 2);
  if (!k) return -1;
  const size_t smem = sweep_smem_bytes(a.W, a.dtype, a.Ms, a.table_in_smem != 0, false, a.warps);
  cudaMemsetAsync(a.counters + kCntGridWork, 0, sizeof(int), st);
  SweepArgs args = a;
  void* params[] = {&args};
  if (cudaLaunchKernel(k, dim3(a.grid_blocks), dim3(32 * a.warps), params, smem, st) != cudaSuccess) return -1;
  const int spill_blocks = (a.item_cap + 7) / 8;  // 8 warps of 256 threads, one per item slot
  if (a.dtype) {
    k_grid_spill<double><<<spill_blocks, 256, 0, st>>>(a.items, a.counters, a.item_cap, a.W, ring_slots(a.W), a.N,
                                                       static_cast<const double2*>(a.spill),
                                                       static_cast<double2*>(a.grid));
  } else {
    k_grid_spill<float><<<spill_blocks, 256, 0, st>>>(a.items, a.counters, a.item_cap, a.W, ring_slots(a.W), a.N,
                                                      static_cast<const float2*>(a.spill),
                                                      static_cast<float2*>(a.grid));
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int degrid_launch(const SweepArgs& a, cudaStream_t st, bool zero_out) {
  void* k = kernel_for(a.W, a.dtype, 0, true, a.interp >= 2);
  if (!k) return -1;
  const size_t smem = sweep_smem_bytes(a.W, a.dtype, a.Ms, a.table_in_smem != 0, true, a.warps);
  // outputs start at zero: each record adds its partial sum (dropped positions stay zero)
  if (zero_out && a.nvis > 0) cudaMemsetAsync(a.vis_out, 0, size_t(a.nvis) * (a.dtype ? 16 : 8), st);
  cudaMemsetAsync(a.counters + kCntDegridWork, 0, sizeof(int), st);
  SweepArgs args = a;
  void* params[] = {&args};
  if (cudaLaunchKernel(k, dim3(a.grid_blocks), dim3(32 * a.warps), params, smem, st) != cudaSuccess) return -1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lmg

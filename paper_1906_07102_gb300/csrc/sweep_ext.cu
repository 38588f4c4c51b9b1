// Sweep kernels of the extended table lookups (Lagrange interpolation of degree 2 and 3,
// direct calculation), compiled apart from the nearest / linear kernels (sweep.cu) so that
// their larger register needs do not spill the common path; same per-item code otherwise.
#include "sweep_body.cuh"

namespace lmg {

void* sweep_kernel_ext(int W, int dtype, int accum, bool degrid) {
  return sweep_kernel_pick<true>(W, dtype, accum, degrid);
}

}  // namespace lmg

// fdlbm_step_wrap_f64.cu -- FP64 instantiation of the fused step for grids whose whole y-periodic
// height fits in one tile (templates in fdlbm_kernels.cuh). A translation unit of its own, so that
// it compiles in parallel with fdlbm_step_f64.cu.
#include "fdlbm_kernels.cuh"

namespace fdlbm {

cudaError_t launch_step_wrap_f64(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c,
                               unsigned* health, cudaStream_t s) {
  return launch_step_wrap_v<double>(variant, f, fn, g, c, health, s);
}

}  // namespace fdlbm

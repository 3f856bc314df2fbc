// fdlbm_step_f32dw.cu -- FDLBM_FP32_STORE_DW instantiation of the fused and split steps: FP32 storage
// with the per-ring equilibrium constants and pairs in double-word FP32 (templates in
// fdlbm_kernels.cuh). A translation unit of its own, compiled in parallel with the others.
#include "fdlbm_kernels.cuh"

namespace fdlbm {

cudaError_t launch_step_f32dw(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                              cudaStream_t s) {
  return launch_step_v<float, true>(variant, f, fn, g, c, health, s);
}

}  // namespace fdlbm

// fdlbm_step_f64.cu -- FP64-storage instantiation of the fused step (templates in fdlbm_kernels.cuh).
#include "fdlbm_kernels.cuh"

namespace fdlbm {

cudaError_t launch_step_f64(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                          cudaStream_t s) {
  return launch_step_v<double>(variant, f, fn, g, c, health, s);
}

cudaError_t launch_batch_f64(int variant, const BatchMember* mem, int nmem, long long tiles, unsigned long long step,
                             const Coeffs& c, cudaStream_t s) {
  return launch_batch_v<double>(variant, mem, nmem, tiles, step, c, s);
}

}  // namespace fdlbm

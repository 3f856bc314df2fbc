// fdlbm_noalloc.cu -- fdlbm_step_noalloc: the fused step for callers that cannot allocate device
// memory. The only scratch the step needs (its health word, here one word per step) lives in a
// file-scope __device__ array that every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/fdlbm.h"
#include "fdlbm_internal.h"

namespace {

// Scratch: one health word per step of a call (FDLBM_NOALLOC_MAX_STEPS * 4 bytes = 16 KiB).
static __device__ __align__(256) unsigned g_noalloc_health[FDLBM_NOALLOC_MAX_STEPS];

// In host code g_noalloc_health is only a host-side stand-in for the device symbol: its device
// address is looked up once per device (with that device current) and cached here.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned* g_scratch[kMaxDevices] = {nullptr};

int fail(int code, const std::string& msg) {
  fdlbm::set_thread_error(msg.c_str());
  return code;
}

}  // namespace

extern "C" int fdlbm_step_noalloc(const fdlbm_config* cfg, void* f_a, void* f_b, long nsteps, long* first_bad_step,
                                  void* cuda_stream) {
  using namespace fdlbm;
  if (first_bad_step) *first_bad_step = -1;
  std::string why;
  if (!valid_cfg(cfg, &why)) return fail(FDLBM_E_ARG, why);
  if (cfg->prec == FDLBM_FP64_STRICT)
    return fail(FDLBM_E_ARG, "FDLBM_FP64_STRICT steps through a handle's moment buffer: use fdlbm_step");
  if (!f_a || !f_b) return fail(FDLBM_E_ARG, "f_a and f_b must be device buffers");
  if ((reinterpret_cast<uintptr_t>(f_a) & 255) || (reinterpret_cast<uintptr_t>(f_b) & 255))
    return fail(FDLBM_E_ARG, "f_a and f_b must be 256-byte aligned");
  if (nsteps < 0 || nsteps > FDLBM_NOALLOC_MAX_STEPS)
    return fail(FDLBM_E_ARG, "nsteps must be in [0, FDLBM_NOALLOC_MAX_STEPS] = [0, 4096]: the static scratch holds "
                             "one health word per step");
  if (nsteps == 0) return FDLBM_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(FDLBM_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(FDLBM_E_ARG, "device index beyond 63");
  unsigned* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_health);
      if (e != cudaSuccess)
        return fail(FDLBM_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch[dev] = static_cast<unsigned*>(p);
    }
    scratch = g_scratch[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const Layout L = layout_of(cfg);
  const Coeffs c = make_coeffs(cfg);
  const int variant = default_variant(cfg);
  // the words of this call start at zero; the array keeps the previous call's contents otherwise
  e = cudaMemsetAsync(scratch, 0, sizeof(unsigned) * (size_t)nsteps, s);
  for (long k = 0; k < nsteps && e == cudaSuccess; ++k) {
    const void* in = (k % 2 == 0) ? f_a : f_b;
    void* out = (k % 2 == 0) ? f_b : f_a;
    e = launch_step(cfg->prec, variant, in, out, L.g, c, scratch + k, s);
  }
  unsigned words[FDLBM_NOALLOC_MAX_STEPS];
  if (e == cudaSuccess) e = cudaMemcpyAsync(words, scratch, sizeof(unsigned) * (size_t)nsteps, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(FDLBM_E_CUDA, std::string("fdlbm_step_noalloc: ") + cudaGetErrorString(e));
  for (long k = 0; k < nsteps; ++k) {
    if (words[k] & H_NUMERIC) {
      if (first_bad_step) *first_bad_step = k;
      return fail(FDLBM_E_NUMERIC, "a node had non-finite moments, n <= 0 or T <= 0 at the input of the step "
                                   "reported in first_bad_step");
    }
  }
  return FDLBM_OK;
}

// fdlbm_step_persist.cu -- persistent steps: one cooperative launch advances a solve by many time
// steps (variants V_PRP8x4 and V_PT32x16).
//
// Small grids are bound by latency, not by throughput: a 400 x 4 tube's step is a few microseconds
// of arithmetic, and every launch adds its start-up and drain. Here all CTAs stay resident (a
// cooperative launch guarantees it), each loops over the tiles of its share of the grid with the
// same tile body as the one-step kernels (the ring-parallel 8 x 4 tile, or the 32 x 16 tile), and
// the CTAs meet at a grid barrier between time steps, ping-ponging the two buffers. Each node's
// arithmetic is that of the one-step variants, so the results are bitwise theirs. A step reads what
// other CTAs wrote in the step before, so f is read with loads cached in L2 only (ldc<true>), never
// through L1, which keeps lines of a buffer from two steps back.
//
// The barrier counts arrivals in an atomic word and releases the CTAs by advancing a generation
// word; its wait polls at most kBarrierIters times. A CTA that gives up records FDLBM_HEALTH_TIMEOUT
// and leaves the kernel; the others then give up at their next barrier, so the launch always ends.
#include <cuda_runtime.h>

#include "fdlbm_kernels.cuh"

namespace fdlbm {

namespace {

constexpr int kBarrierIters = 1 << 22;  // with a 64 ns pause each: about a quarter of a second at least

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier over nblocks co-resident CTAs. bar[0] counts arrivals, bar[1] is the generation,
// gen the generation this CTA last saw (updated). Returns false if the wait gave up.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned& gen, int limit) {
  __shared__ int s_ok;
  __syncthreads();  // the CTA's stores of this step are issued
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();  // ... and visible to every CTA before the arrival
    const unsigned target = gen + 1u;
    if (atomicAdd(&bar[0], 1u) == nblocks - 1u) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    }
    int ok = 0;
    for (int i = 0; i < limit; ++i) {
      if (ld_acquire(&bar[1]) == target) {
        ok = 1;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    gen = target;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ unsigned read_gen(const unsigned* bar) {
  __shared__ unsigned s_gen;
  if (threadIdx.x == 0 && threadIdx.y == 0) s_gen = ld_acquire(&bar[1]);
  __syncthreads();
  return s_gen;
}

// nsteps steps, f0 -> f1 -> f0 ...; the result is in f1 after an odd count, in f0 after an even one.
template <typename S, int TW, int TH>
__global__ void __launch_bounds__(4 * TW * TH) k_persist_rp(S* f0, S* f1, Grid g, Coeffs c,
                                                            unsigned* __restrict__ health, unsigned* bar, int nsteps) {
  const int tiles_x = (g.nx + TW - 1) / TW, tiles = tiles_x * ((g.ny + TH - 1) / TH);
  unsigned gen = read_gen(bar);
  for (int s = 0; s < nsteps; ++s) {
    const S* in = (s & 1) ? f1 : f0;
    S* out = (s & 1) ? f0 : f1;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      rp_tile<S, TW, TH, true>(in, out, g, c, health, t % tiles_x, t / tiles_x);
      __syncthreads();  // the tile's shared memory is reused by the next one
    }
    if (s + 1 < nsteps && !grid_barrier(bar, gridDim.x, gen, kBarrierIters)) {
      if (threadIdx.x == 0) atomicOr(health, H_TIMEOUT);
      return;
    }
  }
}

template <typename S, int BX, int BY, int RY, int MINB, bool WRAPY>
__global__ void __launch_bounds__(BX * BY, MINB) k_persist_tile(S* f0, S* f1, Grid g, Coeffs c,
                                                                unsigned* __restrict__ health, unsigned* bar,
                                                                int nsteps) {
  constexpr int TW = BX, TH = BY * RY;
  const int tiles_x = (g.nx + TW - 1) / TW, tiles = tiles_x * ((g.ny + TH - 1) / TH);
  unsigned gen = read_gen(bar);
  for (int s = 0; s < nsteps; ++s) {
    const S* in = (s & 1) ? f1 : f0;
    S* out = (s & 1) ? f0 : f1;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      step_tile<S, BX, BY, RY, false, WRAPY, false, false, true>(in, out, g, c, health, t % tiles_x, t / tiles_x);
      __syncthreads();
    }
    if (s + 1 < nsteps && !grid_barrier(bar, gridDim.x, gen, kBarrierIters)) {
      if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(health, H_TIMEOUT);
      return;
    }
  }
}

// Self-test of the barrier: nblocks CTAs meet `rounds` times; with skip, CTA 1 never arrives.
__global__ void k_barrier_selftest(unsigned* bar, unsigned* out, int skip, int limit, int rounds) {
  unsigned gen = read_gen(bar);
  if (skip && blockIdx.x == 1) return;
  for (int r = 0; r < rounds; ++r) {
    if (!grid_barrier(bar, gridDim.x, gen, limit)) {
      if (threadIdx.x == 0) atomicOr(out, 1u);  // gave up
      return;
    }
  }
}

// block: the CTA shape the tile body indexes (8 x 4 quads of 4 lanes flat for the ring-parallel
// body; 32 x 8 for the tile body).
template <typename K>
cudaError_t coop_launch(K kernel, int tiles, dim3 block, void** args, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (int)(block.x * block.y * block.z), 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = tiles < per_sm * sms ? tiles : per_sm * sms;
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kernel), dim3(grid), block, args, 0, s);
}

template <typename S>
cudaError_t persist_t(int variant, void* f0, void* f1, int nsteps, const Grid& g, const Coeffs& c, unsigned* health,
                      unsigned* bar, cudaStream_t s) {
  S* a = static_cast<S*>(f0);
  S* b = static_cast<S*>(f1);
  Grid gg = g;
  Coeffs cc = c;
  void* args[] = {&a, &b, &gg, &cc, &health, &bar, &nsteps};
  if (variant == V_PRP8x4) {
    const int tiles = ((g.nx + 7) / 8) * ((g.ny + 3) / 4);
    return coop_launch(k_persist_rp<S, 8, 4>, tiles, dim3(128), args, s);
  }
  // V_PT32x16: the 32 x 16 tile, in its periodic-height form when one tile holds the grid's height
  const int tiles = ((g.nx + 31) / 32) * ((g.ny + 15) / 16);
  if (g.ny <= 16 && g.bc[2] == BC_PERIODIC && g.bc[3] == BC_PERIODIC)
    return coop_launch(k_persist_tile<S, 32, 8, 2, 2, true>, tiles, dim3(32, 8), args, s);
  return coop_launch(k_persist_tile<S, 32, 8, 2, 2, false>, tiles, dim3(32, 8), args, s);
}

}  // namespace

cudaError_t launch_steps_persist(int prec, int variant, void* f0, void* f1, int nsteps, const Grid& g,
                                 const Coeffs& c, unsigned* health, unsigned* bar, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  return prec == FDLBM_FP64 ? persist_t<double>(variant, f0, f1, nsteps, g, c, health, bar, s)
                            : persist_t<float>(variant, f0, f1, nsteps, g, c, health, bar, s);
}

}  // namespace fdlbm

extern "C" int fdlbm_selftest_grid_barrier(int skip, int iters, int rounds, int* completed) {
  if (!completed || iters < 1 || rounds < 1) return FDLBM_E_ARG;
  unsigned* d = nullptr;
  if (cudaMalloc(&d, 3 * sizeof(unsigned)) != cudaSuccess) return FDLBM_E_CUDA;
  unsigned h = 2;
  cudaError_t e = cudaMemset(d, 0, 3 * sizeof(unsigned));
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    unsigned* bar = d;
    unsigned* out = d + 2;
    void* args[] = {&bar, &out, &skip, &iters, &rounds};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(fdlbm::k_barrier_selftest), dim3(sms), dim3(64), args,
                                    0, nullptr);
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d + 2, sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return FDLBM_E_CUDA;
  *completed = h ? 0 : 1;
  return h ? FDLBM_E_TIMEOUT : FDLBM_OK;
}

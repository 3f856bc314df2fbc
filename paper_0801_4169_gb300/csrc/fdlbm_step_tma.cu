// fdlbm_step_tma.cu -- the FP32-storage step with its tile brought into shared memory by the
// tensor memory accelerator (variant V_TMA32x8).
//
// One CTA of 32 x 8 threads updates a 32 x 8 tile. Everything the tile's update reads from f --
// the 33 planes over the tile and its 2-node halo, a 36 x 12 x 33 box of FP32 values (57 KB) --
// arrives with a single cp.async.bulk.tensor copy issued by one thread, which completes on an
// mbarrier in shared memory. The moments of the tile and its 1-node ring (Eqs. 3-5, exact
// fixed-point sums), the switch (Eq. 16) and the Eq. 17 stencils then read shared memory at
// offsets known at compile time, instead of global loads with 64-bit address arithmetic. The
// arithmetic of every node is that of the other FP32-storage variants, so results are bitwise
// the same. The equilibrium is formed ring by ring between the stencils (FP64, or double-word
// FP32 for FDLBM_FP32_STORE_DW). 69 KB of shared memory per CTA: three CTAs per SM. With the
// double-word equilibrium this is the fastest FP32-storage step (2.42 against 3.11 ms per 4096^2
// step for the staged 32 x 8 tile); with the FP64 one the FP64 pipe binds and it gains nothing.
//
// The box is addressed in padded-grid coordinates: for the tile at node (x0, y0) it starts at
// padded column x0 (node x0 - 2) and padded row y0, so its first coordinate is a multiple of 32
// FP32 values (128 bytes). Parts of the box beyond the padded grid (the last tile row or column)
// read as zeros and belong to nodes no update reads.
//
// The mbarrier wait is bounded: after kWaitIters polls the CTA records FDLBM_HEALTH_TIMEOUT, waits
// once more with the same bound for its copy in flight, and returns without writing.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "fdlbm_kernels.cuh"

namespace fdlbm {

namespace {

constexpr int kTW = 32, kTH = 8;                 // tile (threads)
constexpr int kBW = kTW + 2 * NG, kBH = kTH + 2 * NG;  // box: the tile and its 2-node halo
constexpr int kBP = kBW * kBH;                   // values per plane of the box
constexpr int kBoxBytes = Q * kBP * (int)sizeof(float);
constexpr int kSmemBytes = kBoxBytes + 16;       // the box, then the mbarrier (8-byte aligned)
constexpr int kWaitIters = 1 << 20;
static_assert(kBoxBytes % 16 == 0 && (kBW * sizeof(float)) % 16 == 0, "TMA box rows must be 16-byte multiples");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  // make the initialised barrier visible to the tensor-copy unit (async proxy)
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// true once the barrier's phase `parity` has completed; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = kWaitIters) {
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Moments of the node whose box entry (plane 0) is at s[idx]; same arithmetic as node_moments.
__device__ __forceinline__ Macro box_macro(const float* __restrict__ s, int idx) {
  float x[Q];
  int emax = 1, emin = 255;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    x[q] = s[q * kBP + idx];
    const int e = (int)((__float_as_uint(x[q]) >> 23) & 0xffu);
    emax = max(emax, e);
    emin = min(emin, e);
  }
  Mom m;
  if (emax == 255) m = nan_moments();
  else if (emin > 0 && emax - emin <= FIX_TOP) m = fix_node_moments<false>(x, emax);
  else m = fix_node_moments<true>(x, emax);
  return to_macro<100>(m);
}

// Eq. 17 for direction D from the box (p: the node's entry in this velocity's plane).
template <int D>
__device__ __forceinline__ float box_stencil(const float* __restrict__ p, const RingW<float>& w, float rfeq) {
  constexpr int XS = dir_xs(D), YS = dir_ys(D), CL = dir_cls(D), CC = dir_c2(D);
  float acc = fmaf(w.w0[CC], p[0], rfeq);
  if (XS == 0) {
    acc = fmaf(w.nu[0], p[1] + p[-1], acc);
  } else {
    const float cp = XS > 0 ? w.P1[0][CL] : w.M1[0][CL];
    const float cm = XS > 0 ? w.M1[0][CL] : w.P1[0][CL];
    acc = fmaf(cp, p[1], acc);
    acc = fmaf(cm, p[-1], acc);
    const float d2 = p[2] - p[-2];
    acc = XS > 0 ? fmaf(w.Dd[0][CL], d2, acc) : fmaf(-w.Dd[0][CL], d2, acc);
  }
  if (YS == 0) {
    acc = fmaf(w.nu[1], p[kBW] + p[-kBW], acc);
  } else {
    const float cp = YS > 0 ? w.P1[1][CL] : w.M1[1][CL];
    const float cm = YS > 0 ? w.M1[1][CL] : w.P1[1][CL];
    acc = fmaf(cp, p[kBW], acc);
    acc = fmaf(cm, p[-kBW], acc);
    const float d2 = p[2 * kBW] - p[-2 * kBW];
    acc = YS > 0 ? fmaf(w.Dd[1][CL], d2, acc) : fmaf(-w.Dd[1][CL], d2, acc);
  }
  return acc;
}

// The 8 velocities of ring K at one node: their r f_eq (FP64 pairs rounded to FP32, or the
// double-word pairs), the stencils from the box, and the store with the node's ghost copies.
template <typename ES>
__device__ __forceinline__ void box_ring(int K, const float* __restrict__ sp, float* __restrict__ fn, const Grid& g,
                                         const Coeffs& c, int gx, int gy, const GhostOwn& go, const ES& e,
                                         float w0base, float nux, float nuy) {
  using SC = StencilConsts<float>;
  RingW<float> w;
#pragma unroll
  for (int l = 0; l < 3; ++l) w.w0[l] = w0base - SC::C2(c, K, l);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const float nu = a == 0 ? nux : nuy;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      w.P1[a][l] = SC::W1(c, a, K, l) + nu;
      w.M1[a][l] = SC::Wm1(c, a, K, l) + nu;
      w.Dd[a][l] = SC::D(c, a, K, l);
    }
  }
  w.nu[0] = nux;
  w.nu[1] = nuy;
  float fe[8];
  if constexpr (std::is_same<ES, EqSiteDW>::value) {
    const EqRingDW er = eq_ring_dw(e, K, c);
    eq_pair_dw(er, e.p[0], e.x[0], fe[7], fe[3]);
    eq_pair_dw(er, e.p[1], e.x[1], fe[0], fe[4]);
    eq_pair_dw(er, e.p[2], e.x[2], fe[1], fe[5]);
    eq_pair_dw(er, e.p[3], e.x[3], fe[2], fe[6]);
  } else {
    const EqRing er = eq_ring(e, K, c);
    eq_pair_s<float>(er, e.p[0], e.x[0], fe[7], fe[3]);
    eq_pair_s<float>(er, e.p[1], e.x[1], fe[0], fe[4]);
    eq_pair_s<float>(er, e.p[2], e.x[2], fe[1], fe[5]);
    eq_pair_s<float>(er, e.p[3], e.x[3], fe[2], fe[6]);
  }
  const float* pk = sp + (1 + 8 * K) * kBP;
  float out[8];
  out[0] = box_stencil<0>(pk + 0 * kBP, w, fe[0]);
  out[1] = box_stencil<1>(pk + 1 * kBP, w, fe[1]);
  out[2] = box_stencil<2>(pk + 2 * kBP, w, fe[2]);
  out[3] = box_stencil<3>(pk + 3 * kBP, w, fe[3]);
  out[4] = box_stencil<4>(pk + 4 * kBP, w, fe[4]);
  out[5] = box_stencil<5>(pk + 5 * kBP, w, fe[5]);
  out[6] = box_stencil<6>(pk + 6 * kBP, w, fe[6]);
  out[7] = box_stencil<7>(pk + 7 * kBP, w, fe[7]);
  store_ring<float>(fn, g, gx, gy, go, K, out);
}

// ROLL: the four rings run as a loop instead of unrolled (a quarter of phase 2's code).
template <bool DW, int MINB, bool ROLL>
__global__ void __launch_bounds__(kTW * kTH, MINB)
    k_step_tma(const __grid_constant__ CUtensorMap tmap, float* __restrict__ fn, Grid g, Coeffs c,
               unsigned* __restrict__ health) {
  constexpr int SW = kTW + 2, SH = kTH + 2, NT = kTW * kTH;
  extern __shared__ __align__(128) unsigned char s_box[];
  float* s_f = reinterpret_cast<float*>(s_box);  // [Q][kBH][kBW]
  unsigned long long* s_bar = reinterpret_cast<unsigned long long*>(s_box + kBoxBytes);
  __shared__ double s_n[SH][SW], s_ux[SH][SW], s_uy[SH][SW], s_T[SH][SW];
  __shared__ float s_P[SH][SW];
  const int tid = threadIdx.y * kTW + threadIdx.x;
  const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
  const uint32_t bar = smem_u32(s_bar);
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(bar, kBoxBytes);
    tma_load_3d(smem_u32(s_f), &tmap, x0, y0, 0, bar);
  }
  const bool arrived = mbar_wait(bar, 0);
  if (__syncthreads_or(!arrived)) {
    // the copy did not complete in time: report it, let the copy land, write nothing
    if (tid == 0) atomicOr(health, H_TIMEOUT);
    mbar_wait(bar, 0);
    return;
  }

  // Phase 1: moments of the tile and its ring (interior nodes and the ghost layer next to each
  // edge; corners are never read). Node (lx, ly) of the ring region sits at box (lx + 1, ly + 1).
  // Slots 0..32 SH - 1 take the first 32 nodes of each row, one row per warp, so a warp's box reads
  // are consecutive words (no bank conflicts); the last 2 SH slots take columns 32 and 33.
  static_assert(SW == kTW + 2, "the slot map covers rows of kTW + 2 nodes");
  unsigned bits = 0;
  constexpr int NSLOT = (SW * SH + NT - 1) / NT;
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) {
    const int idx = tid + k * NT;
    if ((k + 1) * NT > SW * SH && idx >= SW * SH) continue;
    const bool body = idx < kTW * SH;
    const int lx = body ? idx % kTW : kTW + (idx - kTW * SH) % 2;
    const int ly = body ? idx / kTW : (idx - kTW * SH) / 2;
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    const bool inx = gx >= 0 && gx < g.nx, iny = gy >= 0 && gy < g.ny;
    const bool need = (inx && iny) || (iny && (gx == -1 || gx == g.nx)) || (inx && (gy == -1 || gy == g.ny));
    const Macro m = box_macro(s_f, (ly + 1) * kBW + (lx + 1));
    if (need) {
      if (!macro_ok(m)) bits |= H_NUMERIC;
      s_n[ly][lx] = m.n;
      s_ux[ly][lx] = m.ux;
      s_uy[ly][lx] = m.uy;
      s_T[ly][lx] = m.T;
      s_P[ly][lx] = from_d<float>(m.P);
    }
  }
  __syncthreads();

  // Phase 2: Eq. 17 at the tile's node of this thread.
  const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
  if (gx < g.nx && gy < g.ny) {
    using SC = StencilConsts<float>;
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
    const double n = s_n[ly][lx], ux = s_ux[ly][lx], uy = s_uy[ly][lx], T = s_T[ly][lx];
    float thx, thy;
    if (g.flags & F_SWITCH_CONST) {
      thx = SC::lam(c);
      thy = SC::lam(c);
    } else {
      const float P0 = s_P[ly][lx];
      const float sx = s_P[ly][lx + 1] + s_P[ly][lx - 1], sy = s_P[ly + 1][lx] + s_P[ly - 1][lx];
      thx = SC::lam(c) * fabsf(fmaf(-2.f, P0, sx) * recip(fmaf(2.f, P0, sx)));
      thy = SC::lam(c) * fabsf(fmaf(-2.f, P0, sy) * recip(fmaf(2.f, P0, sy)));
    }
    const float akx = fabsf(from_d<float>(ux) * SC::kx(c)), aky = fabsf(from_d<float>(uy) * SC::ky(c));
    if (akx > 1.f || aky > 1.f) bits |= H_KAPPA;
    float snux = 0.f, snuy = 0.f;
    if (!(g.flags & F_NO_VISC)) {
      snux = 0.5f * thx * akx * (1.f - akx);
      snuy = 0.5f * thy * aky * (1.f - aky);
    }
    const float w0base = (1.f - SC::r(c)) - 2.f * (snux + snuy);
    using ES = typename std::conditional<DW, EqSiteDW, EqSite>::type;
    ES e;
    if constexpr (DW) e = eq_site_dw(n, ux, uy, T, c);
    else e = eq_site(n, ux, uy, T, c);
    const GhostOwn go = ghost_own(g, gx, gy);
    const float* sp = s_f + (threadIdx.y + NG) * kBW + (threadIdx.x + NG);
    {
      float rfeq;
      if constexpr (DW) rfeq = e.rest;
      else rfeq = to_s<float>(e.rest);
      float acc = fmaf(w0base, sp[0], rfeq);
      acc = fmaf(snux, sp[1] + sp[-1], acc);
      acc = fmaf(snuy, sp[kBW] + sp[-kBW], acc);
      store_node<float, 0>(fn, g, gx, gy, go, acc);
    }
    if constexpr (ROLL) {
#pragma unroll 1
      for (int K = 0; K < 4; ++K) box_ring<ES>(K, sp, fn, g, c, gx, gy, go, e, w0base, snux, snuy);
    } else {
      box_ring<ES>(0, sp, fn, g, c, gx, gy, go, e, w0base, snux, snuy);
      box_ring<ES>(1, sp, fn, g, c, gx, gy, go, e, w0base, snux, snuy);
      box_ring<ES>(2, sp, fn, g, c, gx, gy, go, e, w0base, snux, snuy);
      box_ring<ES>(3, sp, fn, g, c, gx, gy, go, e, w0base, snux, snuy);
    }
  }
  if (bits) atomicOr(health, bits);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time dependency on the
// driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

// The tensor map of one FP32 distribution buffer: 3-D (column, row, plane) over the padded grid,
// box kBW x kBH x Q, zeros outside.
static cudaError_t tile_map(CUtensorMap* map, const void* f, const Grid& g) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)g.rows, (cuuint64_t)Q};
  const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * sizeof(float), (cuuint64_t)g.plane * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)kBW, (cuuint32_t)kBH, (cuuint32_t)Q};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(f), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <bool DW, bool ROLL>
static cudaError_t launch_tma_t(const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                                cudaStream_t s) {
  CUtensorMap map;
  cudaError_t e = tile_map(&map, f, g);
  if (e != cudaSuccess) return e;
  static std::atomic<unsigned long long> attr{0};  // devices already opted in
  e = allow_dynamic_smem(k_step_tma<DW, 3, ROLL>, kSmemBytes, attr);
  if (e != cudaSuccess) return e;
  dim3 block(kTW, kTH), grid((g.nx + kTW - 1) / kTW, (g.ny + kTH - 1) / kTH);
  k_step_tma<DW, 3, ROLL><<<grid, block, kSmemBytes, s>>>(map, static_cast<float*>(fn), g, c, health);
  return cudaGetLastError();
}

// The double-word equilibrium runs its rings as a loop (2.42 against 2.57 ms per 4096^2 step: its
// unrolled phase 2 overflows the instruction cache); the FP64 one unrolled (4.77 against 5.65 ms).
// A padded grid smaller than one box (nx + 4 < 36 columns or ny + 4 < 12 rows) runs the 32 x 8 tile.
cudaError_t launch_step_tma(bool dw, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                            cudaStream_t s) {
  if (g.pitch < kBW || g.rows < kBH)
    return dw ? launch_step_f32dw(V_T32x8, f, fn, g, c, health, s) : launch_step_f32(V_T32x8, f, fn, g, c, health, s);
  return dw ? launch_tma_t<true, true>(f, fn, g, c, health, s) : launch_tma_t<false, false>(f, fn, g, c, health, s);
}

namespace {
// Self-test of the bounded wait: one CTA initialises an mbarrier for one arrival, arrives on it or
// not, and every thread waits with the given limit; out[0] = 1 if all saw the phase complete.
__global__ void k_wait_selftest(unsigned* out, int arrive, int iters) {
  __shared__ unsigned long long s_bar;
  const uint32_t bar = smem_u32(&s_bar);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (arrive && threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
  const bool ok = mbar_wait(bar, 0, iters);
  const int all = __syncthreads_and(ok);
  if (threadIdx.x == 0) out[0] = all ? 1u : 0u;
}
}  // namespace

}  // namespace fdlbm

extern "C" int fdlbm_selftest_wait(int arrive, int iters, int* completed) {
  if (!completed || iters < 1) return FDLBM_E_ARG;
  unsigned* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(unsigned));
  if (e != cudaSuccess) return FDLBM_E_CUDA;
  unsigned h = 2;
  fdlbm::k_wait_selftest<<<1, 64>>>(d, arrive, iters);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return FDLBM_E_CUDA;
  *completed = (int)h;
  return h ? FDLBM_OK : FDLBM_E_TIMEOUT;
}

namespace fdlbm {

}  // namespace fdlbm

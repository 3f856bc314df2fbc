// fdlbm_fneq.cu -- FDLBM_FNEQ32: the distribution stored as its departure from the local
// equilibrium (Gan, Xu, Zhang, Yu, Li, arXiv 0801.4169, Eqs. 3-5, 10-17).
//
// Per node a state buffer holds the macros n, ux, uy, T in FP64 and g_q = f_q - f_q^eq(n, u, T)
// (Eq. 10) in FP32. At high Mach number the equilibrium values reach kappa * n with kappa =
// sum |f_eq| / n up to 1e9, and they cancel in the moments: stored in FP32, f itself carries an
// error of kappa * 2^-24 * n, which can exceed the temperature. g is small wherever the flow is
// near equilibrium, so its FP32 rounding (2^-24 |g|) is not.
//
// One step of one CTA tile (TW x TH interior nodes, one thread per node):
//   A  for every node of the tile and its cross-shaped halo of width 2 (the nodes Eq. 17 reads):
//      load (n, u, T), form the equilibrium's site constants (Eqs. 11-13) and P = nT, in FP64,
//      into shared memory. Input nodes of the tile and its 1-node ring are health-checked.
//   B  per velocity ring (the rest velocity with ring 0): every halo node rebuilds its 8 values
//      f = f_eq + g in FP64 into shared memory; then every tile node applies Eq. 17 to them in
//      FP64 (the switch of Eq. 16 and kappa of Eq. 15 in FP64) and keeps f_new in registers,
//      summing the ring's part of the new moments.
//   C  each tile node forms its new moments (Eqs. 3-5, FP64, the pairwise ring tree of the FP64
//      path), their equilibrium, and stores g_new = f_new - f_eq_new in FP32 with the new
//      macros, plus the ghost copies it owns (walls mirror g's directions and reverse the
//      normal velocity of the macros).
// The equilibrium is the FP64 path's even/odd pair form, evaluated with dt/tau = 1 (plain
// f_eq); mirrored states give bit-for-bit mirrored values, so wall ghosts are exact mirrors.
#include "fdlbm_kernels.cuh"

namespace fdlbm {
namespace {

struct FneqState {
  float* g;    // 33 planes
  double* M;   // 4 planes: n, ux, uy, T
};
__device__ __forceinline__ FneqState fneq_state(void* f, const Grid& gr) {
  return FneqState{static_cast<float*>(f),
                   reinterpret_cast<double*>(static_cast<unsigned char*>(f) + gr.aux_off)};
}
__device__ __forceinline__ const float* fneq_g(const void* f) { return static_cast<const float*>(f); }
__device__ __forceinline__ const double* fneq_M(const void* f, const Grid& gr) {
  return reinterpret_cast<const double*>(static_cast<const unsigned char*>(f) + gr.aux_off);
}

// FP32 -> FP64 exactly, with the integer form for normal values (the hardware conversion issues
// on the FP64 pipe); zero keeps its sign; subnormal, infinite and NaN values go out of line.
__device__ __noinline__ double g_to_f64_rare(float x) { return (double)x; }
__device__ __forceinline__ double g_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = u & 0x7f800000u;
  if (__builtin_expect(e - 0x00800000u < 0x7f000000u, 1)) return f32_to_f64_bits(x);
  if ((u << 1) == 0u) return __longlong_as_double((long long)(u & 0x80000000u) << 32);
  return g_to_f64_rare(x);
}

// The equilibrium's site constants with dt/tau = 1 (plain f_eq): the same arithmetic as eq_site
// with r = 1, which is also what the initial condition of every precision uses.
__device__ __forceinline__ EqSite eq_site1(double n, double ux, double uy, double T, const Coeffs& c) {
  EqSite e;
  const double th = T;
  const double ith = rcp64(th);
  const double px = ux * ith, py = uy * ith;
  e.p[0] = px;
  e.p[1] = kS * (px + py);
  e.p[2] = py;
  e.p[3] = kS * (py - px);
#pragma unroll
  for (int t = 0; t < 4; ++t) e.x[t] = e.p[t] * e.p[t];
  const double b2 = fma(ux, px, uy * py);
  e.A1 = fma(-0.5, b2, 1.0);
  e.A0 = fma(0.125 * b2, b2, e.A1);
  const double rn = 1.0 * n, rnth = rn * th;
  double snF = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    e.nF[k] = rnth * fma(th, fma(th, fma(th, c.Fh[k][3], c.Fh[k][2]), c.Fh[k][1]), c.Fh[k][0]);
    snF += e.nF[k];
  }
  e.rest = fma(-8.0, snF, rn) * e.A0;
  return e;
}

// f_eq of ring K's 8 directions (index d as in the velocity ordering) from the site constants.
__device__ __forceinline__ void ring_feq(const EqSite& e, int K, const Coeffs& c, double (&fe)[8]) {
  const EqRing er = eq_ring(e, K, c);
  eq_pair(er, e.p[0], e.x[0], fe[7], fe[3]);
  eq_pair(er, e.p[1], e.x[1], fe[0], fe[4]);
  eq_pair(er, e.p[2], e.x[2], fe[1], fe[5]);
  eq_pair(er, e.p[3], e.x[3], fe[2], fe[6]);
}

// The macros of a node plus the ghost copies it owns (a wall reverses the normal velocity).
__device__ __forceinline__ void store_macros(double* __restrict__ M, const Grid& g, int gx, int gy,
                                             const GhostOwn& go, double n, double ux, double uy, double T) {
  const long long P = g.plane;
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  M[off] = n;
  M[P + off] = ux;
  M[2 * P + off] = uy;
  M[3 * P + off] = T;
  if (go.mx | go.my) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (go.mx & (1u << t)) {
        const int cc = ghost_coord(t, g.nx);
        const bool wall = (cc < 0 ? g.bc[0] : g.bc[1]) == BC_WALL;
        const long long o = (long long)(gy + NG) * g.pitch + (cc + NG);
        M[o] = n;
        M[P + o] = wall ? -ux : ux;
        M[2 * P + o] = uy;
        M[3 * P + o] = T;
      }
      if (go.my & (1u << t)) {
        const int cc = ghost_coord(t, g.ny);
        const bool wall = (cc < 0 ? g.bc[2] : g.bc[3]) == BC_WALL;
        const long long o = (long long)(cc + NG) * g.pitch + (gx + NG);
        M[o] = n;
        M[P + o] = ux;
        M[2 * P + o] = wall ? -uy : uy;
        M[3 * P + o] = T;
      }
    }
  }
}

// Eq. 17 for direction D of a ring at a tile node, from FP64 values in shared memory
// (box row length BW): the fma chain of stencil_dir, with rfe = (dt/tau) f_eq at the node.
template <int D>
__device__ __forceinline__ double stencil_s(const double* p, int bw, const RingW<double>& w, double rfe) {
  constexpr int XS = dir_xs(D), YS = dir_ys(D), CL = dir_cls(D), CC = dir_c2(D);
  double acc = fma(w.w0[CC], p[0], rfe);
  if (XS == 0) {
    acc = fma(w.nu[0], p[1] + p[-1], acc);
  } else {
    const double cp = XS > 0 ? w.P1[0][CL] : w.M1[0][CL];
    const double cm = XS > 0 ? w.M1[0][CL] : w.P1[0][CL];
    acc = fma(cp, p[1], acc);
    acc = fma(cm, p[-1], acc);
    const double d2 = p[2] - p[-2];
    acc = XS > 0 ? fma(w.Dd[0][CL], d2, acc) : fma(-w.Dd[0][CL], d2, acc);
  }
  if (YS == 0) {
    acc = fma(w.nu[1], p[bw] + p[-bw], acc);
  } else {
    const double cp = YS > 0 ? w.P1[1][CL] : w.M1[1][CL];
    const double cm = YS > 0 ? w.M1[1][CL] : w.P1[1][CL];
    acc = fma(cp, p[bw], acc);
    acc = fma(cm, p[-bw], acc);
    const double d2 = p[2 * bw] - p[-2 * bw];
    acc = YS > 0 ? fma(w.Dd[1][CL], d2, acc) : fma(-w.Dd[1][CL], d2, acc);
  }
  return acc;
}

// Shared memory of one CTA (doubles): site constants (15) and P per box node, the rebuilt f of
// the current pass (9 values: a ring's 8 and, in pass 0, the rest velocity) per box node, and the
// same passes' f_eq at the tile nodes. Box = tile + 2 on every side; its corners are unused.
constexpr int SC_N = 15;  // A0, A1, p[4], x[4], nF[4], rest
template <int TW, int TH>
constexpr int fneq_smem_bytes() {
  return ((SC_N + 1 + 9) * (TW + 4) * (TH + 4) + 9 * TW * TH) * (int)sizeof(double);
}

// One tile (tx, ty) of one solve: the body of the single-solve and the batched kernels, so a
// node's arithmetic is the same alone and in a batch.
template <int BX, int BY>
__device__ __forceinline__ void fneq_tile(const void* __restrict__ fin, void* __restrict__ fout, const Grid& g,
                                          const Coeffs& c, unsigned* __restrict__ health, int tile_x, int tile_y,
                                          unsigned char* s_dyn) {
  constexpr int TW = BX, TH = BY, BW = TW + 4, BH = TH + 4, BN = BW * BH, NT = BX * BY, TN = TW * TH;
  double* s_c = reinterpret_cast<double*>(s_dyn);  // [SC_N][BN]
  double* s_P = s_c + SC_N * BN;                    // [BN]
  double* s_f = s_P + BN;                           // [9][BN]
  double* s_fe = s_f + 9 * BN;                      // [9][TN]
  const float* gin = fneq_g(fin);
  const double* Min = fneq_M(fin, g);
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int x0 = tile_x * TW, y0 = tile_y * TH;
  const int xe = min(x0 + TW, g.nx), ye = min(y0 + TH, g.ny);  // end of the tile's real nodes
  unsigned bits = 0;

  // A: site constants of every node the tile's stencils read
  for (int idx = tid; idx < BN; idx += NT) {
    const int lx = idx % BW, ly = idx / BW;
    const int gx = x0 + lx - 2, gy = y0 + ly - 2;
    const bool colband = gx >= x0 && gx < xe && gy >= y0 - 2 && gy < ye + 2;
    const bool rowband = gy >= y0 && gy < ye && gx >= x0 - 2 && gx < xe + 2;
    if (!(colband || rowband)) continue;
    const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
    const double n = Min[off], ux = Min[g.plane + off], uy = Min[2 * g.plane + off], T = Min[3 * g.plane + off];
    // the step's input is checked on the tile and its 1-node ring (where the FP64 path takes moments)
    const bool ring1 = gx >= x0 - 1 && gx <= xe && gy >= y0 - 1 && gy <= ye;
    if (ring1 && !(pos_finite_bits(n) && pos_finite_bits(T) && finite_bits(ux) && finite_bits(uy))) bits |= H_NUMERIC;
    const EqSite e = eq_site1(n, ux, uy, T, c);
    s_c[0 * BN + idx] = e.A0;
    s_c[1 * BN + idx] = e.A1;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      s_c[(2 + t) * BN + idx] = e.p[t];
      s_c[(6 + t) * BN + idx] = e.x[t];
      s_c[(10 + t) * BN + idx] = e.nF[t];
    }
    s_c[14 * BN + idx] = e.rest;
    s_P[idx] = n * T;
  }
  __syncthreads();

  // this thread's tile node
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool mine = gx < g.nx && gy < g.ny;
  const int bidx = (ty + 2) * BW + (tx + 2), tidx = ty * TW + tx;
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  double snux = 0.0, snuy = 0.0, w0base = 0.0;
  if (mine) {
    const double ux = Min[g.plane + off], uy = Min[2 * g.plane + off];
    double thx, thy;
    if (g.flags & F_SWITCH_CONST) {
      thx = c.lam;
      thy = c.lam;
    } else {
      const double P0 = s_P[bidx];
      const double sx = s_P[bidx + 1] + s_P[bidx - 1], sy = s_P[bidx + BW] + s_P[bidx - BW];
      thx = c.lam * fabs(fma(-2.0, P0, sx) * rcp64(fma(2.0, P0, sx)));
      thy = c.lam * fabs(fma(-2.0, P0, sy) * rcp64(fma(2.0, P0, sy)));
    }
    const double akx = fabs(ux * c.kx), aky = fabs(uy * c.ky);
    if (akx > 1.0 || aky > 1.0) bits |= H_KAPPA;
    if (!(g.flags & F_NO_VISC)) {
      snux = 0.5 * thx * akx * (1.0 - akx);
      snuy = 0.5 * thy * aky * (1.0 - aky);
    }
    w0base = (1.0 - c.r) - 2.0 * (snux + snuy);
  }

  // B: per ring, rebuild f = f_eq + g on the box, then Eq. 17 at the tile node
  double fnew[Q];
  double S[4], X[4], Y[4];
#pragma unroll
  for (int K = 0; K < 4; ++K) {
    for (int idx = tid; idx < BN; idx += NT) {
      const int lx = idx % BW, ly = idx / BW;
      const int hx = x0 + lx - 2, hy = y0 + ly - 2;
      const bool colband = hx >= x0 && hx < xe && hy >= y0 - 2 && hy < ye + 2;
      const bool rowband = hy >= y0 && hy < ye && hx >= x0 - 2 && hx < xe + 2;
      if (!(colband || rowband)) continue;
      EqSite e;
      e.A0 = s_c[0 * BN + idx];
      e.A1 = s_c[1 * BN + idx];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        e.p[t] = s_c[(2 + t) * BN + idx];
        e.x[t] = s_c[(6 + t) * BN + idx];
        e.nF[t] = s_c[(10 + t) * BN + idx];
      }
      double fe[8];
      ring_feq(e, K, c, fe);
      const long long hoff = (long long)(hy + NG) * g.pitch + (hx + NG);
      const bool tile = hx >= x0 && hx < x0 + TW && hy >= y0 && hy < y0 + TH;
      const int ti = (hy - y0) * TW + (hx - x0);
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        const double gv = g_to_f64(ld(gin + (long long)(1 + 8 * K + d) * g.plane + hoff));
        s_f[d * BN + idx] = fe[d] + gv;
        if (tile) s_fe[d * TN + ti] = fe[d];
      }
      if (K == 0) {
        const double fe0 = s_c[14 * BN + idx];
        s_f[8 * BN + idx] = fe0 + g_to_f64(ld(gin + hoff));
        if (tile) s_fe[8 * TN + ti] = fe0;
      }
    }
    __syncthreads();
    if (mine) {
      RingW<double> w;
#pragma unroll
      for (int l = 0; l < 3; ++l) w.w0[l] = w0base - c.C2[K][l];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const double nu = a == 0 ? snux : snuy;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          w.P1[a][l] = c.W1[a][K][l] + nu;
          w.M1[a][l] = c.Wm1[a][K][l] + nu;
          w.Dd[a][l] = c.D[a][K][l];
        }
      }
      w.nu[0] = snux;
      w.nu[1] = snuy;
      double o[8];
      o[0] = stencil_s<0>(s_f + 0 * BN + bidx, BW, w, c.r * s_fe[0 * TN + tidx]);
      o[1] = stencil_s<1>(s_f + 1 * BN + bidx, BW, w, c.r * s_fe[1 * TN + tidx]);
      o[2] = stencil_s<2>(s_f + 2 * BN + bidx, BW, w, c.r * s_fe[2 * TN + tidx]);
      o[3] = stencil_s<3>(s_f + 3 * BN + bidx, BW, w, c.r * s_fe[3 * TN + tidx]);
      o[4] = stencil_s<4>(s_f + 4 * BN + bidx, BW, w, c.r * s_fe[4 * TN + tidx]);
      o[5] = stencil_s<5>(s_f + 5 * BN + bidx, BW, w, c.r * s_fe[5 * TN + tidx]);
      o[6] = stencil_s<6>(s_f + 6 * BN + bidx, BW, w, c.r * s_fe[6 * TN + tidx]);
      o[7] = stencil_s<7>(s_f + 7 * BN + bidx, BW, w, c.r * s_fe[7 * TN + tidx]);
#pragma unroll
      for (int d = 0; d < 8; ++d) fnew[1 + 8 * K + d] = o[d];
      ring_sums(o, S[K], X[K], Y[K]);
      if (K == 0) {
        // rest velocity: c = 0 on both axes, line IV only
        const double* p = s_f + 8 * BN + bidx;
        double acc = fma(w0base, p[0], c.r * s_fe[8 * TN + tidx]);
        acc = fma(snux, p[1] + p[-1], acc);
        acc = fma(snuy, p[BW] + p[-BW], acc);
        fnew[0] = acc;
      }
    }
    __syncthreads();
  }

  // C: new moments, their equilibrium, and g_new = f_new - f_eq_new
  if (mine) {
    const Macro m = to_macro<1>(combine_rings(fnew[0], S, X, Y, c));
    const EqSite e = eq_site1(m.n, m.ux, m.uy, m.T, c);
    const GhostOwn go = ghost_own(g, gx, gy);
    FneqState out = fneq_state(fout, g);
    store_node<float, 0>(out.g, g, gx, gy, go, f64_to_f32_rn(fnew[0] - e.rest));
#pragma unroll
    for (int K = 0; K < 4; ++K) {
      double fe[8];
      ring_feq(e, K, c, fe);
      float v[8];
#pragma unroll
      for (int d = 0; d < 8; ++d) v[d] = f64_to_f32_rn(fnew[1 + 8 * K + d] - fe[d]);
      store_ring<float>(out.g, g, gx, gy, go, K, v);
    }
    store_macros(out.M, g, gx, gy, go, m.n, m.ux, m.uy, m.T);
  }
  if (bits) atomicOr(health, bits);
}

template <int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB) k_step_fneq(const void* __restrict__ fin, void* __restrict__ fout,
                                                         Grid g, Coeffs c, unsigned* __restrict__ health) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  fneq_tile<BX, BY>(fin, fout, g, c, health, blockIdx.x, blockIdx.y, s_dyn);
}

// Batched step: block b runs tile (b - tile0) of the member whose [tile0, tile0 + tiles) holds b
// (members sorted by tile0), as k_step_batch does for the other precisions.
template <int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB) k_step_batch_fneq(const BatchMember* __restrict__ mem, int nmem,
                                                               unsigned long long step, Coeffs c) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ int s_sel;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const long long b = blockIdx.x;
    int lo = 0, hi = nmem - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (mem[mid].tile0 <= b) lo = mid;
      else hi = mid - 1;
    }
    s_sel = lo;
  }
  __syncthreads();
  const BatchMember& m = mem[s_sel];
  const Grid g = m.g;
  const long long local = (long long)blockIdx.x - m.tile0;
  const int tx = (int)(local % m.tiles_x), ty = (int)(local / m.tiles_x);
  const int par = (int)((m.cur0 + step) & 1ull);
  fneq_tile<BX, BY>(m.f[par], m.f[par ^ 1], g, c, m.health, tx, ty, s_dyn);
}

// Opt the batched kernel in to its dynamic shared memory (once per device); called outside any
// stream capture, before the batch's graph is recorded.
template <int BX, int BY, int MINB>
cudaError_t prepare_batch_fneq_t() {
  static std::atomic<unsigned long long> attr{0};
  return allow_dynamic_smem(k_step_batch_fneq<BX, BY, MINB>, fneq_smem_bytes<BX, BY>(), attr);
}

template <int BX, int BY, int MINB>
cudaError_t launch_batch_fneq_t(const BatchMember* mem, int nmem, long long tiles, unsigned long long step,
                                const Coeffs& c, cudaStream_t s) {
  constexpr int smem = fneq_smem_bytes<BX, BY>();
  const cudaError_t e = prepare_batch_fneq_t<BX, BY, MINB>();
  if (e != cudaSuccess) return e;
  k_step_batch_fneq<BX, BY, MINB><<<dim3((unsigned)tiles), dim3(BX, BY), smem, s>>>(mem, nmem, step, c);
  return cudaGetLastError();
}

template <int BX, int BY, int MINB>
cudaError_t launch_fneq_t(const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                          cudaStream_t s) {
  constexpr int smem = fneq_smem_bytes<BX, BY>();
  static std::atomic<unsigned long long> attr{0};
  const cudaError_t e = allow_dynamic_smem(k_step_fneq<BX, BY, MINB>, smem, attr);
  if (e != cudaSuccess) return e;
  dim3 block(BX, BY), grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY);
  k_step_fneq<BX, BY, MINB><<<grid, block, smem, s>>>(f, fn, g, c, health);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// set-up and read-out kernels

// f = f_eq(macros): macros stored, g = 0 (interior and owned ghosts).
__global__ void k_init_fneq(void* f, Grid g, const double* __restrict__ rho, const double* __restrict__ u,
                            const double* __restrict__ v, const double* __restrict__ T) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const long long m = (long long)gy * g.nx + gx;
  const GhostOwn go = ghost_own(g, gx, gy);
  FneqState st = fneq_state(f, g);
  store_node<float, 0>(st.g, g, gx, gy, go, 0.0f);
  const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int K = 0; K < 4; ++K) store_ring<float>(st.g, g, gx, gy, go, K, z);
  store_macros(st.M, g, gx, gy, go, rho[m], u[m], v[m], T[m]);
}

// Dirichlet ghosts: the side's state, g = 0, at both ghost layers next to the interior.
__global__ void k_dirichlet_fneq(void* f, Grid g, BState bs) {
  const int side = blockIdx.y;
  if (g.bc[side] != BC_DIRICHLET) return;
  const int len = side < 2 ? g.ny : g.nx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * len) return;
  const int along = t % len, layer = t / len;
  int gx, gy;
  if (side == 0) { gx = -1 - layer; gy = along; }
  else if (side == 1) { gx = g.nx + layer; gy = along; }
  else if (side == 2) { gx = along; gy = -1 - layer; }
  else { gx = along; gy = g.ny + layer; }
  GhostOwn none;
  none.mx = 0;
  none.my = 0;
  FneqState st = fneq_state(f, g);
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  for (int q = 0; q < Q; ++q) st.g[(long long)q * g.plane + off] = 0.0f;
  store_macros(st.M, g, gx, gy, none, bs.s[side][0], bs.s[side][1], bs.s[side][2], bs.s[side][3]);
}

// A side's Dirichlet segment (see launch_segment): the state's macros with g = 0.
__global__ void k_segment_fneq(void* f, Grid g, Segment sg, double d) {
  const int len = sg.side < 2 ? g.ny : g.nx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * len) return;
  const int along = t % len, layer = t / len;
  int gx, gy;
  if (sg.side == 0) { gx = -1 - layer; gy = along; }
  else if (sg.side == 1) { gx = g.nx + layer; gy = along; }
  else if (sg.side == 2) { gx = along; gy = -1 - layer; }
  else { gx = along; gy = g.ny + layer; }
  const double pos = ((double)along + 0.5) * d;
  const bool in = sg.lower ? (pos < sg.split) : !(pos < sg.split);
  if (!in && !sg.base_dirichlet) return;
  const double* st = in ? sg.seg : sg.base;
  GhostOwn none;
  none.mx = 0;
  none.my = 0;
  FneqState s = fneq_state(f, g);
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  for (int q = 0; q < Q; ++q) s.g[(long long)q * g.plane + off] = 0.0f;
  store_macros(s.M, g, gx, gy, none, st[0], st[1], st[2], st[3]);
}

__global__ void k_macro_fneq(const void* f, Grid g, double* __restrict__ rho, double* __restrict__ u,
                             double* __restrict__ v, double* __restrict__ T) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const double* M = fneq_M(f, g);
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  const long long o = (long long)gy * g.nx + gx;
  rho[o] = M[off];
  u[o] = M[g.plane + off];
  v[o] = M[2 * g.plane + off];
  T[o] = M[3 * g.plane + off];
}

// f = f_eq + g over a node window, FP64, layout [q][j][i].
__global__ void k_get_region_fneq(const void* f, Grid g, Coeffs c, int x0, int y0, int w, int h,
                                  double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= w || j >= h) return;
  const float* gq = fneq_g(f);
  const double* M = fneq_M(f, g);
  const long long off = (long long)(y0 + j + NG) * g.pitch + (x0 + i + NG);
  const EqSite e = eq_site1(M[off], M[g.plane + off], M[2 * g.plane + off], M[3 * g.plane + off], c);
  const long long cell = (long long)h * w, o = (long long)j * w + i;
  out[o] = e.rest + g_to_f64(gq[off]);
#pragma unroll
  for (int K = 0; K < 4; ++K) {
    double fe[8];
    ring_feq(e, K, c, fe);
#pragma unroll
    for (int d = 0; d < 8; ++d)
      out[(long long)(1 + 8 * K + d) * cell + o] = fe[d] + g_to_f64(gq[(long long)(1 + 8 * K + d) * g.plane + off]);
  }
}

// From raw f (FP64, [q][j][i]): macros = moments of f (Eqs. 3-5, FP64), g = f - f_eq(macros).
__global__ void k_set_f_fneq(void* f, Grid g, Coeffs c, const double* __restrict__ in) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const long long plane = (long long)g.nx * g.ny, o = (long long)gy * g.nx + gx;
  const Macro m = to_macro<1>(node_moments(in, plane, o, c));
  const EqSite e = eq_site1(m.n, m.ux, m.uy, m.T, c);
  const GhostOwn go = ghost_own(g, gx, gy);
  FneqState st = fneq_state(f, g);
  store_node<float, 0>(st.g, g, gx, gy, go, f64_to_f32_rn(in[o] - e.rest));
#pragma unroll
  for (int K = 0; K < 4; ++K) {
    double fe[8];
    ring_feq(e, K, c, fe);
    float v[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) v[d] = f64_to_f32_rn(in[(long long)(1 + 8 * K + d) * plane + o] - fe[d]);
    store_ring<float>(st.g, g, gx, gy, go, K, v);
  }
  store_macros(st.M, g, gx, gy, go, m.n, m.ux, m.uy, m.T);
}

}  // namespace

// Tile shapes (one thread per node, 256 threads unless noted; every shape gives bit-for-bit the
// same result): V_T32x4 32 x 4 (128 threads), V_T32x8 32 x 8 at <= 128 registers for 2 CTAs per
// SM (the fastest measured at 4096^2: 29.4 ms per step, 0.57 GLUPS), V_T16x4 16 x 16, V_T64x8
// 64 x 4; every other variant 32 x 8 at up to 255 registers (1 CTA per SM).
cudaError_t launch_step_fneq(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                             cudaStream_t s) {
  if (variant == V_T32x4) return launch_fneq_t<32, 4, 2>(f, fn, g, c, health, s);
  if (variant == V_T32x8) return launch_fneq_t<32, 8, 2>(f, fn, g, c, health, s);
  if (variant == V_T16x4) return launch_fneq_t<16, 16, 1>(f, fn, g, c, health, s);
  if (variant == V_T64x8) return launch_fneq_t<64, 4, 2>(f, fn, g, c, health, s);
  return launch_fneq_t<32, 8, 1>(f, fn, g, c, health, s);
}

// Batches of FNEQ32 solves take the 32 x 4 (V_T32x4) or the 32 x 8 (V_T32x8) tile, the shapes
// variant_tile gives for those variants.
cudaError_t launch_batch_fneq(int variant, const BatchMember* mem, int nmem, long long tiles, unsigned long long step,
                              const Coeffs& c, cudaStream_t s) {
  if (variant == V_T32x4) return launch_batch_fneq_t<32, 4, 2>(mem, nmem, tiles, step, c, s);
  if (variant == V_T32x8) return launch_batch_fneq_t<32, 8, 2>(mem, nmem, tiles, step, c, s);
  return cudaErrorInvalidValue;
}

cudaError_t prepare_batch_fneq(int variant) {
  if (variant == V_T32x4) return prepare_batch_fneq_t<32, 4, 2>();
  if (variant == V_T32x8) return prepare_batch_fneq_t<32, 8, 2>();
  return cudaErrorInvalidValue;
}

cudaError_t launch_init_fneq(void* f, const Grid& g, const Coeffs& c, const double* rho, const double* u,
                             const double* v, const double* T, cudaStream_t s) {
  (void)c;
  dim3 b(32, 4);
  k_init_fneq<<<grid2d(g, b), b, 0, s>>>(f, g, rho, u, v, T);
  return cudaGetLastError();
}

cudaError_t launch_dirichlet_fneq(void* f, const Grid& g, const double bstate[4][4], cudaStream_t s) {
  BState bs;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) bs.s[i][j] = bstate[i][j];
  const int len = 2 * (g.nx > g.ny ? g.nx : g.ny);
  dim3 b(128), grid((len + 127) / 128, 4);
  k_dirichlet_fneq<<<grid, b, 0, s>>>(f, g, bs);
  return cudaGetLastError();
}

cudaError_t launch_segment_fneq(void* f, const Grid& g, const Segment& sg, double dx, double dy, cudaStream_t s) {
  const int len = sg.side < 2 ? g.ny : g.nx;
  dim3 b(128), grid((2 * len + 127) / 128);
  k_segment_fneq<<<grid, b, 0, s>>>(f, g, sg, sg.side < 2 ? dy : dx);
  return cudaGetLastError();
}

cudaError_t launch_macro_fneq(const void* f, const Grid& g, double* rho, double* u, double* v, double* T,
                              cudaStream_t s) {
  dim3 b(32, 4);
  k_macro_fneq<<<grid2d(g, b), b, 0, s>>>(f, g, rho, u, v, T);
  return cudaGetLastError();
}

cudaError_t launch_get_region_fneq(const void* f, const Grid& g, const Coeffs& c, int x0, int y0, int w, int h,
                                   double* out, cudaStream_t s) {
  dim3 b(32, 4), grid((w + 31) / 32, (h + 3) / 4);
  k_get_region_fneq<<<grid, b, 0, s>>>(f, g, c, x0, y0, w, h, out);
  return cudaGetLastError();
}

cudaError_t launch_set_f_fneq(void* f, const Grid& g, const Coeffs& c, const double* in, cudaStream_t s) {
  dim3 b(32, 4);
  k_set_f_fneq<<<grid2d(g, b), b, 0, s>>>(f, g, c, in);
  return cudaGetLastError();
}

}  // namespace fdlbm

// fdlbm_strict.cu -- FDLBM_FP64_STRICT: the FP64 method in one canonical order of operations.
//
// Every value is formed from its defining equation one IEEE-754 FP64 operation at a time, in the
// order written below, each with an explicitly rounded intrinsic (__dadd_rn, __dsub_rn, __dmul_rn,
// __ddiv_rn, __dsqrt_rn): nothing is fused into a multiply-add, reassociated or replaced by a
// reciprocal. Any IEEE FP64 program that takes the same operations in the same order therefore
// produces the same bits, on any machine and under any compiler that keeps IEEE semantics.
//
//   velocities (Eq. 1)    v_q = v_k (cos, sin)(i pi/4) with the components 0, +-1, +-sqrt(1/2);
//                          q = 0 rest, q = 1 + 8k + d for ring k (speed v_{k+1}), angle (d + 1) pi/4.
//   moments (Eqs. 3-5)    n, jx, jy summed over q = 0..32 in turn (each product rounded before
//                          its sum); u = j / n; P = sum over q of ((1/2)(wx^2 + wy^2)) f_q with
//                          w = v_q - u; T = P / n (m = 1, so theta = T).
//   weights (Eqs. 11-13)  with a, b, c the squared speeds of the cyclic indices k+1, k+2, k+3:
//                          F_k = (((48 th^4 - (6 ((a + b) + c)) th^3) + (((ab + bc) + ca)) th^2)
//                                 - ((ab)c / 4) th) / (((v_k^2 (v_k^2 - a))(v_k^2 - b))(v_k^2 - c)),
//                          th^2 = th th, th^3 = th^2 th, th^4 = th^3 th; F_0 = 1 - 8 (((F_1 + F_2) + F_3) + F_4).
//   equilibrium (Eq. 10)  (n F_k) ((((t0 + t1) + t2) + t3) + t4) with h = 1 - u^2 / (2 th),
//                          t0 = h + u^4 / ((8 th) th), t1 = (v.u / th) h, t2 = ((v.u)^2 / ((2 th) th)) h,
//                          t3 = (v.u)^3 / (((6 th) th) th), t4 = (v.u)^4 / ((((24 th) th) th) th),
//                          powers by repeated products from the left, u^2 = ux ux + uy uy.
//   update (Eq. 17)       acc = f - r (f - f_eq), r = dt / tau; then for alpha = x, y in turn, with
//                          c = (v_alpha dt) / dr_alpha, kappa = (u_alpha dt) / dr_alpha:
//                          acc - (c / 2)(f+1 - f-1)                                       line I
//                          acc + ((c c) / 2)((f+1 - 2 f) + f-1)                           line II
//                          acc + ((c (1 - c c)) / 12)(((f+2 - 2 f+1) + 2 f-1) - f-2)      line III
//                          acc + (((theta_a |kappa|)(1 - |kappa|)) / 2)((f+1 - 2 f) + f-1) line IV
//                          theta_a = lambda |((P+ - 2 P0) + P-) / ((P+ + 2 P0) + P-)| (Eq. 16),
//                          P = n T at I+1, I, I-1 along alpha.
//
// It is the library's reference-grade path, not its fast one: one thread per node, no shared
// memory, every division a division. Two launches per step: the moments of every node that the
// update reads (the interior and the ghost layer next to each edge) into the moment buffer, then
// the update of every interior node with the ghost copies it owns (periodic, zero-gradient,
// mirror). Dirichlet ghosts, the initial condition and boundary segments take the same f_eq.
#include "fdlbm_kernels.cuh"

namespace fdlbm {

namespace {
namespace strict {

__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dvd(double a, double b) { return __ddiv_rn(a, b); }

// v_q of Eq. 1 (see the header comment for the ordering)
__device__ __forceinline__ void vel(int q, double& vx, double& vy) {
  if (q == 0) {
    vx = 0.0;
    vy = 0.0;
    return;
  }
  const int k = (q - 1) / 8, d = (q - 1) % 8;
  const double s = __dsqrt_rn(0.5);
  double cx, cy;
  switch (d) {
    case 0: cx = s; cy = s; break;        // 45 deg
    case 1: cx = 0.0; cy = 1.0; break;    // 90 deg
    case 2: cx = -s; cy = s; break;       // 135 deg
    case 3: cx = -1.0; cy = 0.0; break;   // 180 deg
    case 4: cx = -s; cy = -s; break;      // 225 deg
    case 5: cx = 0.0; cy = -1.0; break;   // 270 deg
    case 6: cx = s; cy = -s; break;       // 315 deg
    default: cx = 1.0; cy = 0.0; break;   // 0 deg
  }
  vx = mul(speed(k), cx);
  vy = mul(speed(k), cy);
}

// F_0..F_4 of Eqs. 11-13 at theta
__device__ __forceinline__ void weights(double th, double (&F)[5]) {
  double sumF = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double vk = speed(k), va = speed((k + 1) % 4), vb = speed((k + 2) % 4), vc = speed((k + 3) % 4);
    const double vk2 = mul(vk, vk), a = mul(va, va), b = mul(vb, vb), c = mul(vc, vc);
    const double den = mul(mul(mul(vk2, sub(vk2, a)), sub(vk2, b)), sub(vk2, c));
    const double t2 = mul(th, th), t3 = mul(t2, th), t4 = mul(t3, th);
    const double num = sub(add(sub(mul(48.0, t4), mul(mul(6.0, add(add(a, b), c)), t3)),
                               mul(add(add(mul(a, b), mul(b, c)), mul(c, a)), t2)),
                           mul(dvd(mul(mul(a, b), c), 4.0), th));
    F[k + 1] = dvd(num, den);
    sumF = add(sumF, F[k + 1]);
  }
  F[0] = sub(1.0, mul(8.0, sumF));
}

// f_eq of velocity q (Eq. 10)
__device__ __forceinline__ double feq(int q, double n, double ux, double uy, double th, const double (&F)[5]) {
  double vx, vy;
  vel(q, vx, vy);
  const double Fk = F[q == 0 ? 0 : 1 + (q - 1) / 8];
  const double u2 = add(mul(ux, ux), mul(uy, uy));
  const double vu = add(mul(vx, ux), mul(vy, uy));
  const double h = sub(1.0, dvd(u2, mul(2.0, th)));
  const double t0 = add(h, dvd(mul(u2, u2), mul(mul(8.0, th), th)));
  const double t1 = mul(dvd(vu, th), h);
  const double t2 = mul(dvd(mul(vu, vu), mul(mul(2.0, th), th)), h);
  const double t3 = dvd(mul(mul(vu, vu), vu), mul(mul(mul(6.0, th), th), th));
  const double t4 = dvd(mul(mul(mul(vu, vu), vu), vu), mul(mul(mul(mul(24.0, th), th), th), th));
  return mul(mul(n, Fk), add(add(add(add(t0, t1), t2), t3), t4));
}

struct Mac {
  double n, ux, uy, T;
};

// Eqs. 3-5 at the node at offset off
__device__ __forceinline__ Mac moments(const double* __restrict__ f, long long plane, long long off) {
  double x[Q];
  double n = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    x[q] = f[(long long)q * plane + off];
    double vx, vy;
    vel(q, vx, vy);
    n = add(n, x[q]);
    jx = add(jx, mul(vx, x[q]));
    jy = add(jy, mul(vy, x[q]));
  }
  Mac m;
  m.n = n;
  m.ux = dvd(jx, n);
  m.uy = dvd(jy, n);
  double P = 0.0;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    double vx, vy;
    vel(q, vx, vy);
    const double wx = sub(vx, m.ux), wy = sub(vy, m.uy);
    P = add(P, mul(mul(0.5, add(mul(wx, wx), mul(wy, wy))), x[q]));
  }
  m.T = dvd(P, n);
  return m;
}

__device__ __forceinline__ bool mac_ok(const Mac& m) {
  return isfinite(m.n) && isfinite(m.ux) && isfinite(m.uy) && isfinite(m.T) && m.n > 0.0 && m.T > 0.0;
}

// Raw scheme parameters: the ratios are formed on the device, in the order above.
struct Params {
  double dt, tau, dr[2], lam;
  int flags;
};

template <int QQ>
__device__ __forceinline__ void update_one(const double* __restrict__ f, double* __restrict__ fn, const Grid& g,
                                           const Params& p, long long off, int gx, int gy, const GhostOwn& go,
                                           const Mac& m, const double (&F)[5], double r, const double (&sw)[2],
                                           const double (&kap)[2]) {
  double vx, vy;
  vel(QQ, vx, vy);
  const double fe = feq(QQ, m.n, m.ux, m.uy, m.T, F);
  const double* fq = f + (long long)QQ * g.plane + off;
  const double f0 = fq[0];
  double acc = sub(f0, mul(r, sub(f0, fe)));
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const long long st = a == 0 ? 1 : g.pitch;
    const double fp1 = fq[st], fm1 = fq[-st], fp2 = fq[2 * st], fm2 = fq[-2 * st];
    const double c = dvd(mul(a == 0 ? vx : vy, p.dt), p.dr[a]);
    acc = sub(acc, mul(dvd(c, 2.0), sub(fp1, fm1)));
    if (!(p.flags & F_NO_LW)) acc = add(acc, mul(dvd(mul(c, c), 2.0), add(sub(fp1, mul(2.0, f0)), fm1)));
    if (!(p.flags & F_NO_DISP))
      acc = add(acc, mul(dvd(mul(c, sub(1.0, mul(c, c))), 12.0),
                         sub(add(sub(fp2, mul(2.0, fp1)), mul(2.0, fm1)), fm2)));
    if (!(p.flags & F_NO_VISC)) {
      const double ak = fabs(kap[a]);
      acc = add(acc, mul(dvd(mul(mul(sw[a], ak), sub(1.0, ak)), 2.0), add(sub(fp1, mul(2.0, f0)), fm1)));
    }
  }
  store_node<double, QQ>(fn, g, gx, gy, go, acc);
}

template <int... QS>
__device__ __forceinline__ void update_all(const double* __restrict__ f, double* __restrict__ fn, const Grid& g,
                                           const Params& p, long long off, int gx, int gy, const GhostOwn& go,
                                           const Mac& m, const double (&F)[5], double r, const double (&sw)[2],
                                           const double (&kap)[2]) {
  (update_one<QS>(f, fn, g, p, off, gx, gy, go, m, F, r, sw, kap), ...);
}

template <int QQ>
__device__ __forceinline__ void feq_one(double* __restrict__ f, const Grid& g, int gx, int gy, const GhostOwn& go,
                                        double n, double ux, double uy, double T, const double (&F)[5]) {
  store_node<double, QQ>(f, g, gx, gy, go, feq(QQ, n, ux, uy, T, F));
}
template <int... QS>
__device__ __forceinline__ void feq_all(double* __restrict__ f, const Grid& g, int gx, int gy, const GhostOwn& go,
                                        double n, double ux, double uy, double T) {
  double F[5];
  weights(T, F);
  (feq_one<QS>(f, g, gx, gy, go, n, ux, uy, T, F), ...);
}
__device__ __forceinline__ void write_feq(double* __restrict__ f, const Grid& g, int gx, int gy, const GhostOwn& go,
                                          double n, double ux, double uy, double T) {
  feq_all<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28,
          29, 30, 31, 32>(f, g, gx, gy, go, n, ux, uy, T);
}

// Moment-buffer planes (the grid's split-step buffer): n, ux, uy, T.
__device__ __forceinline__ double* mplane(const Grid& g, int a) { return static_cast<double*>(g.mom) + a * g.plane; }

// Pass 1: moments of the interior and of the ghost layer next to each edge (no corners).
__global__ void k_moments(const double* __restrict__ f, Grid g, unsigned* __restrict__ health) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x - 1, gy = blockIdx.y * blockDim.y + threadIdx.y - 1;
  if (gx > g.nx || gy > g.ny || !ring_node_needed(g, gx, gy)) return;
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  const Mac m = moments(f, g.plane, off);
  if (!mac_ok(m)) atomicOr(health, H_NUMERIC);
  mplane(g, 0)[off] = m.n;
  mplane(g, 1)[off] = m.ux;
  mplane(g, 2)[off] = m.uy;
  mplane(g, 3)[off] = m.T;
}

// Pass 2: Eq. 17 at every interior node.
__global__ void __launch_bounds__(128) k_update(const double* __restrict__ f, double* __restrict__ fn, Grid g,
                                                Params p, unsigned* __restrict__ health) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  const double* Mn = mplane(g, 0);
  const double* MT = mplane(g, 3);
  Mac m;
  m.n = Mn[off];
  m.ux = mplane(g, 1)[off];
  m.uy = mplane(g, 2)[off];
  m.T = MT[off];
  double F[5];
  weights(m.T, F);
  double sw[2], kap[2];
  unsigned bits = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const long long st = a == 0 ? 1 : g.pitch;
    const double Pp = mul(Mn[off + st], MT[off + st]);
    const double P0 = mul(m.n, m.T);
    const double Pm = mul(Mn[off - st], MT[off - st]);
    sw[a] = (p.flags & F_SWITCH_CONST)
                ? p.lam
                : mul(p.lam, fabs(dvd(add(sub(Pp, mul(2.0, P0)), Pm), add(add(Pp, mul(2.0, P0)), Pm))));
    kap[a] = dvd(mul(a == 0 ? m.ux : m.uy, p.dt), p.dr[a]);
    if (fabs(kap[a]) > 1.0) bits |= H_KAPPA;
  }
  const double r = dvd(p.dt, p.tau);
  update_all<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28,
             29, 30, 31, 32>(f, fn, g, p, off, gx, gy, ghost_own(g, gx, gy), m, F, r, sw, kap);
  if (bits) atomicOr(health, bits);
}

__global__ void k_init(double* __restrict__ f, Grid g, const double* __restrict__ rho, const double* __restrict__ u,
                       const double* __restrict__ v, const double* __restrict__ T) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const long long i = (long long)gy * g.nx + gx;
  write_feq(f, g, gx, gy, ghost_own(g, gx, gy), rho[i], u[i], v[i], T[i]);
}

// the ghost node t of a side's two layers (t < 2 len): coordinates and index along the side
__device__ __forceinline__ void side_ghost(const Grid& g, int side, int t, int& gx, int& gy, int& along) {
  const int len = side < 2 ? g.ny : g.nx;
  along = t % len;
  const int layer = t / len;
  if (side == 0) { gx = -1 - layer; gy = along; }
  else if (side == 1) { gx = g.nx + layer; gy = along; }
  else if (side == 2) { gx = along; gy = -1 - layer; }
  else { gx = along; gy = g.ny + layer; }
}

__global__ void k_dirichlet(double* __restrict__ f, Grid g, BState bs) {
  const int side = blockIdx.y;
  if (g.bc[side] != BC_DIRICHLET) return;
  const int len = side < 2 ? g.ny : g.nx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * len) return;
  int gx, gy, along;
  side_ghost(g, side, t, gx, gy, along);
  GhostOwn none;
  none.mx = 0;
  none.my = 0;
  write_feq(f, g, gx, gy, none, bs.s[side][0], bs.s[side][1], bs.s[side][2], bs.s[side][3]);
}

__global__ void k_segment(double* __restrict__ f, Grid g, Segment sg, double d) {
  const int len = sg.side < 2 ? g.ny : g.nx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * len) return;
  int gx, gy, along;
  side_ghost(g, sg.side, t, gx, gy, along);
  const double pos = mul(add((double)along, 0.5), d);
  const bool in = sg.lower ? (pos < sg.split) : !(pos < sg.split);
  if (!in && !sg.base_dirichlet) return;
  const double* st = in ? sg.seg : sg.base;
  GhostOwn none;
  none.mx = 0;
  none.my = 0;
  write_feq(f, g, gx, gy, none, st[0], st[1], st[2], st[3]);
}

__global__ void k_macro(const double* __restrict__ f, Grid g, double* __restrict__ rho, double* __restrict__ u,
                        double* __restrict__ v, double* __restrict__ T) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const Mac m = moments(f, g.plane, (long long)(gy + NG) * g.pitch + (gx + NG));
  const long long o = (long long)gy * g.nx + gx;
  rho[o] = m.n;
  u[o] = m.ux;
  v[o] = m.uy;
  T[o] = m.T;
}

}  // namespace strict
}  // namespace

cudaError_t launch_step_strict(const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                               cudaStream_t s) {
  if (!g.mom) return cudaErrorInvalidValue;
  strict::Params p;
  p.dt = c.sdt;
  p.tau = c.stau;
  p.dr[0] = c.sdr[0];
  p.dr[1] = c.sdr[1];
  p.lam = c.lam;
  p.flags = g.flags;
  dim3 mb(32, 4), mg((g.nx + 2 + 31) / 32, (g.ny + 2 + 3) / 4);
  strict::k_moments<<<mg, mb, 0, s>>>(static_cast<const double*>(f), g, health);
  dim3 ub(32, 4);
  strict::k_update<<<grid2d(g, ub), ub, 0, s>>>(static_cast<const double*>(f), static_cast<double*>(fn), g, p,
                                                health);
  return cudaGetLastError();
}

cudaError_t launch_init_strict(void* f, const Grid& g, const double* rho, const double* u, const double* v,
                               const double* T, cudaStream_t s) {
  dim3 b(32, 4);
  strict::k_init<<<grid2d(g, b), b, 0, s>>>(static_cast<double*>(f), g, rho, u, v, T);
  return cudaGetLastError();
}

cudaError_t launch_dirichlet_strict(void* f, const Grid& g, const double bstate[4][4], cudaStream_t s) {
  BState bs;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) bs.s[i][j] = bstate[i][j];
  const int len = 2 * (g.nx > g.ny ? g.nx : g.ny);
  dim3 b(128), grid((len + 127) / 128, 4);
  strict::k_dirichlet<<<grid, b, 0, s>>>(static_cast<double*>(f), g, bs);
  return cudaGetLastError();
}

cudaError_t launch_segment_strict(void* f, const Grid& g, const Segment& sg, double dx, double dy, cudaStream_t s) {
  const int len = sg.side < 2 ? g.ny : g.nx;
  dim3 b(128), grid((2 * len + 127) / 128);
  strict::k_segment<<<grid, b, 0, s>>>(static_cast<double*>(f), g, sg, sg.side < 2 ? dy : dx);
  return cudaGetLastError();
}

cudaError_t launch_macro_strict(const void* f, const Grid& g, double* rho, double* u, double* v, double* T,
                                cudaStream_t s) {
  dim3 b(32, 4);
  strict::k_macro<<<grid2d(g, b), b, 0, s>>>(static_cast<const double*>(f), g, rho, u, v, T);
  return cudaGetLastError();
}

}  // namespace fdlbm

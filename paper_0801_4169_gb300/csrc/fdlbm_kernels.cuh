#pragma once
// fdlbm_kernels.cuh -- sm_103a kernels of the FDLBM step (Gan, Xu, Zhang, Yu, Li, arXiv 0801.4169).
// Included by fdlbm_step_f64.cu / fdlbm_step_f32.cu (one precision each, compiled in parallel)
// and fdlbm_aux.cu (initial condition, boundary, moment and copy kernels).
//
// One fused kernel per time step computes, for every interior node of its tile:
//   moments n, u, T, P of Eqs. 3-5            (FP64, tile + 1-node ring, staged in shared memory)
//   switch theta_alphaI (Eq. 16), kappa (Eq. 15)
//   weights F_k(theta) (Eqs. 11-13) and f_eq (Eq. 10)        (FP64)
//   Eq. 17 for all 33 velocities, both axes, relaxation once  (storage precision)
// and writes f_new plus the ghost copies it owns (periodic wrap, zero-gradient copy, specular
// mirror), so the next step needs no separate boundary pass.
//
// On this GPU an FP64 instruction (including an FP32<->FP64 conversion) issues at ~1.6/clk/SM,
// ~73x below FP32, so the step is bound by the FP64 pipe, not by HBM. The code is arranged to
// issue as few FP64 operations per node as the method allows:
//   * ring moments from shared differences (S, X, Y per ring: 15 ops);
//   * f_eq by the even/odd split of each opposite-direction pair: with x = p^2,
//       nF_k E = alpha + x (beta + gamma x),  nF_k O = p (delta + eps x),  f_eq(+-) = nF_k (E +- O),
//     where (alpha..eps) are 5 per-ring constants (6 ops per pair);
//   * dt/tau folded into nF_k, so r*f_eq costs nothing extra;
//   * the Eq. 17 weights of the +-1 neighbours combined with the node's viscosity once per
//     (axis, |c| class, ring), shared by the 2-4 directions of that class.
#include "fdlbm_internal.h"

namespace fdlbm {

namespace {

constexpr double kS = 0.70710678118654752440;  // cos(pi/4)

__device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }

// FP32 <-> FP64 conversions issue on the (slow) FP64 pipe. For normal numbers both directions
// are done bit-exactly with integer operations instead; zero, subnormal, inf/nan and values
// outside the FP32 normal range take the hardware conversion.
//   up:   exponent += 1023 - 127, mantissa shifted left by 29 (exact).
//   down: round to nearest even on the 29 dropped mantissa bits (a carry into the exponent is
//         the correct rounding, up to +inf).
__device__ __forceinline__ bool f32_special(float x) {
  const unsigned a = __float_as_uint(x) & 0x7fffffffu;
  return a - 0x00800000u >= 0x7f000000u;  // a < 2^-126 (zero/subnormal) or inf/nan
}
__device__ __forceinline__ double f32_to_f64_bits(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + 0x38000000u);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ah = hi & 0x7fffffffu;
  if (ah - (897u << 20) >= (254u << 20)) return __double2float_rn(x);  // not an FP32 normal
  unsigned t = ((ah - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  t += (rem > 0x10000000u) | ((rem == 0x10000000u) & (t & 1u));
  return __uint_as_float(t | (hi & 0x80000000u));
}

// 1/x for x in the FP32 normal range: an FP32 seed (relative error e ~ 2^-23) refined by one
// third-order Newton step y (1 + e + e^2), e = 1 - x y, leaving O(e^3) ~ 2^-69: full FP64
// accuracy up to the last-bit rounding, in 3 FMAs. Outside that range: IEEE division.
__device__ __forceinline__ double rcp64(double x) {
  const unsigned ah = (unsigned)__double2hiint(x) & 0x7fffffffu;
  if (ah - (897u << 20) >= (252u << 20)) return 1.0 / x;
  const double y = f32_to_f64_bits(__frcp_rn(f64_to_f32_rn(x)));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// Health tests on the bits (integer pipe): finite, and finite with x > 0.
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}
__device__ __forceinline__ bool pos_finite_bits(double x) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  return hi >= 0 && hi < 0x7ff00000 && (hi | lo) != 0;
}

template <typename S>
__device__ __forceinline__ S from_d(double x);
template <>
__device__ __forceinline__ double from_d<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_d<float>(double x) { return f64_to_f32_rn(x); }

// ---------------------------------------------------------------------------------------------
// Velocity ordering (Eq. 1): q = 0 rest, q = 1 + 8k + d for ring k = 0..3 (speed v_{k+1}) and
// direction d = 0..7 at angle (d+1)*pi/4: d0 45, d1 90, d2 135, d3 180, d4 225, d5 270, d6 315,
// d7 0 degrees. Sign of c_x, c_y per direction (0: that component is zero):
__host__ __device__ constexpr int dir_xs(int d) { return (d == 0 || d == 6 || d == 7) ? 1 : (d == 2 || d == 3 || d == 4) ? -1 : 0; }
__host__ __device__ constexpr int dir_ys(int d) { return (d == 0 || d == 1 || d == 2) ? 1 : (d == 4 || d == 5 || d == 6) ? -1 : 0; }
// |c| class along the axis (0: axis-aligned direction, 1: diagonal)
__host__ __device__ constexpr int dir_cls(int d) { return (d == 1 || d == 3 || d == 5 || d == 7) ? 0 : 1; }
// centre class of line II (C2 index): 0 x-axis dirs, 1 y-axis dirs, 2 diagonals
__host__ __device__ constexpr int dir_c2(int d) { return (d == 3 || d == 7) ? 0 : (d == 1 || d == 5) ? 1 : 2; }
// specular mirrors: x-wall maps angle -> pi - angle, y-wall maps angle -> -angle
__host__ __device__ constexpr int mirror_x(int q) {
  return q == 0 ? 0 : 1 + 8 * ((q - 1) / 8) + ((((4 - (((q - 1) % 8) + 1)) % 8 + 8) % 8 + 7) % 8);
}
__host__ __device__ constexpr int mirror_y(int q) {
  return q == 0 ? 0 : 1 + 8 * ((q - 1) / 8) + ((((8 - (((q - 1) % 8) + 1)) % 8 + 8) % 8 + 7) % 8);
}
static_assert(mirror_x(1 + 7) == 1 + 3, "x-mirror maps 0 deg to 180 deg");
static_assert(mirror_x(1 + 0) == 1 + 2, "x-mirror maps 45 deg to 135 deg");
static_assert(mirror_x(1 + 1) == 1 + 1, "x-mirror keeps 90 deg");
static_assert(mirror_y(1 + 0) == 1 + 6, "y-mirror maps 45 deg to 315 deg");
static_assert(mirror_y(1 + 7) == 1 + 7, "y-mirror keeps 0 deg");
static_assert(mirror_y(1 + 1) == 1 + 5, "y-mirror maps 90 deg to 270 deg");

// ---------------------------------------------------------------------------------------------
// Ghost copies owned by an interior node (boundary kinds of Sec. 5.2; mechanics as documented in
// fdlbm.h). Ghost coordinate c in {-2, -1, n, n+1} copies interior node src(c).
__device__ __forceinline__ int ghost_src(int c, int n, int lo, int hi) {
  if (c < 0) {
    if (lo == BC_PERIODIC) return ((c % n) + n) % n;
    if (lo == BC_OUTFLOW) return 0;
    if (lo == BC_WALL) return -1 - c;
    return -1000;
  }
  if (hi == BC_PERIODIC) return c % n;
  if (hi == BC_OUTFLOW) return n - 1;
  if (hi == BC_WALL) return 2 * n - 1 - c;
  return -1000;
}
__device__ __forceinline__ unsigned ghost_mask(int i, int n, int lo, int hi) {
  unsigned m = 0;
  if (ghost_src(-2, n, lo, hi) == i) m |= 1u;
  if (ghost_src(-1, n, lo, hi) == i) m |= 2u;
  if (ghost_src(n, n, lo, hi) == i) m |= 4u;
  if (ghost_src(n + 1, n, lo, hi) == i) m |= 8u;
  return m;
}
__device__ __forceinline__ int ghost_coord(int t, int n) { return t < 2 ? t - 2 : n + (t - 2); }

struct GhostOwn {
  unsigned mx, my;  // 4-bit masks over ghost columns / rows
};

template <typename S, int QQ>
__device__ __forceinline__ void store_node(S* __restrict__ fn, const Grid& g, int gx, int gy, const GhostOwn& go,
                                           S val) {
  const long long base = (long long)QQ * g.plane;
  fn[base + (long long)(gy + NG) * g.pitch + (gx + NG)] = val;
  if (go.mx | go.my) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (go.mx & (1u << t)) {
        const int c = ghost_coord(t, g.nx);
        const bool wall = (c < 0 ? g.bc[0] : g.bc[1]) == BC_WALL;
        const int qq = wall ? mirror_x(QQ) : QQ;
        fn[(long long)qq * g.plane + (long long)(gy + NG) * g.pitch + (c + NG)] = val;
      }
      if (go.my & (1u << t)) {
        const int c = ghost_coord(t, g.ny);
        const bool wall = (c < 0 ? g.bc[2] : g.bc[3]) == BC_WALL;
        const int qq = wall ? mirror_y(QQ) : QQ;
        fn[(long long)qq * g.plane + (long long)(c + NG) * g.pitch + (gx + NG)] = val;
      }
    }
  }
}

// Store the 8 directions of ring K at an interior node, then the ghost copies it owns.
template <typename S, int K>
__device__ __forceinline__ void store_ring(S* __restrict__ fn, const Grid& g, int gx, int gy, const GhostOwn& go,
                                           const S (&v)[8]) {
  const long long node = (long long)(gy + NG) * g.pitch + (gx + NG);
#pragma unroll
  for (int d = 0; d < 8; ++d) fn[(long long)(1 + 8 * K + d) * g.plane + node] = v[d];
  if (go.mx | go.my) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (go.mx & (1u << t)) {
        const int c = ghost_coord(t, g.nx);
        const bool wall = (c < 0 ? g.bc[0] : g.bc[1]) == BC_WALL;
        const long long gn = (long long)(gy + NG) * g.pitch + (c + NG);
#pragma unroll
        for (int d = 0; d < 8; ++d) {
          const int q = 1 + 8 * K + d;
          fn[(long long)(wall ? mirror_x(q) : q) * g.plane + gn] = v[d];
        }
      }
      if (go.my & (1u << t)) {
        const int c = ghost_coord(t, g.ny);
        const bool wall = (c < 0 ? g.bc[2] : g.bc[3]) == BC_WALL;
        const long long gn = (long long)(c + NG) * g.pitch + (gx + NG);
#pragma unroll
        for (int d = 0; d < 8; ++d) {
          const int q = 1 + 8 * K + d;
          fn[(long long)(wall ? mirror_y(q) : q) * g.plane + gn] = v[d];
        }
      }
    }
  }
}

__device__ __forceinline__ GhostOwn ghost_own(const Grid& g, int gx, int gy) {
  GhostOwn go;
  go.mx = ghost_mask(gx, g.nx, g.bc[0], g.bc[1]);
  go.my = ghost_mask(gy, g.ny, g.bc[2], g.bc[3]);
  return go;
}

// ---------------------------------------------------------------------------------------------
// Moments of Eqs. 3-5 (FP64). One ring of 8 values g[d]:
//   S = sum g,  X = (g7 - g3) + s((g0 - g4) + (g6 - g2)),  Y = (g1 - g5) + s((g0 - g4) - (g6 - g2))
// with n += S, j_x += v X, j_y += v Y, sum |v|^2 f += v^2 S.
struct Mom {
  double n, jx, jy, e2;
};

__device__ __forceinline__ void ring_moments(const double g[8], double vk, double vk2, Mom& m) {
  const double S = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]));
  const double a = g[0] - g[4];
  const double b = g[6] - g[2];
  const double X = fma(kS, a + b, g[7] - g[3]);
  const double Y = fma(kS, a - b, g[1] - g[5]);
  m.n += S;
  m.jx = fma(vk, X, m.jx);
  m.jy = fma(vk, Y, m.jy);
  m.e2 = fma(vk2, S, m.e2);
}

__device__ __forceinline__ Mom node_moments(const double* __restrict__ f, long long plane, long long off,
                                            const Coeffs& c) {
  Mom m;
  m.n = ld(f + off);
  m.jx = 0.0;
  m.jy = 0.0;
  m.e2 = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double g[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) g[d] = ld(f + (long long)(1 + 8 * k + d) * plane + off);
    ring_moments(g, c.v[k], c.v2[k], m);
  }
  return m;
}

// FP32 storage: the 33 values are widened to FP64 exactly (integer path), then summed in FP64.
__device__ __forceinline__ Mom node_moments(const float* __restrict__ f, long long plane, long long off,
                                            const Coeffs& c) {
  float x[Q];
  bool special = false;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    x[q] = ld(f + (long long)q * plane + off);
    special |= f32_special(x[q]);
  }
  Mom m;
  m.jx = 0.0;
  m.jy = 0.0;
  m.e2 = 0.0;
  if (!special) {
    m.n = f32_to_f64_bits(x[0]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double g[8];
#pragma unroll
      for (int d = 0; d < 8; ++d) g[d] = f32_to_f64_bits(x[1 + 8 * k + d]);
      ring_moments(g, c.v[k], c.v2[k], m);
    }
  } else {
    m.n = (double)x[0];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double g[8];
#pragma unroll
      for (int d = 0; d < 8; ++d) g[d] = (double)x[1 + 8 * k + d];
      ring_moments(g, c.v[k], c.v2[k], m);
    }
  }
  return m;
}

// (n, ux, uy, T, P) from the sums; T = (sum |v|^2 f)/(2n) - |u|^2/2  (Eq. 5 with P = nT).
struct Macro {
  double n, ux, uy, T, P;
};
__device__ __forceinline__ Macro to_macro(const Mom& m) {
  Macro o;
  const double in = rcp64(m.n);
  o.n = m.n;
  o.ux = m.jx * in;
  o.uy = m.jy * in;
  const double u2 = fma(o.ux, o.ux, o.uy * o.uy);
  o.T = 0.5 * fma(m.e2, in, -u2);
  o.P = m.n * o.T;
  return o;
}

__device__ __forceinline__ bool macro_ok(const Macro& o) {
  // finite, n > 0, T > 0 (so P > 0 and the switch denominator of Eq. 16 is positive)
  return pos_finite_bits(o.n) && pos_finite_bits(o.T) && finite_bits(o.ux) && finite_bits(o.uy);
}

// ---------------------------------------------------------------------------------------------
// Equilibrium constants of one node (Eqs. 10-13), with dt/tau folded in (rn = r * n).
struct EqSite {
  double rn, A0, A1, A2;   // A0 = 1 - b + b^2/2, A1 = 1 - b, A2 = (1-b)/2, b = |u|^2/(2 theta)
  double p[4];             // projections (e.u)/theta for d = 7 (x), 0 (diag), 1 (y), 2 (anti-diag)
  double x[4];             // p^2
  double F[4];             // F_1..F_4
  double F0;
};

__device__ __forceinline__ EqSite eq_site(double n, double ux, double uy, double T, const Coeffs& c) {
  EqSite e;
  const double th = T;  // theta = T/m, m = 1
  const double ith = rcp64(th);
  const double px = ux * ith, py = uy * ith;
  e.p[0] = px;
  e.p[1] = kS * (px + py);
  e.p[2] = py;
  e.p[3] = kS * (py - px);
#pragma unroll
  for (int t = 0; t < 4; ++t) e.x[t] = e.p[t] * e.p[t];
  const double b = 0.5 * fma(ux, ux, uy * uy) * ith;
  e.A1 = 1.0 - b;
  e.A0 = fma(0.5 * b, b, e.A1);
  e.A2 = 0.5 * e.A1;
  double sF = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    e.F[k] = th * fma(th, fma(th, fma(th, c.Fh[k][3], c.Fh[k][2]), c.Fh[k][1]), c.Fh[k][0]);
    sF += e.F[k];
  }
  e.F0 = fma(-8.0, sF, 1.0);
  e.rn = c.r * n;
  return e;
}

// Per-ring constants alpha..eps (times r n F_k).
struct EqRing {
  double al, be, ga, de, ep;
};
__device__ __forceinline__ EqRing eq_ring(const EqSite& e, int k, const Coeffs& c) {
  EqRing r;
  const double nF = e.rn * e.F[k];
  r.al = nF * e.A0;
  r.be = nF * (e.A2 * c.v2[k]);
  r.ga = nF * c.v4_24[k];
  r.de = nF * (e.A1 * c.v[k]);
  r.ep = nF * c.v3_6[k];
  return r;
}
// r f_eq for the direction with projection p and its opposite, from the even part
// NE = alpha + x (beta + gamma x) and the odd part NO = p (delta + eps x), both in FP64. The
// FP64 path forms NE +- NO in FP64; the FP32-storage path rounds NE and NO to FP32 and forms
// the pair there, the precision the sum is stored in.
__device__ __forceinline__ void eq_parts(const EqRing& r, double p, double x, double& NE, double& NO) {
  NE = fma(x, fma(r.ga, x, r.be), r.al);
  NO = p * fma(r.ep, x, r.de);
}
__device__ __forceinline__ void eq_pair(const EqRing& r, double p, double x, double& fp, double& fm) {
  double NE, NO;
  eq_parts(r, p, x, NE, NO);
  fp = NE + NO;
  fm = NE - NO;
}
template <typename S>
__device__ __forceinline__ void eq_pair_s(const EqRing& r, double p, double x, S& fp, S& fm);
template <>
__device__ __forceinline__ void eq_pair_s<double>(const EqRing& r, double p, double x, double& fp, double& fm) {
  eq_pair(r, p, x, fp, fm);
}
template <>
__device__ __forceinline__ void eq_pair_s<float>(const EqRing& r, double p, double x, float& fp, float& fm) {
  double NE, NO;
  eq_parts(r, p, x, NE, NO);
  const float e = f64_to_f32_rn(NE), o = f64_to_f32_rn(NO);
  fp = e + o;
  fm = e - o;
}

// ---------------------------------------------------------------------------------------------
// Stencil of Eq. 17 for one velocity (storage precision S):
//   f_new = W0 f_I + r f_eq + sum_alpha [ W+ f_{I+1} + W- f_{I-1} + D (f_{I+2} - f_{I-2}) ]
// W0 = 1 - r - sum_alpha (c_alpha^2 [line II] + 2 nu_alpha [line IV]),
// W+ = -c/2 + c^2/2 - 2d + nu, W- = c/2 + c^2/2 + 2d + nu, D = d = c(1-c^2)/12,
// nu_alpha = theta_alphaI |kappa_alpha| (1 - |kappa_alpha|) / 2.
template <typename S>
struct RingW {
  S w0[3];          // centre weight per C2 class
  S P1[2][2];       // W+ for (axis, class), positive-c direction
  S M1[2][2];       // W-
  S Dd[2][2];       // D
  S nu[2];
};

template <typename S, int D>
__device__ __forceinline__ S stencil_dir(const S* __restrict__ p, int pitch, const RingW<S>& w, S rfeq) {
  constexpr int XS = dir_xs(D), YS = dir_ys(D), CL = dir_cls(D), CC = dir_c2(D);
  S acc = fma(w.w0[CC], ld(p), rfeq);
  if (XS == 0) {
    acc = fma(w.nu[0], ld(p + 1) + ld(p - 1), acc);
  } else {
    const S cp = XS > 0 ? w.P1[0][CL] : w.M1[0][CL];
    const S cm = XS > 0 ? w.M1[0][CL] : w.P1[0][CL];
    acc = fma(cp, ld(p + 1), acc);
    acc = fma(cm, ld(p - 1), acc);
    const S d2 = ld(p + 2) - ld(p - 2);
    acc = XS > 0 ? fma(w.Dd[0][CL], d2, acc) : fma(-w.Dd[0][CL], d2, acc);
  }
  if (YS == 0) {
    acc = fma(w.nu[1], ld(p + pitch) + ld(p - pitch), acc);
  } else {
    const S cp = YS > 0 ? w.P1[1][CL] : w.M1[1][CL];
    const S cm = YS > 0 ? w.M1[1][CL] : w.P1[1][CL];
    acc = fma(cp, ld(p + pitch), acc);
    acc = fma(cm, ld(p - pitch), acc);
    const S d2 = ld(p + 2 * pitch) - ld(p - 2 * pitch);
    acc = YS > 0 ? fma(w.Dd[1][CL], d2, acc) : fma(-w.Dd[1][CL], d2, acc);
  }
  return acc;
}

template <typename S>
struct StencilConsts;
template <>
struct StencilConsts<double> {
  __device__ static double W1(const Coeffs& c, int a, int k, int l) { return c.W1[a][k][l]; }
  __device__ static double Wm1(const Coeffs& c, int a, int k, int l) { return c.Wm1[a][k][l]; }
  __device__ static double D(const Coeffs& c, int a, int k, int l) { return c.D[a][k][l]; }
  __device__ static double C2(const Coeffs& c, int k, int l) { return c.C2[k][l]; }
  __device__ static double r(const Coeffs& c) { return c.r; }
  __device__ static double kx(const Coeffs& c) { return c.kx; }
  __device__ static double ky(const Coeffs& c) { return c.ky; }
  __device__ static double lam(const Coeffs& c) { return c.lam; }
};
template <>
struct StencilConsts<float> {
  __device__ static float W1(const Coeffs& c, int a, int k, int l) { return c.fW1[a][k][l]; }
  __device__ static float Wm1(const Coeffs& c, int a, int k, int l) { return c.fWm1[a][k][l]; }
  __device__ static float D(const Coeffs& c, int a, int k, int l) { return c.fD[a][k][l]; }
  __device__ static float C2(const Coeffs& c, int k, int l) { return c.fC2[k][l]; }
  __device__ static float r(const Coeffs& c) { return c.fr; }
  __device__ static float kx(const Coeffs& c) { return c.fkx; }
  __device__ static float ky(const Coeffs& c) { return c.fky; }
  __device__ static float lam(const Coeffs& c) { return c.flam; }
};

// Update of all 33 velocities at one interior node, given its moments and nu_x, nu_y.
template <typename S, int K>
__device__ __forceinline__ void update_ring(const S* __restrict__ f, S* __restrict__ fn, const Grid& g,
                                            const Coeffs& c, long long off, int gx, int gy, const GhostOwn& go,
                                            const EqSite& e, S w0base, S nux, S nuy) {
  using SC = StencilConsts<S>;
  RingW<S> w;
#pragma unroll
  for (int l = 0; l < 3; ++l) w.w0[l] = w0base - SC::C2(c, K, l);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const S nu = a == 0 ? nux : nuy;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      w.P1[a][l] = SC::W1(c, a, K, l) + nu;
      w.M1[a][l] = SC::Wm1(c, a, K, l) + nu;
      w.Dd[a][l] = SC::D(c, a, K, l);
    }
  }
  w.nu[0] = nux;
  w.nu[1] = nuy;
  const EqRing er = eq_ring(e, K, c);
  const S* fq = f + off;
  // All 8 directions of the ring are computed before any store, so the ring is one basic block
  // the compiler can interleave (the ghost-copy branch comes once per ring, not per velocity).
  S out[8], fp, fm;
  // pair (d7: 0 deg, d3: 180 deg), projection p_x
  eq_pair_s<S>(er, e.p[0], e.x[0], fp, fm);
  out[7] = stencil_dir<S, 7>(fq + (long long)(1 + 8 * K + 7) * g.plane, g.pitch, w, fp);
  out[3] = stencil_dir<S, 3>(fq + (long long)(1 + 8 * K + 3) * g.plane, g.pitch, w, fm);
  // pair (d0: 45 deg, d4: 225 deg), projection s(p_x + p_y)
  eq_pair_s<S>(er, e.p[1], e.x[1], fp, fm);
  out[0] = stencil_dir<S, 0>(fq + (long long)(1 + 8 * K + 0) * g.plane, g.pitch, w, fp);
  out[4] = stencil_dir<S, 4>(fq + (long long)(1 + 8 * K + 4) * g.plane, g.pitch, w, fm);
  // pair (d1: 90 deg, d5: 270 deg), projection p_y
  eq_pair_s<S>(er, e.p[2], e.x[2], fp, fm);
  out[1] = stencil_dir<S, 1>(fq + (long long)(1 + 8 * K + 1) * g.plane, g.pitch, w, fp);
  out[5] = stencil_dir<S, 5>(fq + (long long)(1 + 8 * K + 5) * g.plane, g.pitch, w, fm);
  // pair (d2: 135 deg, d6: 315 deg), projection s(p_y - p_x)
  eq_pair_s<S>(er, e.p[3], e.x[3], fp, fm);
  out[2] = stencil_dir<S, 2>(fq + (long long)(1 + 8 * K + 2) * g.plane, g.pitch, w, fp);
  out[6] = stencil_dir<S, 6>(fq + (long long)(1 + 8 * K + 6) * g.plane, g.pitch, w, fm);
  store_ring<S, K>(fn, g, gx, gy, go, out);
}

template <typename S>
__device__ __forceinline__ S to_s(double x) { return from_d<S>(x); }

__device__ __forceinline__ double recip(double x) { return rcp64(x); }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// ---------------------------------------------------------------------------------------------
// The fused step. CTA = BX x BY threads; tile TW x TH = BX x (BY*RY) nodes. Shared memory holds
// n, ux, uy, T, P of the tile and its 1-node ring (corners excluded), computed once per node.
// One tile (tx, ty) of one solve: the body shared by the single-solve kernel (k_step) and the
// batched kernel (k_step_batch), so a node's arithmetic is the same alone and in a batch.
template <typename S, int BX, int BY, int RY>
__device__ __forceinline__ void step_tile(const S* __restrict__ f, S* __restrict__ fn, const Grid& g, const Coeffs& c,
                                          unsigned* __restrict__ health, int tx, int ty) {
  constexpr int TW = BX, TH = BY * RY, SW = TW + 2, SH = TH + 2, NT = BX * BY;
  using SC = StencilConsts<S>;
  // P is staged in the storage precision: the switch of Eq. 16 is a limiter coefficient, and in
  // the FP32-storage path it is evaluated in FP32 like the rest of the stencil weights.
  __shared__ double s_n[SH][SW], s_ux[SH][SW], s_uy[SH][SW], s_T[SH][SW];
  __shared__ S s_P[SH][SW];
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int x0 = tx * TW, y0 = ty * TH;
  unsigned bits = 0;

  // Phase 1: moments on the tile and its ring (needed: interior nodes and the ghost layer next
  // to an edge, never the corners).
  for (int idx = tid; idx < SW * SH; idx += NT) {
    const int lx = idx % SW, ly = idx / SW;
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    const bool inx = gx >= 0 && gx < g.nx, iny = gy >= 0 && gy < g.ny;
    const bool need = (inx && iny) || (iny && (gx == -1 || gx == g.nx)) || (inx && (gy == -1 || gy == g.ny));
    if (!need) continue;
    const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
    const Macro m = to_macro(node_moments(f, g.plane, off, c));
    if (!macro_ok(m)) bits |= H_NUMERIC;
    s_n[ly][lx] = m.n;
    s_ux[ly][lx] = m.ux;
    s_uy[ly][lx] = m.uy;
    s_T[ly][lx] = m.T;
    s_P[ly][lx] = from_d<S>(m.P);
  }
  __syncthreads();

  // Phase 2: Eq. 17 at the tile's interior nodes.
#pragma unroll 1
  for (int rr = 0; rr < RY; ++rr) {
    const int lx = threadIdx.x + 1, ly = threadIdx.y + rr * BY + 1;
    const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y + rr * BY;
    if (gx >= g.nx || gy >= g.ny) continue;
    const double n = s_n[ly][lx], ux = s_ux[ly][lx], uy = s_uy[ly][lx], T = s_T[ly][lx];
    // switch of Eq. 16 and kappa of Eq. 15 (storage precision)
    S thx, thy;
    if (g.flags & F_SWITCH_CONST) {
      thx = SC::lam(c);
      thy = SC::lam(c);
    } else {
      const S P0 = s_P[ly][lx];
      const S sx = s_P[ly][lx + 1] + s_P[ly][lx - 1], sy = s_P[ly + 1][lx] + s_P[ly - 1][lx];
      thx = SC::lam(c) * fabs(fma((S)-2, P0, sx) * recip(fma((S)2, P0, sx)));
      thy = SC::lam(c) * fabs(fma((S)-2, P0, sy) * recip(fma((S)2, P0, sy)));
    }
    const S akx = fabs(from_d<S>(ux) * SC::kx(c)), aky = fabs(from_d<S>(uy) * SC::ky(c));
    if (akx > (S)1 || aky > (S)1) bits |= H_KAPPA;
    S snux = 0, snuy = 0;
    if (!(g.flags & F_NO_VISC)) {
      snux = (S)0.5 * thx * akx * ((S)1 - akx);
      snuy = (S)0.5 * thy * aky * ((S)1 - aky);
    }
    const S w0base = ((S)1 - SC::r(c)) - (S)2 * (snux + snuy);
    const EqSite e = eq_site(n, ux, uy, T, c);
    const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
    const GhostOwn go = ghost_own(g, gx, gy);
    // rest velocity: f_eq = n F_0 A0; c = 0 on both axes (line IV only)
    {
      const S rfeq = to_s<S>(e.rn * e.F0 * e.A0);
      const S* p = f + off;
      S acc = fma(w0base, ld(p), rfeq);
      acc = fma(snux, ld(p + 1) + ld(p - 1), acc);
      acc = fma(snuy, ld(p + g.pitch) + ld(p - g.pitch), acc);
      store_node<S, 0>(fn, g, gx, gy, go, acc);
    }
    update_ring<S, 0>(f, fn, g, c, off, gx, gy, go, e, w0base, snux, snuy);
    update_ring<S, 1>(f, fn, g, c, off, gx, gy, go, e, w0base, snux, snuy);
    update_ring<S, 2>(f, fn, g, c, off, gx, gy, go, e, w0base, snux, snuy);
    update_ring<S, 3>(f, fn, g, c, off, gx, gy, go, e, w0base, snux, snuy);
  }
  if (bits) atomicOr(health, bits);
}

template <typename S, int BX, int BY, int RY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB) k_step(const S* __restrict__ f, S* __restrict__ fn, Grid g, Coeffs c,
                                                  unsigned* __restrict__ health) {
  step_tile<S, BX, BY, RY>(f, fn, g, c, health, blockIdx.x, blockIdx.y);
}

// Batched step: every member solve of a batch advances one time step in one launch. Members share
// the scheme constants (dx, dy, dt, tau, lambda, flags, precision), not their grids, boundaries or
// buffers. Block b runs tile (b - tile0) of the member whose [tile0, tile0 + tiles) holds b.
template <typename S, int BX, int BY, int RY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB) k_step_batch(const BatchMember* __restrict__ mem, int nmem,
                                                        unsigned long long step, Coeffs c) {
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
  const S* in = static_cast<const S*>(m.f[par]);
  S* out = static_cast<S*>(m.f[par ^ 1]);
  step_tile<S, BX, BY, RY>(in, out, g, c, m.health, tx, ty);
}

// health words of the members into one array (one device-to-host copy per batch round)
__global__ void k_gather_health(const BatchMember* __restrict__ mem, int nmem, unsigned* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nmem) out[i] = *mem[i].health;
}

// ---------------------------------------------------------------------------------------------
// f = f_eq(macros) at interior nodes (+ owned ghost copies): the initial condition (Eq. 10).
template <typename S, int K>
__device__ __forceinline__ void init_ring(S* __restrict__ f, const Grid& g, const Coeffs& c, int gx, int gy,
                                          const GhostOwn& go, const EqSite& e) {
  const EqRing er = eq_ring(e, K, c);
  double fp, fm;
  eq_pair(er, e.p[0], e.x[0], fp, fm);
  store_node<S, 1 + 8 * K + 7>(f, g, gx, gy, go, from_d<S>(fp));
  store_node<S, 1 + 8 * K + 3>(f, g, gx, gy, go, from_d<S>(fm));
  eq_pair(er, e.p[1], e.x[1], fp, fm);
  store_node<S, 1 + 8 * K + 0>(f, g, gx, gy, go, from_d<S>(fp));
  store_node<S, 1 + 8 * K + 4>(f, g, gx, gy, go, from_d<S>(fm));
  eq_pair(er, e.p[2], e.x[2], fp, fm);
  store_node<S, 1 + 8 * K + 1>(f, g, gx, gy, go, from_d<S>(fp));
  store_node<S, 1 + 8 * K + 5>(f, g, gx, gy, go, from_d<S>(fm));
  eq_pair(er, e.p[3], e.x[3], fp, fm);
  store_node<S, 1 + 8 * K + 2>(f, g, gx, gy, go, from_d<S>(fp));
  store_node<S, 1 + 8 * K + 6>(f, g, gx, gy, go, from_d<S>(fm));
}

template <typename S>
__device__ __forceinline__ void write_feq(S* __restrict__ f, const Grid& g, const Coeffs& cr, int gx, int gy,
                                          const GhostOwn& go, double n, double ux, double uy, double T) {
  Coeffs c = cr;
  c.r = 1.0;  // plain f_eq (no dt/tau factor)
  const EqSite e = eq_site(n, ux, uy, T, c);
  store_node<S, 0>(f, g, gx, gy, go, from_d<S>(e.rn * e.F0 * e.A0));
  init_ring<S, 0>(f, g, c, gx, gy, go, e);
  init_ring<S, 1>(f, g, c, gx, gy, go, e);
  init_ring<S, 2>(f, g, c, gx, gy, go, e);
  init_ring<S, 3>(f, g, c, gx, gy, go, e);
}

template <typename S>
__global__ void k_init(S* __restrict__ f, Grid g, Coeffs c, const double* __restrict__ rho,
                       const double* __restrict__ u, const double* __restrict__ v, const double* __restrict__ T) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const long long m = (long long)gy * g.nx + gx;
  write_feq<S>(f, g, c, gx, gy, ghost_own(g, gx, gy), rho[m], u[m], v[m], T[m]);
}

// Dirichlet ghosts: f_eq of the side's prescribed state at every ghost node of that side next to
// the interior (the two ghost columns on interior rows, or the two ghost rows on interior columns).
struct BState {
  double s[4][4];
};
template <typename S>
__global__ void k_dirichlet(S* __restrict__ f, Grid g, Coeffs c, BState bs) {
  const int side = blockIdx.y;
  if (g.bc[side] != BC_DIRICHLET) return;
  const int len = side < 2 ? g.ny : g.nx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * len) return;
  const int along = t % len, layer = t / len;  // layer 0: next to the interior, 1: outer
  int gx, gy;
  if (side == 0) { gx = -1 - layer; gy = along; }
  else if (side == 1) { gx = g.nx + layer; gy = along; }
  else if (side == 2) { gx = along; gy = -1 - layer; }
  else { gx = along; gy = g.ny + layer; }
  GhostOwn none;
  none.mx = 0;
  none.my = 0;
  write_feq<S>(f, g, c, gx, gy, none, bs.s[side][0], bs.s[side][1], bs.s[side][2], bs.s[side][3]);
}

// Moments of the interior (Eqs. 3-5) into FP64 arrays, x fastest.
template <typename S>
__global__ void k_macro(const S* __restrict__ f, Grid g, Coeffs c, double* __restrict__ rho, double* __restrict__ u,
                        double* __restrict__ v, double* __restrict__ T) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  const Macro m = to_macro(node_moments(f, g.plane, off, c));
  const long long o = (long long)gy * g.nx + gx;
  rho[o] = m.n;
  u[o] = m.ux;
  v[o] = m.uy;
  T[o] = m.T;
}

template <typename S>
__global__ void k_get_f(const S* __restrict__ f, Grid g, double* __restrict__ out) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  for (int q = 0; q < Q; ++q) out[((long long)q * g.ny + gy) * g.nx + gx] = to_d(f[(long long)q * g.plane + off]);
}

template <typename S>
__global__ void k_get_region(const S* __restrict__ f, Grid g, int x0, int y0, int w, int h, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= w || j >= h) return;
  const long long off = (long long)(y0 + j + NG) * g.pitch + (x0 + i + NG);
  for (int q = 0; q < Q; ++q) out[((long long)q * h + j) * w + i] = to_d(f[(long long)q * g.plane + off]);
}

template <typename S, int QQ>
__device__ __forceinline__ void set_one(S* f, const Grid& g, int gx, int gy, const GhostOwn& go, const double* in) {
  store_node<S, QQ>(f, g, gx, gy, go, from_d<S>(in[((long long)QQ * g.ny + gy) * g.nx + gx]));
}
template <typename S, int... QS>
__device__ __forceinline__ void set_all(S* f, const Grid& g, int gx, int gy, const GhostOwn& go, const double* in) {
  (set_one<S, QS>(f, g, gx, gy, go, in), ...);
}
template <typename S>
__global__ void k_set_f(S* __restrict__ f, Grid g, const double* __restrict__ in) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const GhostOwn go = ghost_own(g, gx, gy);
  set_all<S, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28,
          29, 30, 31, 32>(f, g, gx, gy, go, in);
}

// MINB: CTAs per SM the register allocation must allow (1 = no cap, 2 or 4 = <= 128 registers).
template <typename S, int BX, int BY, int RY, int MINB>
cudaError_t launch_step_t(const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                          cudaStream_t s) {
  dim3 block(BX, BY);
  dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY * RY - 1) / (BY * RY));
  k_step<S, BX, BY, RY, MINB><<<grid, block, 0, s>>>(static_cast<const S*>(f), static_cast<S*>(fn), g, c, health);
  return cudaGetLastError();
}

template <typename S, int BX, int BY, int RY, int MINB>
cudaError_t launch_batch_t(const BatchMember* mem, int nmem, long long tiles, unsigned long long step, const Coeffs& c,
                           cudaStream_t s) {
  k_step_batch<S, BX, BY, RY, MINB><<<dim3((unsigned)tiles), dim3(BX, BY), 0, s>>>(mem, nmem, step, c);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_batch_v(int variant, const BatchMember* mem, int nmem, long long tiles, unsigned long long step,
                           const Coeffs& c, cudaStream_t s) {
  switch (variant) {
    case V_T32x4: return launch_batch_t<S, 32, 4, 1, 4>(mem, nmem, tiles, step, c, s);
    case V_T32x8: return launch_batch_t<S, 32, 4, 2, 4>(mem, nmem, tiles, step, c, s);
    case V_T32x16: return launch_batch_t<S, 32, 8, 2, 2>(mem, nmem, tiles, step, c, s);
    case V_T16x4: return launch_batch_t<S, 16, 4, 1, 1>(mem, nmem, tiles, step, c, s);
    case V_T64x8: return launch_batch_t<S, 64, 4, 2, 2>(mem, nmem, tiles, step, c, s);
    case V_T32x32: return launch_batch_t<S, 32, 8, 4, 2>(mem, nmem, tiles, step, c, s);
    case V_T32x16_R: return launch_batch_t<S, 32, 8, 2, 1>(mem, nmem, tiles, step, c, s);
    case V_T32x32_R: return launch_batch_t<S, 32, 8, 4, 1>(mem, nmem, tiles, step, c, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename S>
cudaError_t launch_step_v(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                          cudaStream_t s) {
  switch (variant) {
    case V_T32x4: return launch_step_t<S, 32, 4, 1, 4>(f, fn, g, c, health, s);
    case V_T32x8: return launch_step_t<S, 32, 4, 2, 4>(f, fn, g, c, health, s);
    case V_T32x16: return launch_step_t<S, 32, 8, 2, 2>(f, fn, g, c, health, s);
    case V_T16x4: return launch_step_t<S, 16, 4, 1, 1>(f, fn, g, c, health, s);
    case V_T64x8: return launch_step_t<S, 64, 4, 2, 2>(f, fn, g, c, health, s);
    case V_T32x32: return launch_step_t<S, 32, 8, 4, 2>(f, fn, g, c, health, s);
    case V_T32x16_R: return launch_step_t<S, 32, 8, 2, 1>(f, fn, g, c, health, s);
    case V_T32x32_R: return launch_step_t<S, 32, 8, 4, 1>(f, fn, g, c, health, s);
    default: return cudaErrorInvalidValue;
  }
}

inline dim3 grid2d(const Grid& g, dim3 b) { return dim3((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y); }

}  // namespace
}  // namespace fdlbm

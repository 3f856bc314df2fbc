#pragma once
// fdlbm_kernels.cuh -- sm_103a kernels of the FDLBM step (Gan, Xu, Zhang, Yu, Li, arXiv 0801.4169).
// Included by fdlbm_step_f64.cu / fdlbm_step_f32.cu (one precision each, compiled in parallel),
// fdlbm_step_wrap_*.cu (tiles that hold a periodic grid's height) and fdlbm_aux.cu (initial
// condition, boundary, moment and copy kernels).
//
// One fused kernel per time step computes, for every interior node of its tile:
//   moments n, u, T, P of Eqs. 3-5            (tile + 1-node ring, staged in shared memory; FP64
//                                              sums, or exact fixed-point sums for FP32 storage)
//   switch theta_alphaI (Eq. 16), kappa (Eq. 15)
//   weights F_k(theta) (Eqs. 11-13) and f_eq (Eq. 10)        (FP64)
//   Eq. 17 for all 33 velocities, both axes, relaxation once  (storage precision)
// and writes f_new plus the ghost copies it owns (periodic wrap, zero-gradient copy, specular
// mirror), so the next step needs no separate boundary pass. With FP32 storage the 32 x 16 and
// 64 x 8 tiles stage the f_eq of all their nodes in shared memory first and run the stencils after
// (STAGE), so that each warp's FP64 work comes in one dense stretch.
//
// On this GPU an FP64 instruction (including an FP32<->FP64 conversion) issues at 2/clk/SM, ~64x
// below FP32, so the step is bound by the FP64 pipe, not by HBM. The code is arranged to issue as
// few FP64 operations per node as the method allows:
//   * ring moments from shared differences (S, X, Y per ring: 15 ops with FP64 storage); with
//     FP32 storage the ring, speed-weighted momentum and energy sums are exact 64-bit integers,
//     and only sqrt(1/2), the two energy parts' sum and 1/100, 10^-4 are applied in FP64;
//   * f_eq by the even/odd split of each opposite-direction pair: with x = p^2,
//       nF_k E = alpha + x (beta + gamma x),  nF_k O = p (delta + eps x),  f_eq(+-) = nF_k (E +- O),
//     where (alpha..eps) are 5 per-ring constants (6 ops per ring, 4 per pair);
//   * dt/tau and n folded into the weights' polynomials, so r*f_eq costs nothing extra;
//   * the Eq. 17 weights of the +-1 neighbours combined with the node's viscosity once per
//     (axis, |c| class, ring), shared by the 2-4 directions of that class.
#include <atomic>
#include <type_traits>

#include "fdlbm_internal.h"

namespace fdlbm {

namespace {

constexpr double kS = 0.70710678118654752440;  // cos(pi/4)

__device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
// COH: a load that stays coherent with stores other CTAs made earlier in the same launch, for the
// persistent kernels, whose steps read what the previous step wrote. It is cached in L2 only (the
// point of coherence): an L1 line of the buffer from two steps back would be stale, and the
// read-only path of __ldg is only valid for data that no thread of the launch writes.
template <bool COH, typename T>
__device__ __forceinline__ T ldc(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }

// FP32 <-> FP64 conversions issue on the (slow) FP64 pipe, so both directions are done bit-exactly
// with integer operations instead, from the IEEE-754 formats:
//   up (normal FP32 values only): exponent += 1023 - 127, significand shifted left by 29 (exact).
//   down: round to nearest even on the 29 dropped significand bits (a carry into the exponent is
//         the correct rounding, up to +inf). Values below 2^-126 round to the subnormal grid
//         2^-149, values from 2^128 up become inf, and NaN stays NaN.
// The rare cases are integer code in a function that is not inlined, behind a branch: a hardware
// conversion, or an inlined rare path, under a predicate would still issue with every call.
__device__ __forceinline__ double f32_to_f64_bits(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + 0x38000000u);
  return __hiloint2double((int)hi, (int)(u << 29));
}
// |x| in [2^-126, 2^128) from its FP64 bits without the sign (ah: high word, lo: low word)
__device__ __forceinline__ unsigned f64_to_f32_normal(unsigned ah, unsigned lo) {
  const unsigned t = ((ah - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  return t + ((rem > 0x10000000u) | ((rem == 0x10000000u) & (t & 1u)));
}
// |x| outside [2^-126, 2^128): NaN, inf, or an FP32 subnormal or zero
__device__ __noinline__ unsigned f64_to_f32_rare(unsigned ah, unsigned lo) {
  if (ah >= 0x7ff00000u) return (ah > 0x7ff00000u || lo != 0u) ? 0x7fc00000u : 0x7f800000u;
  if (ah >= (1151u << 20)) return 0x7f800000u;
  // below 2^-126: the significand m has unit 2^(E-1075) (E the biased exponent, 1 for FP64
  // subnormals) and the result unit 2^-149, so the result is m 2^-sh rounded, sh = 926 - E >= 30
  const unsigned E = ah >> 20;
  const unsigned sh = 926u - (E ? E : 1u);
  if (sh >= 64u) return 0u;  // m < 2^53: below half the result unit
  const unsigned long long m = ((unsigned long long)((ah & 0xfffffu) | (E ? 0x100000u : 0u)) << 32) | lo;
  const unsigned long long q = m >> sh, r = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1u);
  return (unsigned)q + (unsigned)((r > half) | ((r == half) & (q & 1ull)));  // a carry gives 2^-126
}
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ah = hi & 0x7fffffffu;
  unsigned t;
  if (__builtin_expect(ah - (897u << 20) < (254u << 20), 1)) t = f64_to_f32_normal(ah, lo);
  else t = f64_to_f32_rare(ah, lo);
  return __uint_as_float(t | (hi & 0x80000000u));
}

// 1/x for x in the FP32 normal range: an FP32 seed (relative error e ~ 2^-23) refined by one
// third-order Newton step y (1 + e + e^2), e = 1 - x y, leaving O(e^3) ~ 2^-69: full FP64
// accuracy up to the last-bit rounding, in 3 FMAs. Outside that range: IEEE division, in a
// function that is not inlined, so that its FP64 instructions never issue under a predicate.
__device__ __noinline__ double rcp64_rare(double x) { return 1.0 / x; }
__device__ __forceinline__ double rcp64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), ah = hi & 0x7fffffffu;
  if (__builtin_expect(ah - (897u << 20) >= (252u << 20), 0)) return rcp64_rare(x);
  const float xs = __uint_as_float(f64_to_f32_normal(ah, (unsigned)__double2loint(x)) | (hi & 0x80000000u));
  const double y = f32_to_f64_bits(__frcp_rn(xs));
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
template <typename S>
__device__ __forceinline__ void store_ring(S* __restrict__ fn, const Grid& g, int gx, int gy, const GhostOwn& go, int K,
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
//   S = sum g,  X = (g7 - g3) + s((g0 - g4) + (g6 - g2)),  Y = (g1 - g5) + s((g0 - g4) - (g6 - g2)),
// and the rings combine pairwise, (ring 0 + ring 1) + (ring 2 + ring 3):
//   n  = ((f_0 + S_0) + S_1) + (S_2 + S_3)
//   jx = fma(v_0, X_0, v_1 X_1) + fma(v_2, X_2, v_3 X_3)      (jy with Y; sum |v|^2 f with v^2, S)
// The tree is fixed so that the ring-parallel kernel, whose four lanes hold one ring each, forms
// exactly the same sums with two shuffle stages as the kernels that hold all rings in one thread.
struct Mom {
  double n, jx, jy, e2;
};

__device__ __forceinline__ void ring_sums(const double g[8], double& S, double& X, double& Y) {
  S = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]));
  const double a = g[0] - g[4];
  const double b = g[6] - g[2];
  X = fma(kS, a + b, g[7] - g[3]);
  Y = fma(kS, a - b, g[1] - g[5]);
}

__device__ __forceinline__ double pair_dot(double va, double xa, double vb, double xb) { return fma(va, xa, vb * xb); }

__device__ __forceinline__ Mom combine_rings(double f0, const double S[4], const double X[4], const double Y[4],
                                             const Coeffs& c) {
  Mom m;
  m.n = ((f0 + S[0]) + S[1]) + (S[2] + S[3]);
  m.jx = pair_dot(c.v[0], X[0], c.v[1], X[1]) + pair_dot(c.v[2], X[2], c.v[3], X[3]);
  m.jy = pair_dot(c.v[0], Y[0], c.v[1], Y[1]) + pair_dot(c.v[2], Y[2], c.v[3], Y[3]);
  m.e2 = pair_dot(c.v2[0], S[0], c.v2[1], S[1]) + pair_dot(c.v2[2], S[2], c.v2[3], S[3]);
  return m;
}

template <bool COH = false>
__device__ __forceinline__ Mom node_moments(const double* __restrict__ f, long long plane, long long off,
                                            const Coeffs& c) {
  double S[4], X[4], Y[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double g[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) g[d] = ldc<COH>(f + (long long)(1 + 8 * k + d) * plane + off);
    ring_sums(g, S[k], X[k], Y[k]);
  }
  return combine_rings(ldc<COH>(f + off), S, X, Y, c);
}

// FP32 storage: the moments are summed exactly in 64-bit fixed point on the integer pipes, which
// replaces ~75 of the ~80 FP64 operations of the FP64 summation.
//  - Scale: with e* the largest biased exponent of the node's 33 values (subnormals count as 1), a
//    value x = +-m 2^(e-150) (m its 24-bit significand) enters as the integer +-m 2^(26-e*+e): the
//    largest value's top bit lands on bit 49. A term more than 2^26 below the largest has its
//    significand shifted right (arithmetic shift, rounding towards -inf) and loses the bits under
//    the unit, less than 2^-49 of the largest value per term (the FP32 values themselves carry
//    2^-24). Every sum below stays under 2^63 (the speed-weighted ones under 1040 * 4 * 2^50).
//  - Each term is one 32 x 32 -> 64-bit multiply-add of the signed significand by a power of two,
//    accumulated straight into the ring sums (the multiply-add runs on the FMA pipe, which the
//    step leaves idle, instead of the shifts and 64-bit adds of the integer ALU):
//    S = sum g, AX = g7 - g3, DX = (g0 - g4) + (g6 - g2), AY = g1 - g5, DY = (g0 - g4) - (g6 - g2).
//    The speeds have two decimals, so with V_k = 100 v_k (integers) the momentum sums are exact
//    integers too:
//      N = f_0 + sum_k S_k,  Ax = sum_k V_k AX_k,  Dx = sum_k V_k DX_k  (Ay, Dy alike).
//    So is the energy sum, 10^4 sum |v|^2 f = sum_k V_k^2 S_k, held as two parts (energy_parts).
//    They are converted to FP64 by integer bit operations with one rounding each (fix_to_f64).
//    In FP64:
//      n = N,  100 jx = fma(s, Dx, Ax),  100 jy = fma(s, Dy, Ay),  10^4 sum |v|^2 f = EH 2^32 + EL,
//    and the factors 1/100 and 10^-4 are applied with 1/n (to_macro<100>).
//  - Integer sums are associative, so the ring-parallel kernel, which adds its lanes' integers in
//    another order, forms bit-identical moments.
//  - A node holding an infinity or NaN (biased exponent 255) gets NaN moments, which the health
//    check reports.
__device__ __forceinline__ int f32_exp1(float x) {
  const int e = (int)((__float_as_uint(x) >> 23) & 0xffu);
  return e ? e : 1;
}
// The term of x as (significand, power of two): x enters the sums as (long long)sm * p.
struct FixTerm {
  int sm, p;
};
constexpr int FIX_TOP = 26;          // the largest term is m 2^26 < 2^50
constexpr int FIX_E2 = 150 + FIX_TOP;  // a sum V stands for V 2^(e* - FIX_E2)
// FULL = false when the caller has checked that the node's values are all normal and lie within
// 2^FIX_TOP of the largest, so that no term needs the right shift or lacks the hidden bit.
template <bool FULL = true>
__device__ __forceinline__ FixTerm fix_term(float x, int emax) {
  const unsigned u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xffu);
  FixTerm t;
  if constexpr (FULL) {
    const int m = (int)((u & 0x7fffffu) | (e ? 0x800000u : 0u));
    const int sm = (int)(u >> 31) ? -m : m;
    const int k = FIX_TOP - (emax - (e ? e : 1));  // <= FIX_TOP
    t.sm = k >= 0 ? sm : (sm >> min(-k, 31));
    t.p = k >= 0 ? (1 << k) : 1;
  } else {
    const int m = (int)((u & 0x7fffffu) | 0x800000u);
    t.sm = (int)(u >> 31) ? -m : m;
    t.p = 1 << (FIX_TOP - (emax - e));
  }
  return t;
}
template <bool FULL = true>
__device__ __forceinline__ long long to_fix(float x, int emax) {
  const FixTerm t = fix_term<FULL>(x, emax);
  return (long long)t.sm * t.p;
}
// V * 2^e2, rounded to nearest even, built from the integer's bits (|V| < 2^63, normal result).
__device__ __forceinline__ double fix_to_f64(long long V, int e2) {
  if (V == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)V & 0x8000000000000000ull;
  const unsigned long long A = V < 0 ? 0ull - (unsigned long long)V : (unsigned long long)V;
  const int lz = __clzll((long long)A);  // >= 1
  const unsigned long long U = A << (lz - 1);  // leading one at bit 62
  // round to nearest even at bit 10: add 2^9 - 1 plus the lowest kept bit, then drop the 10 bits
  // (no overflow: U < 2^63). M has its leading one at bit 52, or is 2^53 after a carry.
  const unsigned long long M = (U + 0x1ffull + ((U >> 10) & 1ull)) >> 10;
  const unsigned long long E = (unsigned long long)(1086 - lz + e2);  // biased exponent
  // the leading one (bit 52) adds the last 1 to the exponent field; a carry to 2^53 adds one more,
  // which is the correct result
  return __longlong_as_double((long long)(sgn | (((E - 1ull) << 52) + M)));
}
struct RingFix {
  long long S, AX, DX, AY, DY;
};
template <bool FULL = true>
__device__ __forceinline__ RingFix ring_fix(const float (&x)[8], int emax) {
  FixTerm t[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) t[d] = fix_term<FULL>(x[d], emax);
  RingFix r;
  r.S = 0;
#pragma unroll
  for (int d = 0; d < 8; ++d) r.S += (long long)t[d].sm * t[d].p;
  r.AX = (long long)t[7].sm * t[7].p - (long long)t[3].sm * t[3].p;
  r.AY = (long long)t[1].sm * t[1].p - (long long)t[5].sm * t[5].p;
  const long long a = (long long)t[0].sm * t[0].p - (long long)t[4].sm * t[4].p;
  const long long b = (long long)t[6].sm * t[6].p - (long long)t[2].sm * t[2].p;
  r.DX = a + b;
  r.DY = a - b;
  return r;
}
__device__ __forceinline__ Mom nan_moments() {
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  return Mom{nan, nan, nan, nan};
}

// The energy sum 10^4 sum_k v_k^2 S_k = sum_k V_k^2 S_k needs up to 71 bits, so each S_k is split
// as hi 2^32 + lo (lo unsigned): EH = sum_k V_k^2 hi_k (|EH| < 2^41) and EL = sum_k V_k^2 lo_k
// (< 2^52) are exact integers.
__device__ __forceinline__ void energy_parts(int k, long long S, long long& EH, long long& EL) {
  const long long v2 = (long long)speed_c(k) * speed_c(k);
  EH += v2 * (long long)(int)(S >> 32);
  EL += v2 * (long long)(unsigned)S;
}
// n, 100 jx, 100 jy and 10^4 sum |v|^2 f from the exact sums. EH 2^32 and EL convert to FP64
// exactly (both below 2^53), so their one FP64 sum is the correctly rounded energy sum.
__device__ __forceinline__ Mom fix_moments(long long N, long long Ax, long long Dx, long long Ay, long long Dy,
                                           long long EH, long long EL, int e2) {
  Mom m;
  m.n = fix_to_f64(N, e2);
  m.jx = fma(kS, fix_to_f64(Dx, e2), fix_to_f64(Ax, e2));
  m.jy = fma(kS, fix_to_f64(Dy, e2), fix_to_f64(Ay, e2));
  m.e2 = fix_to_f64(EH, e2 + 32) + fix_to_f64(EL, e2);
  return m;
}

template <bool FULL>
__device__ __forceinline__ Mom fix_node_moments(const float (&x)[Q], int emax) {
  const int e2 = emax - FIX_E2;
  long long N = to_fix<FULL>(x[0], emax), Ax = 0, Dx = 0, Ay = 0, Dy = 0, EH = 0, EL = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float g[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) g[d] = x[1 + 8 * k + d];
    const RingFix r = ring_fix<FULL>(g, emax);
    N += r.S;
    Ax += speed_c(k) * r.AX;
    Dx += speed_c(k) * r.DX;
    Ay += speed_c(k) * r.AY;
    Dy += speed_c(k) * r.DY;
    energy_parts(k, r.S, EH, EL);
  }
  return fix_moments(N, Ax, Dx, Ay, Dy, EH, EL, e2);
}

// Moments of an FP32-storage node; jx, jy in hundredths and the energy in 10^-4 (to_macro<100>).
// When the node's values are all normal and lie within 2^FIX_TOP of its largest (the usual case),
// the terms take the short form; the results are the same.
template <bool COH = false>
__device__ __forceinline__ Mom node_moments(const float* __restrict__ f, long long plane, long long off,
                                            const Coeffs& c) {
  float x[Q];
  int emax = 1, emin = 255;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    x[q] = ldc<COH>(f + (long long)q * plane + off);
    const int e = (int)((__float_as_uint(x[q]) >> 23) & 0xffu);
    emax = max(emax, e);
    emin = min(emin, e);
  }
  if (emax == 255) return nan_moments();
  if (emin > 0 && emax - emin <= FIX_TOP) return fix_node_moments<false>(x, emax);
  return fix_node_moments<true>(x, emax);
}

// One ring of a node (ring-parallel kernel, FP64 storage): S, X, Y of ring k, and f_0 (read by
// every lane).
template <bool COH = false>
__device__ __forceinline__ void ring_of_node(const double* __restrict__ f, long long plane, long long off, int k,
                                             double& f0, double& S, double& X, double& Y) {
  double g[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) g[d] = ldc<COH>(f + (long long)(1 + 8 * k + d) * plane + off);
  f0 = ldc<COH>(f + off);
  ring_sums(g, S, X, Y);
}

// (n, ux, uy, T, P) from the sums; T = (sum |v|^2 f)/(2n) - |u|^2/2  (Eq. 5 with P = nT). JS is
// the unit of jx, jy in the sums: 1 for the FP64 sums, 100 for the fixed-point ones (hundredths,
// with the energy sum in units of 1/JS^2).
struct Macro {
  double n, ux, uy, T, P;
};
template <int JS>
__device__ __forceinline__ Macro to_macro(const Mom& m) {
  Macro o;
  const double in = rcp64(m.n);
  const double ij = JS == 1 ? in : in * (1.0 / JS);
  const double ie = JS == 1 ? in : in * (1.0 / ((double)JS * JS));
  o.n = m.n;
  o.ux = m.jx * ij;
  o.uy = m.jy * ij;
  const double u2 = fma(o.ux, o.ux, o.uy * o.uy);
  o.T = 0.5 * fma(m.e2, ie, -u2);
  o.P = m.n * o.T;
  return o;
}
template <bool COH = false>
__device__ __forceinline__ Macro node_macro(const double* __restrict__ f, long long plane, long long off,
                                            const Coeffs& c) {
  return to_macro<1>(node_moments<COH>(f, plane, off, c));
}
template <bool COH = false>
__device__ __forceinline__ Macro node_macro(const float* __restrict__ f, long long plane, long long off,
                                            const Coeffs& c) {
  return to_macro<100>(node_moments<COH>(f, plane, off, c));
}

// Ring-parallel kernel: the macros of the quad's node, lane r of the quad (r = 0..3) summing ring
// r. Every lane ends with the same values, bit for bit those of node_macro. All four lanes must
// call it together.
template <bool COH = false>
__device__ __forceinline__ Macro quad_macro(const double* __restrict__ f, long long plane, long long off, int r,
                                            const Coeffs& c) {
  const unsigned ALL = 0xffffffffu;
  double f0, S, X, Y;
  ring_of_node<COH>(f, plane, off, r, f0, S, X, Y);
  Mom m;
  // n = ((f_0 + S_0) + S_1) + (S_2 + S_3), the tree of combine_rings
  const double pn = (r == 0) ? f0 + S : S;
  const double n2 = pn + __shfl_xor_sync(ALL, pn, 1);
  m.n = n2 + __shfl_xor_sync(ALL, n2, 2);
  // stage 1 (lanes r, r^1): j pair = fma(v_e, X_e, v_o X_o). The even lane sends its X (Y, S),
  // the odd lane its product v X; each then forms the pair from identical operands.
  const bool even = (r & 1) == 0;
  const double prodx = c.v[r] * X, prody = c.v[r] * Y, prode = c.v2[r] * S;
  const double o_x = __shfl_xor_sync(ALL, even ? X : prodx, 1);
  const double o_y = __shfl_xor_sync(ALL, even ? Y : prody, 1);
  const double o_e = __shfl_xor_sync(ALL, even ? S : prode, 1);
  const int re = r & 2;  // the even lane of the pair
  const double jx2 = even ? fma(c.v[re], X, o_x) : fma(c.v[re], o_x, prodx);
  const double jy2 = even ? fma(c.v[re], Y, o_y) : fma(c.v[re], o_y, prody);
  const double e22 = even ? fma(c.v2[re], S, o_e) : fma(c.v2[re], o_e, prode);
  // stage 2 (pairs 01 and 23): commutative sums, equal in all four lanes
  m.jx = jx2 + __shfl_xor_sync(ALL, jx2, 2);
  m.jy = jy2 + __shfl_xor_sync(ALL, jy2, 2);
  m.e2 = e22 + __shfl_xor_sync(ALL, e22, 2);
  return to_macro<1>(m);
}
// FP32 storage: each lane forms its ring's exact sums, the quad adds the integers (exact, so in
// any order) and exchanges the four S_k, and every lane finishes as node_moments does.
template <bool COH = false>
__device__ __forceinline__ Macro quad_macro(const float* __restrict__ f, long long plane, long long off, int r,
                                            const Coeffs& c) {
  const unsigned ALL = 0xffffffffu;
  float x[8];
  const float x0 = ldc<COH>(f + off);
  int emax = f32_exp1(x0);
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    x[d] = ldc<COH>(f + (long long)(1 + 8 * r + d) * plane + off);
    emax = max(emax, f32_exp1(x[d]));
  }
  emax = max(emax, __shfl_xor_sync(ALL, emax, 1));
  emax = max(emax, __shfl_xor_sync(ALL, emax, 2));
  const RingFix rf = ring_fix(x, emax);
  const long long V = speed_c(r);
  long long N = rf.S + (r == 0 ? to_fix(x0, emax) : 0ll);
  long long Ax = V * rf.AX, Dx = V * rf.DX, Ay = V * rf.AY, Dy = V * rf.DY;
  long long EH = V * V * (long long)(int)(rf.S >> 32), EL = V * V * (long long)(unsigned)rf.S;
#pragma unroll
  for (int lm = 1; lm <= 2; lm <<= 1) {
    N += __shfl_xor_sync(ALL, N, lm);
    Ax += __shfl_xor_sync(ALL, Ax, lm);
    Dx += __shfl_xor_sync(ALL, Dx, lm);
    Ay += __shfl_xor_sync(ALL, Ay, lm);
    Dy += __shfl_xor_sync(ALL, Dy, lm);
    EH += __shfl_xor_sync(ALL, EH, lm);
    EL += __shfl_xor_sync(ALL, EL, lm);
  }
  const int e2 = emax - FIX_E2;
  const Mom m = emax == 255 ? nan_moments() : fix_moments(N, Ax, Dx, Ay, Dy, EH, EL, e2);
  return to_macro<100>(m);
}

__device__ __forceinline__ bool macro_ok(const Macro& o) {
  // finite, n > 0, T > 0 (so P > 0 and the switch denominator of Eq. 16 is positive)
  return pos_finite_bits(o.n) && pos_finite_bits(o.T) && finite_bits(o.ux) && finite_bits(o.uy);
}

// ---------------------------------------------------------------------------------------------
// Equilibrium constants of one node (Eqs. 10-13), with dt/tau folded in (r = dt/tau): 41 FP64
// ops. F_k(theta) = theta P_k(theta) (P_k cubic) enters only as r n F_k = (r n theta) P_k(theta),
// and the rest velocity's r f_eq = r n F_0 A0 with r n F_0 = r n - 8 sum_k r n F_k.
struct EqSite {
  double A0, A1;           // A0 = 1 - b + b^2/2, A1 = 1 - b, b = |u|^2/(2 theta)
  double p[4];             // projections (e.u)/theta for d = 7 (x), 0 (diag), 1 (y), 2 (anti-diag)
  double x[4];             // p^2
  double nF[4];            // r n F_1..r n F_4
  double rest;             // r f_eq of the rest velocity
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
  const double b2 = fma(ux, px, uy * py);  // 2b = |u|^2/theta
  e.A1 = fma(-0.5, b2, 1.0);
  e.A0 = fma(0.125 * b2, b2, e.A1);      // A1 + (2b)^2/8
  const double rn = c.r * n, rnth = rn * th;
  double snF = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    e.nF[k] = rnth * fma(th, fma(th, fma(th, c.Fh[k][3], c.Fh[k][2]), c.Fh[k][1]), c.Fh[k][0]);
    snF += e.nF[k];
  }
  e.rest = fma(-8.0, snF, rn) * e.A0;
  return e;
}

// Per-ring constants alpha..eps (times r n F_k), 6 FP64 ops per ring: with t = r n F_k (1 - b),
//   alpha = r n F_k A0,  beta = t v_k^2/2,  gamma = r n F_k v_k^4/24,  delta = t v_k,  eps = r n F_k v_k^3/6.
struct EqRing {
  double al, be, ga, de, ep;
};
__device__ __forceinline__ EqRing eq_ring(const EqSite& e, int k, const Coeffs& c) {
  EqRing r;
  // select, not e.nF[k]: k may be a run-time ring index (ring-parallel kernel)
  const double nF = k == 0 ? e.nF[0] : k == 1 ? e.nF[1] : k == 2 ? e.nF[2] : e.nF[3];
  const double t = nF * e.A1;
  r.al = nF * e.A0;
  r.be = t * c.v2h[k];
  r.ga = nF * c.v4_24[k];
  r.de = t * c.v[k];
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
// Double-word FP32 (FDLBM_FP32_STORE_DW): a value is hi + lo, two FP32 numbers. The site constants
// stay FP64 (eq_site) and are split into double words; the ring constants are double-word products
// and the pairs' even and odd parts are evaluated by compensated Horner steps. The building blocks
// are the error-free transformations of Knuth (TwoSum: a + b = s + e exactly) and of Dekker with a
// fused multiply-add (a b = p + e exactly, e = fma(a, b, -p)), and the double-word product of
// Joldes, Muller and Popescu (2017, "DWTimesDW" without the lo*lo term; relative error below 7 u^2,
// u = 2^-24). The compensated Horner step is that of Graillat, Langlois and Louvet (2005): the
// running value and the sum of the steps' exact rounding errors, which gives the result as if
// computed with twice the working precision before the final rounding. Every operation is an
// explicitly rounded intrinsic, so nothing is contracted or reassociated.
struct dw {
  float h, l;
};
// x with its 29 low significand bits dropped, as an FP32 number (exact for |x| in the FP32 normal
// range); 0 below 2^-126, far under any equilibrium value the scheme adds to others.
__device__ __forceinline__ float f64_trunc32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ah = hi & 0x7fffffffu;
  const unsigned t = ((ah - (896u << 20)) << 3) | (lo >> 29);
  return __uint_as_float(ah < (897u << 20) ? 0u : (t | (hi & 0x80000000u)));
}
// x = hi + lo: hi its leading 24 bits, lo the (exact, FP64) remainder truncated to FP32, so
// |x - hi - lo| < 2^-47 |x|. One FP64 operation.
__device__ __forceinline__ dw split_dw(double x) {
  dw r;
  r.h = f64_trunc32(x);
  const double hi64 = __hiloint2double(__double2hiint(x), (int)((unsigned)__double2loint(x) & 0xe0000000u));
  r.l = f64_trunc32(__dsub_rn(x, hi64));
  return r;
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {  // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return dw{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ dw mul_dw(dw a, dw b) {
  const float ch = __fmul_rn(a.h, b.h);
  const float cl1 = __fmaf_rn(a.h, b.h, -ch);
  const float cl2 = __fmaf_rn(a.h, b.l, __fmul_rn(a.l, b.h));
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}
__device__ __forceinline__ dw dw_of(const float (&c)[2]) { return dw{c[0], c[1]}; }
// One compensated Horner step, (r + c) <- (r + c) x + a, with x and a double words: r carries the
// rounded values, c the sum of the exact errors.
__device__ __forceinline__ void horner_c(float& r, float& c, dw x, dw a) {
  const float p = __fmul_rn(r, x.h);
  const float e1 = __fmaf_rn(r, x.h, -p);
  float s, e2;
  two_sum(p, a.h, s, e2);
  c = __fmaf_rn(c, x.h, __fadd_rn(__fadd_rn(e1, e2), __fmaf_rn(r, x.l, a.l)));
  r = s;
}
// (r + c) <- (r + c) x with x a double word
__device__ __forceinline__ void times_c(float& r, float& c, dw x) {
  const float p = __fmul_rn(r, x.h);
  const float e1 = __fmaf_rn(r, x.h, -p);
  c = __fmaf_rn(c, x.h, __fmaf_rn(r, x.l, e1));
  r = p;
}
// Double-word sum with both operands double words (Joldes, Muller and Popescu 2017,
// "AccurateDWPlusDW": two TwoSums and two Fast2Sums; relative error below 3 u^2 + 13 u^3, also
// under cancellation).
__device__ __forceinline__ dw add_dw(dw a, dw b) {
  float sh, sl, th, tl;
  two_sum(a.h, b.h, sh, sl);
  two_sum(a.l, b.l, th, tl);
  const dw v = fast_two_sum(sh, __fadd_rn(sl, th));
  return fast_two_sum(v.h, __fadd_rn(tl, v.l));
}
__device__ __forceinline__ dw scale_dw(dw a, float s) {  // s a power of two: exact
  return dw{__fmul_rn(a.h, s), __fmul_rn(a.l, s)};
}
__device__ __forceinline__ dw neg_dw(dw a) { return dw{-a.h, -a.l}; }
// 1/t for a double word t with t.h normal and positive: the FP32 reciprocal y refined by one Newton
// step in double-word form, y + y e with e = 1 - t y formed with the exact product error (1 - t.h y is
// exact by Sterbenz's lemma, t.h y being within an ulp of 1): relative error O(e^2) ~ 2^-46.
__device__ __forceinline__ dw rcp_dw(dw t) {
  const float y = __frcp_rn(t.h);
  const float p = __fmul_rn(t.h, y);
  const float ep = __fmaf_rn(t.h, y, -p);
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), ep), __fmul_rn(t.l, y));
  return fast_two_sum(y, __fmul_rn(y, e));
}
struct EqSiteDW {
  dw A0, A1, p[4], x[4], nF[4];
  float rest;  // r f_eq of the rest velocity, rounded to FP32
};
// eq_site in double-word FP32 from the FP64 macros (split once each): 1/theta by rcp_dw, the
// projections and |u|^2/theta by double-word products and sums, A0 and A1 with accurate sums (they
// cancel when |u|^2/(2 theta) is near 1), and r n F_k = (r n theta) P_k(theta) with each cubic by
// compensated Horner steps over its double-word coefficients.
__device__ __forceinline__ EqSiteDW eq_site_dw(double n, double ux, double uy, double T, const Coeffs& c) {
  const dw dn = split_dw(n), dux = split_dw(ux), duy = split_dw(uy), th = split_dw(T);
  const dw ith = rcp_dw(th);
  const dw px = mul_dw(dux, ith), py = mul_dw(duy, ith);
  const dw kS = dw_of(c.dkS);
  EqSiteDW e;
  e.p[0] = px;
  e.p[1] = mul_dw(kS, add_dw(px, py));
  e.p[2] = py;
  e.p[3] = mul_dw(kS, add_dw(py, neg_dw(px)));
#pragma unroll
  for (int t = 0; t < 4; ++t) e.x[t] = mul_dw(e.p[t], e.p[t]);
  const dw b2 = add_dw(mul_dw(dux, px), mul_dw(duy, py));  // |u|^2 / theta
  e.A1 = add_dw(dw{1.0f, 0.0f}, scale_dw(neg_dw(b2), 0.5f));
  e.A0 = add_dw(e.A1, scale_dw(mul_dw(b2, b2), 0.125f));
  const dw rn = mul_dw(dw_of(c.dr), dn), rnth = mul_dw(rn, th);
  dw snF = dw{0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float r = c.dFh[k][3][0], cc = c.dFh[k][3][1];
    horner_c(r, cc, th, dw_of(c.dFh[k][2]));
    horner_c(r, cc, th, dw_of(c.dFh[k][1]));
    horner_c(r, cc, th, dw_of(c.dFh[k][0]));
    e.nF[k] = mul_dw(rnth, fast_two_sum(r, cc));
    snF = add_dw(snF, e.nF[k]);
  }
  const dw rest = mul_dw(add_dw(rn, scale_dw(neg_dw(snF), 8.0f)), e.A0);
  e.rest = __fadd_rn(rest.h, rest.l);
  return e;
}
// The ring constants of eq_ring as double words (6 products).
struct EqRingDW {
  dw al, be, ga, de, ep;
};
__device__ __forceinline__ EqRingDW eq_ring_dw(const EqSiteDW& e, int k, const Coeffs& c) {
  const dw nF = k == 0 ? e.nF[0] : k == 1 ? e.nF[1] : k == 2 ? e.nF[2] : e.nF[3];
  const dw t = mul_dw(nF, e.A1);
  EqRingDW r;
  r.al = mul_dw(nF, e.A0);
  r.be = mul_dw(t, dw_of(c.dv2h[k]));
  r.ga = mul_dw(nF, dw_of(c.dv4_24[k]));
  r.de = mul_dw(t, dw_of(c.dv[k]));
  r.ep = mul_dw(nF, dw_of(c.dv3_6[k]));
  return r;
}
// r f_eq for the pair with projection p (x = p^2): NE = alpha + x (beta + gamma x) and
// NO = p (delta + eps x) by compensated Horner steps, each rounded to FP32 once; the pair is then
// formed in FP32 as in eq_pair_s<float>.
__device__ __forceinline__ void eq_pair_dw(const EqRingDW& r, dw p, dw x, float& fp, float& fm) {
  float ne = r.ga.h, nc = r.ga.l;
  horner_c(ne, nc, x, r.be);
  horner_c(ne, nc, x, r.al);
  float no = r.ep.h, oc = r.ep.l;
  horner_c(no, oc, x, r.de);
  times_c(no, oc, p);
  const float e = __fadd_rn(ne, nc), o = __fadd_rn(no, oc);
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

template <typename S, int D, bool COH = false>
__device__ __forceinline__ S stencil_dir(const S* __restrict__ p, int pitch, const RingW<S>& w, S rfeq) {
  constexpr int XS = dir_xs(D), YS = dir_ys(D), CL = dir_cls(D), CC = dir_c2(D);
  S acc = fma(w.w0[CC], ldc<COH>(p), rfeq);
  if (XS == 0) {
    acc = fma(w.nu[0], ldc<COH>(p + 1) + ldc<COH>(p - 1), acc);
  } else {
    const S cp = XS > 0 ? w.P1[0][CL] : w.M1[0][CL];
    const S cm = XS > 0 ? w.M1[0][CL] : w.P1[0][CL];
    acc = fma(cp, ldc<COH>(p + 1), acc);
    acc = fma(cm, ldc<COH>(p - 1), acc);
    const S d2 = ldc<COH>(p + 2) - ldc<COH>(p - 2);
    acc = XS > 0 ? fma(w.Dd[0][CL], d2, acc) : fma(-w.Dd[0][CL], d2, acc);
  }
  if (YS == 0) {
    acc = fma(w.nu[1], ldc<COH>(p + pitch) + ldc<COH>(p - pitch), acc);
  } else {
    const S cp = YS > 0 ? w.P1[1][CL] : w.M1[1][CL];
    const S cm = YS > 0 ? w.M1[1][CL] : w.P1[1][CL];
    acc = fma(cp, ldc<COH>(p + pitch), acc);
    acc = fma(cm, ldc<COH>(p - pitch), acc);
    const S d2 = ldc<COH>(p + 2 * pitch) - ldc<COH>(p - 2 * pitch);
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

// Update of all 33 velocities at one interior node, given its moments and nu_x, nu_y. ES is the
// equilibrium's site constants: EqSite, or EqSiteDW for the double-word variant (S = float).
template <typename S, typename ES = EqSite, bool COH = false>
__device__ __forceinline__ void update_ring(int K, const S* __restrict__ f, S* __restrict__ fn, const Grid& g,
                                            const Coeffs& c, long long off, int gx, int gy, const GhostOwn& go,
                                            const ES& e, S w0base, S nux, S nuy) {
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
  const S* fq = f + off;
  // All 8 directions of the ring are computed before any store, so the ring is one basic block
  // the compiler can interleave (the ghost-copy branch comes once per ring, not per velocity).
  S out[8];
  if constexpr (std::is_same<ES, EqSiteDW>::value) {
    S fe[8];
    const EqRingDW er = eq_ring_dw(e, K, c);
    eq_pair_dw(er, e.p[0], e.x[0], fe[7], fe[3]);
    eq_pair_dw(er, e.p[1], e.x[1], fe[0], fe[4]);
    eq_pair_dw(er, e.p[2], e.x[2], fe[1], fe[5]);
    eq_pair_dw(er, e.p[3], e.x[3], fe[2], fe[6]);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const S* p = fq + (long long)(1 + 8 * K + d) * g.plane;
      switch (d) {
        case 0: out[0] = stencil_dir<S, 0, COH>(p, g.pitch, w, fe[0]); break;
        case 1: out[1] = stencil_dir<S, 1, COH>(p, g.pitch, w, fe[1]); break;
        case 2: out[2] = stencil_dir<S, 2, COH>(p, g.pitch, w, fe[2]); break;
        case 3: out[3] = stencil_dir<S, 3, COH>(p, g.pitch, w, fe[3]); break;
        case 4: out[4] = stencil_dir<S, 4, COH>(p, g.pitch, w, fe[4]); break;
        case 5: out[5] = stencil_dir<S, 5, COH>(p, g.pitch, w, fe[5]); break;
        case 6: out[6] = stencil_dir<S, 6, COH>(p, g.pitch, w, fe[6]); break;
        default: out[7] = stencil_dir<S, 7, COH>(p, g.pitch, w, fe[7]); break;
      }
    }
  } else {
    const EqRing er = eq_ring(e, K, c);
    S fp, fm;
    // pair (d7: 0 deg, d3: 180 deg), projection p_x
    eq_pair_s<S>(er, e.p[0], e.x[0], fp, fm);
    out[7] = stencil_dir<S, 7, COH>(fq + (long long)(1 + 8 * K + 7) * g.plane, g.pitch, w, fp);
    out[3] = stencil_dir<S, 3, COH>(fq + (long long)(1 + 8 * K + 3) * g.plane, g.pitch, w, fm);
    // pair (d0: 45 deg, d4: 225 deg), projection s(p_x + p_y)
    eq_pair_s<S>(er, e.p[1], e.x[1], fp, fm);
    out[0] = stencil_dir<S, 0, COH>(fq + (long long)(1 + 8 * K + 0) * g.plane, g.pitch, w, fp);
    out[4] = stencil_dir<S, 4, COH>(fq + (long long)(1 + 8 * K + 4) * g.plane, g.pitch, w, fm);
    // pair (d1: 90 deg, d5: 270 deg), projection p_y
    eq_pair_s<S>(er, e.p[2], e.x[2], fp, fm);
    out[1] = stencil_dir<S, 1, COH>(fq + (long long)(1 + 8 * K + 1) * g.plane, g.pitch, w, fp);
    out[5] = stencil_dir<S, 5, COH>(fq + (long long)(1 + 8 * K + 5) * g.plane, g.pitch, w, fm);
    // pair (d2: 135 deg, d6: 315 deg), projection s(p_y - p_x)
    eq_pair_s<S>(er, e.p[3], e.x[3], fp, fm);
    out[2] = stencil_dir<S, 2, COH>(fq + (long long)(1 + 8 * K + 2) * g.plane, g.pitch, w, fp);
    out[6] = stencil_dir<S, 6, COH>(fq + (long long)(1 + 8 * K + 6) * g.plane, g.pitch, w, fm);
  }
  store_ring<S>(fn, g, gx, gy, go, K, out);
}

// Eq. 17 for ring K's 8 velocities at one interior node, with their r f_eq given (fe[d] for
// direction d): the staged step's second half.
template <typename S, bool COH = false>
__device__ __forceinline__ void ring_stencil(int K, const S* __restrict__ f, S* __restrict__ fn, const Grid& g,
                                             const Coeffs& c, long long off, int gx, int gy, const GhostOwn& go,
                                             const S (&fe)[8], S w0base, S nux, S nuy) {
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
  const S* fq = f + off;
  S out[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const S* p = fq + (long long)(1 + 8 * K + d) * g.plane;
    switch (d) {
      case 0: out[0] = stencil_dir<S, 0, COH>(p, g.pitch, w, fe[0]); break;
      case 1: out[1] = stencil_dir<S, 1, COH>(p, g.pitch, w, fe[1]); break;
      case 2: out[2] = stencil_dir<S, 2, COH>(p, g.pitch, w, fe[2]); break;
      case 3: out[3] = stencil_dir<S, 3, COH>(p, g.pitch, w, fe[3]); break;
      case 4: out[4] = stencil_dir<S, 4, COH>(p, g.pitch, w, fe[4]); break;
      case 5: out[5] = stencil_dir<S, 5, COH>(p, g.pitch, w, fe[5]); break;
      case 6: out[6] = stencil_dir<S, 6, COH>(p, g.pitch, w, fe[6]); break;
      default: out[7] = stencil_dir<S, 7, COH>(p, g.pitch, w, fe[7]); break;
    }
  }
  store_ring<S>(fn, g, gx, gy, go, K, out);
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
// Moment buffer planes (split step): n, ux, uy, T in FP64, then P in the storage precision.
template <typename S>
struct MomPlanes {
  double *n, *ux, *uy, *T;
  S* P;
};
template <typename S>
__device__ __forceinline__ MomPlanes<S> mom_planes(const Grid& g) {
  double* b = static_cast<double*>(g.mom);
  return MomPlanes<S>{b, b + g.plane, b + 2 * g.plane, b + 3 * g.plane, reinterpret_cast<S*>(b + 4 * g.plane)};
}
// a node of the tile ring is needed unless it is a corner of the padded region
__device__ __forceinline__ bool ring_node_needed(const Grid& g, int gx, int gy) {
  const bool inx = gx >= 0 && gx < g.nx, iny = gy >= 0 && gy < g.ny;
  return (inx && iny) || (iny && (gx == -1 || gx == g.nx)) || (inx && (gy == -1 || gy == g.ny));
}

// Split step, pass 1: the moments of every interior node and of the ghost layer next to each edge,
// once, into the moment buffer (with the NUMERIC health check).
template <typename S>
__global__ void k_moments(const S* __restrict__ f, Grid g, Coeffs c, unsigned* __restrict__ health) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x - 1, gy = blockIdx.y * blockDim.y + threadIdx.y - 1;
  if (gx > g.nx || gy > g.ny || !ring_node_needed(g, gx, gy)) return;
  const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
  const Macro m = node_macro(f, g.plane, off, c);
  if (!macro_ok(m)) atomicOr(health, H_NUMERIC);
  const MomPlanes<S> M = mom_planes<S>(g);
  M.n[off] = m.n;
  M.ux[off] = m.ux;
  M.uy[off] = m.uy;
  M.T[off] = m.T;
  M.P[off] = from_d<S>(m.P);
}

// The 33 r f_eq of one node into a stage s_fe[q][node] (NN nodes per plane). DW: the double-word
// evaluation of the rings (FDLBM_FP32_STORE_DW, S = float).
template <typename S, int NN, bool DW = false>
__device__ __forceinline__ void stage_feq(S* __restrict__ s_fe, int node, double n, double ux, double uy, double T,
                                          const Coeffs& c) {
  if constexpr (DW) {
    const EqSiteDW e = eq_site_dw(n, ux, uy, T, c);
    s_fe[node] = e.rest;
#pragma unroll
    for (int K = 0; K < 4; ++K) {
      const EqRingDW er = eq_ring_dw(e, K, c);
      S fp, fm;
      eq_pair_dw(er, e.p[0], e.x[0], fp, fm);
      s_fe[(1 + 8 * K + 7) * NN + node] = fp;
      s_fe[(1 + 8 * K + 3) * NN + node] = fm;
      eq_pair_dw(er, e.p[1], e.x[1], fp, fm);
      s_fe[(1 + 8 * K + 0) * NN + node] = fp;
      s_fe[(1 + 8 * K + 4) * NN + node] = fm;
      eq_pair_dw(er, e.p[2], e.x[2], fp, fm);
      s_fe[(1 + 8 * K + 1) * NN + node] = fp;
      s_fe[(1 + 8 * K + 5) * NN + node] = fm;
      eq_pair_dw(er, e.p[3], e.x[3], fp, fm);
      s_fe[(1 + 8 * K + 2) * NN + node] = fp;
      s_fe[(1 + 8 * K + 6) * NN + node] = fm;
    }
    return;
  }
  const EqSite e = eq_site(n, ux, uy, T, c);
  s_fe[node] = to_s<S>(e.rest);
#pragma unroll
  for (int K = 0; K < 4; ++K) {
    const EqRing er = eq_ring(e, K, c);
    S fp, fm;
    eq_pair_s<S>(er, e.p[0], e.x[0], fp, fm);
    s_fe[(1 + 8 * K + 7) * NN + node] = fp;
    s_fe[(1 + 8 * K + 3) * NN + node] = fm;
    eq_pair_s<S>(er, e.p[1], e.x[1], fp, fm);
    s_fe[(1 + 8 * K + 0) * NN + node] = fp;
    s_fe[(1 + 8 * K + 4) * NN + node] = fm;
    eq_pair_s<S>(er, e.p[2], e.x[2], fp, fm);
    s_fe[(1 + 8 * K + 1) * NN + node] = fp;
    s_fe[(1 + 8 * K + 5) * NN + node] = fm;
    eq_pair_s<S>(er, e.p[3], e.x[3], fp, fm);
    s_fe[(1 + 8 * K + 2) * NN + node] = fp;
    s_fe[(1 + 8 * K + 6) * NN + node] = fm;
  }
}

// One node of phase 1: the moments of local node (lx, ly) of the tile whose first node is (x0, y0)
// (local (1, 1)), stored if an update needs them: every interior node and the ghost layer next to
// an edge, never a grid corner. Its loads take an address clamped into the padded grid, so that a
// caller can run it branch-free on slots it does not need.
template <typename S, int SW, bool COH>
__device__ __forceinline__ void moment_slot(const S* __restrict__ f, const Grid& g, const Coeffs& c, int x0, int y0,
                                            int lx, int ly, double (*s_n)[SW], double (*s_ux)[SW],
                                            double (*s_uy)[SW], double (*s_T)[SW], S (*s_P)[SW], unsigned& bits) {
  const int gx = x0 + lx - 1, gy = y0 + ly - 1;
  const bool inx = gx >= 0 && gx < g.nx, iny = gy >= 0 && gy < g.ny;
  const bool need = (inx && iny) || (iny && (gx == -1 || gx == g.nx)) || (inx && (gy == -1 || gy == g.ny));
  const int cx = min(max(gx, -1), g.nx), cy = min(max(gy, -1), g.ny);  // inside the padded grid
  const long long off = (long long)(cy + NG) * g.pitch + (cx + NG);
  const Macro m = node_macro<COH>(f, g.plane, off, c);
  if (need) {
    if (!macro_ok(m)) bits |= H_NUMERIC;
    s_n[ly][lx] = m.n;
    s_ux[ly][lx] = m.ux;
    s_uy[ly][lx] = m.uy;
    s_T[ly][lx] = m.T;
    s_P[ly][lx] = from_d<S>(m.P);
  }
}

// Staged phase 2 of a BX x (BY RY) tile (FP32 storage), from the moments of the tile and its ring
// in shared memory: first the thread's nodes' 33 r f_eq each (the FP64 work) into s_fe[q][node],
// then their stencils (FP32 and memory work) from there.
template <typename S, int BX, int BY, int RY, int SW, bool DW, bool COH>
__device__ __forceinline__ void staged_update(const S* __restrict__ f, S* __restrict__ fn, const Grid& g,
                                              const Coeffs& c, int x0, int y0, const double (*s_n)[SW],
                                              const double (*s_ux)[SW], const double (*s_uy)[SW],
                                              const double (*s_T)[SW], const S (*s_P)[SW], S* __restrict__ s_fe,
                                              unsigned& bits) {
  constexpr int TW = BX, TH = BY * RY;
  using SC = StencilConsts<S>;
  constexpr int NN = TW * TH;
#pragma unroll 1
  for (int rr = 0; rr < RY; ++rr) {
    const int lx = threadIdx.x + 1, ly = threadIdx.y + rr * BY + 1;
    const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y + rr * BY;
    if (gx >= g.nx || gy >= g.ny) continue;
    const int node = (threadIdx.y + rr * BY) * TW + threadIdx.x;
    stage_feq<S, NN, DW>(s_fe, node, s_n[ly][lx], s_ux[ly][lx], s_uy[ly][lx], s_T[ly][lx], c);
  }
  // no barrier: a thread reads back only its own nodes' f_eq (a node's stencil takes r f_eq at
  // the node itself), so its warps run on into their stencils as soon as they are done
#pragma unroll 1
  for (int rr = 0; rr < RY; ++rr) {
    const int lx = threadIdx.x + 1, ly = threadIdx.y + rr * BY + 1;
    const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y + rr * BY;
    if (gx >= g.nx || gy >= g.ny) continue;
    const int node = (threadIdx.y + rr * BY) * TW + threadIdx.x;
    const double ux = s_ux[ly][lx], uy = s_uy[ly][lx];
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
    const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
    const GhostOwn go = ghost_own(g, gx, gy);
    {
      const S* p = f + off;
      S acc = fma(w0base, ldc<COH>(p), s_fe[node]);
      acc = fma(snux, ldc<COH>(p + 1) + ldc<COH>(p - 1), acc);
      acc = fma(snuy, ldc<COH>(p + g.pitch) + ldc<COH>(p - g.pitch), acc);
      store_node<S, 0>(fn, g, gx, gy, go, acc);
    }
#pragma unroll
    for (int K = 0; K < 4; ++K) {
      S fe[8];
#pragma unroll
      for (int d = 0; d < 8; ++d) fe[d] = s_fe[(1 + 8 * K + d) * NN + node];
      ring_stencil<S, COH>(K, f, fn, g, c, off, gx, gy, go, fe, w0base, snux, snuy);
    }
  }
}

// WRAPY (batched kernel): a tile that holds a y-periodic grid's whole height takes its two ghost
// rows' moments from the interior rows they copy (bit for bit the same values) instead of summing
// them again: 4-row serving tubes in 32 x 4 tiles sum 4 rows of moments instead of 6.
// DW (S = float only): the double-word equilibrium of FDLBM_FP32_STORE_DW.
template <typename S, int BX, int BY, int RY, bool FROM_BUF = false, bool WRAPY = false, bool STAGE = false,
          bool DW = false, bool COH = false>
__device__ __forceinline__ void step_tile(const S* __restrict__ f, S* __restrict__ fn, const Grid& g, const Coeffs& c,
                                          unsigned* __restrict__ health, int tx, int ty, S* s_fe = nullptr) {
  static_assert(!DW || std::is_same<S, float>::value, "the double-word equilibrium is for FP32 storage");
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
  // to an edge, never the corners). Branch-free and unrolled over a thread's slots, so the FP64
  // chains of its 2-3 nodes interleave: every slot loads from an address clamped into the padded
  // grid, and only needed nodes are stored and health-checked. The split step reads them from
  // the moment buffer instead.
  constexpr int NSLOT = (SW * SH + NT - 1) / NT;
  if constexpr (FROM_BUF) {
    const MomPlanes<S> M = mom_planes<S>(g);
    for (int idx = tid; idx < SW * SH; idx += NT) {
      const int lx = idx % SW, ly = idx / SW;
      const int gx = x0 + lx - 1, gy = y0 + ly - 1;
      if (gx > g.nx || gy > g.ny || !ring_node_needed(g, gx, gy)) continue;
      const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
      s_n[ly][lx] = M.n[off];
      s_ux[ly][lx] = M.ux[off];
      s_uy[ly][lx] = M.uy[off];
      s_T[ly][lx] = M.T[off];
      s_P[ly][lx] = M.P[off];
    }
  } else {
  const bool wrap = WRAPY && y0 == 0 && g.ny <= TH && g.bc[2] == BC_PERIODIC && g.bc[3] == BC_PERIODIC;
  const int nslot = wrap ? SW * g.ny : SW * SH;  // with wrap: local rows 1..ny only
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) {
    const int idx = tid + k * NT;
    // the slots before the last always lie in the tile ring (no branch); the last one is guarded
    if (WRAPY ? idx >= nslot : ((k + 1) * NT > SW * SH && idx >= SW * SH)) continue;
    moment_slot<S, SW, COH>(f, g, c, x0, y0, idx % SW, idx / SW + (wrap ? 1 : 0), s_n, s_ux, s_uy, s_T, s_P, bits);
  }
  if (wrap) {  // CTA-uniform
    __syncthreads();
    // ghost row y = -1 (local row 0) copies row ny - 1 (local row ny); y = ny copies row 0
    const int ny = g.ny;
    for (int lx = tid; lx < SW; lx += NT) {
      s_n[0][lx] = s_n[ny][lx], s_n[ny + 1][lx] = s_n[1][lx];
      s_ux[0][lx] = s_ux[ny][lx], s_ux[ny + 1][lx] = s_ux[1][lx];
      s_uy[0][lx] = s_uy[ny][lx], s_uy[ny + 1][lx] = s_uy[1][lx];
      s_T[0][lx] = s_T[ny][lx], s_T[ny + 1][lx] = s_T[1][lx];
      s_P[0][lx] = s_P[ny][lx], s_P[ny + 1][lx] = s_P[1][lx];
    }
  }
  }
  __syncthreads();

  if constexpr (STAGE) {
    staged_update<S, BX, BY, RY, SW, DW, COH>(f, fn, g, c, x0, y0, s_n, s_ux, s_uy, s_T, s_P, s_fe, bits);
  } else {
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
    using ES = typename std::conditional<DW, EqSiteDW, EqSite>::type;
    ES e;
    if constexpr (DW) e = eq_site_dw(n, ux, uy, T, c);
    else e = eq_site(n, ux, uy, T, c);
    const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
    const GhostOwn go = ghost_own(g, gx, gy);
    // rest velocity: f_eq = n F_0 A0; c = 0 on both axes (line IV only)
    {
      S rfeq;
      if constexpr (DW) rfeq = e.rest;
      else rfeq = to_s<S>(e.rest);
      const S* p = f + off;
      S acc = fma(w0base, ldc<COH>(p), rfeq);
      acc = fma(snux, ldc<COH>(p + 1) + ldc<COH>(p - 1), acc);
      acc = fma(snuy, ldc<COH>(p + g.pitch) + ldc<COH>(p - g.pitch), acc);
      store_node<S, 0>(fn, g, gx, gy, go, acc);
    }
    update_ring<S, ES, COH>(0, f, fn, g, c, off, gx, gy, go, e, w0base, snux, snuy);
    update_ring<S, ES, COH>(1, f, fn, g, c, off, gx, gy, go, e, w0base, snux, snuy);
    update_ring<S, ES, COH>(2, f, fn, g, c, off, gx, gy, go, e, w0base, snux, snuy);
    update_ring<S, ES, COH>(3, f, fn, g, c, off, gx, gy, go, e, w0base, snux, snuy);
  }
  }
  if (bits) atomicOr(health, bits);
}

// STAGE (FP32 storage, the 32 x 16 and 64 x 8 tiles): phase 2 goes through shared memory. The
// tile's 33 r f_eq per node, the FP64 work, are formed first for every node and the stencils
// follow. Dynamic shared memory of stage_bytes holds them: 66 KB beside the 22 KB of moments
// still allows 2 CTAs per SM. Smaller tiles (4 CTAs per SM) and larger ones measured slower
// staged; FP64 storage would need twice the bytes and does not stage.
template <typename S, int TW, int TH, bool STAGE>
constexpr int stage_bytes() {
  return STAGE && sizeof(S) == 4 ? Q * TW * TH * (int)sizeof(S) : 0;
}
template <typename S, int BX, int BY, int RY, int MINB, bool WRAPY = false, bool STAGE = false, bool DW = false>
__global__ void __launch_bounds__(BX * BY, MINB) k_step(const S* __restrict__ f, S* __restrict__ fn, Grid g, Coeffs c,
                                                  unsigned* __restrict__ health) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  step_tile<S, BX, BY, RY, false, WRAPY, STAGE && sizeof(S) == 4, DW>(f, fn, g, c, health, blockIdx.x, blockIdx.y,
                                                                      reinterpret_cast<S*>(s_dyn));
}
// Split step, pass 2: the update with the tile's moments read from the moment buffer.
template <typename S, int BX, int BY, int RY, int MINB, bool STAGE = false, bool DW = false>
__global__ void __launch_bounds__(BX * BY, MINB) k_update(const S* __restrict__ f, S* __restrict__ fn, Grid g,
                                                    Coeffs c, unsigned* __restrict__ health) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  step_tile<S, BX, BY, RY, true, false, STAGE && sizeof(S) == 4, DW>(f, fn, g, c, health, blockIdx.x, blockIdx.y,
                                                                     reinterpret_cast<S*>(s_dyn));
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
  step_tile<S, BX, BY, RY, false, true>(in, out, g, c, m.health, tx, ty);
}

// Ring-parallel step for small grids, where one thread per node leaves the GPU's FP64 pipes
// waiting on long dependency chains. Four lanes share a node, lane r holding velocity ring r:
// - Moments (quad_macro): each lane sums its ring. With FP64 storage two shuffle stages combine
//   the rings in the same pairwise tree as node_moments; with FP32 storage the quad adds the exact
//   integer sums. Either way the moments are bit for bit those of k_step.
// - Update: all four lanes evaluate the node's constants (switch, weights, f_eq site terms).
//   That costs no extra issue slots: it is one warp instruction whether one lane or four use it.
//   Each lane then updates its own 8 velocities, and lane 0 also the rest velocity.
// Each thread thus issues about half of k_step's FP64 chain. Results are bitwise those of k_step.
// One TW x TH tile (tile_x, tile_y) of the ring-parallel step, by a CTA of 4 TW TH threads: the
// body shared by k_step_rp (one tile per CTA) and the persistent kernel (tiles and steps in a loop).
template <typename S, int TW, int TH, bool COH = false>
__device__ __forceinline__ void rp_tile(const S* __restrict__ f, S* __restrict__ fn, const Grid& g, const Coeffs& c,
                                        unsigned* __restrict__ health, int tile_x, int tile_y) {
  constexpr int SW = TW + 2, SH = TH + 2, NQ = TW * TH;
  using SC = StencilConsts<S>;
  __shared__ double s_n[SH][SW], s_ux[SH][SW], s_uy[SH][SW], s_T[SH][SW];
  __shared__ S s_P[SH][SW];
  const int r = threadIdx.x & 3, quad = threadIdx.x >> 2;
  const int x0 = tile_x * TW, y0 = tile_y * TH;
  unsigned bits = 0;

  // Phase 1: moments on the tile and its ring; every lane takes part in every shuffle.
  constexpr int NSLOT = (SW * SH + NQ - 1) / NQ;
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) {
    const int idx = quad + k * NQ;
    const bool inslot = idx < SW * SH;
    const int lx = inslot ? idx % SW : 0, ly = inslot ? idx / SW : 0;
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    const bool inx = gx >= 0 && gx < g.nx, iny = gy >= 0 && gy < g.ny;
    const bool need =
        inslot && ((inx && iny) || (iny && (gx == -1 || gx == g.nx)) || (inx && (gy == -1 || gy == g.ny)));
    const int cx = min(max(gx, -1), g.nx), cy = min(max(gy, -1), g.ny);
    const long long off = (long long)(cy + NG) * g.pitch + (cx + NG);
    const Macro mm = quad_macro<COH>(f, g.plane, off, r, c);
    if (need && r == 0) {
      if (!macro_ok(mm)) bits |= H_NUMERIC;
      s_n[ly][lx] = mm.n;
      s_ux[ly][lx] = mm.ux;
      s_uy[ly][lx] = mm.uy;
      s_T[ly][lx] = mm.T;
      s_P[ly][lx] = from_d<S>(mm.P);
    }
  }
  __syncthreads();

  // Phase 2: the quad's node.
  const int tx = quad % TW, ty = quad / TW;
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx < g.nx && gy < g.ny) {
    const int lx = tx + 1, ly = ty + 1;
    const double n = s_n[ly][lx], ux = s_ux[ly][lx], uy = s_uy[ly][lx], T = s_T[ly][lx];
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
    if (r == 0 && (akx > (S)1 || aky > (S)1)) bits |= H_KAPPA;
    S snux = 0, snuy = 0;
    if (!(g.flags & F_NO_VISC)) {
      snux = (S)0.5 * thx * akx * ((S)1 - akx);
      snuy = (S)0.5 * thy * aky * ((S)1 - aky);
    }
    const S w0base = ((S)1 - SC::r(c)) - (S)2 * (snux + snuy);
    const EqSite e = eq_site(n, ux, uy, T, c);
    const long long off = (long long)(gy + NG) * g.pitch + (gx + NG);
    const GhostOwn go = ghost_own(g, gx, gy);
    if (r == 0) {
      const S rfeq = to_s<S>(e.rest);
      const S* p = f + off;
      S acc = fma(w0base, ldc<COH>(p), rfeq);
      acc = fma(snux, ldc<COH>(p + 1) + ldc<COH>(p - 1), acc);
      acc = fma(snuy, ldc<COH>(p + g.pitch) + ldc<COH>(p - g.pitch), acc);
      store_node<S, 0>(fn, g, gx, gy, go, acc);
    }
    update_ring<S, EqSite, COH>(r, f, fn, g, c, off, gx, gy, go, e, w0base, snux, snuy);
  }
  if (bits) atomicOr(health, bits);
}
template <typename S, int TW, int TH>
__global__ void __launch_bounds__(4 * TW * TH) k_step_rp(const S* __restrict__ f, S* __restrict__ fn, Grid g,
                                                       Coeffs c, unsigned* __restrict__ health) {
  rp_tile<S, TW, TH>(f, fn, g, c, health, blockIdx.x, blockIdx.y);
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
  store_node<S, 0>(f, g, gx, gy, go, from_d<S>(e.rest));
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
  const Macro m = node_macro(f, g.plane, off, c);
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
// Opt a kernel in to `bytes` of dynamic shared memory (above 48 KB the default limit refuses the
// launch), once per instantiation and device: `done` holds one bit per device ordinal.
template <typename K>
cudaError_t allow_dynamic_smem(K kernel, int bytes, std::atomic<unsigned long long>& done) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <typename S, int BX, int BY, int RY, int MINB, bool WRAPY = false, bool STAGE = false, bool DW = false>
cudaError_t launch_step_t(const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                          cudaStream_t s) {
  constexpr int smem = stage_bytes<S, BX, BY * RY, STAGE>();
  static std::atomic<unsigned long long> attr{0};  // devices already opted in
  const cudaError_t e = allow_dynamic_smem(k_step<S, BX, BY, RY, MINB, WRAPY, STAGE, DW>, smem, attr);
  if (e != cudaSuccess) return e;
  dim3 block(BX, BY);
  dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY * RY - 1) / (BY * RY));
  k_step<S, BX, BY, RY, MINB, WRAPY, STAGE, DW><<<grid, block, smem, s>>>(static_cast<const S*>(f),
                                                                          static_cast<S*>(fn), g, c, health);
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
    case V_T32x24: return launch_batch_t<S, 32, 4, 6, 4>(mem, nmem, tiles, step, c, s);
    case V_T32x28: return launch_batch_t<S, 32, 4, 7, 4>(mem, nmem, tiles, step, c, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename S, int TW, int TH>
cudaError_t launch_rp_t(const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health, cudaStream_t s) {
  dim3 grid((g.nx + TW - 1) / TW, (g.ny + TH - 1) / TH);
  k_step_rp<S, TW, TH><<<grid, 4 * TW * TH, 0, s>>>(static_cast<const S*>(f), static_cast<S*>(fn), g, c, health);
  return cudaGetLastError();
}

template <typename S, int BX, int BY, int RY, int MINB, bool STAGE = false, bool DW = false>
cudaError_t launch_split_t(const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health, cudaStream_t s) {
  if (!g.mom) return cudaErrorInvalidValue;
  constexpr int smem = stage_bytes<S, BX, BY * RY, STAGE>();
  static std::atomic<unsigned long long> attr{0};  // devices already opted in
  const cudaError_t e = allow_dynamic_smem(k_update<S, BX, BY, RY, MINB, STAGE, DW>, smem, attr);
  if (e != cudaSuccess) return e;
  dim3 mb(32, 8), mg((g.nx + 2 + 31) / 32, (g.ny + 2 + 7) / 8);
  k_moments<S><<<mg, mb, 0, s>>>(static_cast<const S*>(f), g, c, health);
  dim3 block(BX, BY);
  dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY * RY - 1) / (BY * RY));
  k_update<S, BX, BY, RY, MINB, STAGE, DW><<<grid, block, smem, s>>>(static_cast<const S*>(f), static_cast<S*>(fn),
                                                                     g, c, health);
  return cudaGetLastError();
}

// DW: the double-word equilibrium (FDLBM_FP32_STORE_DW, S = float); it has no ring-parallel kernel,
// so those variants take the 32 x 8 tile.
template <typename S, bool DW = false>
cudaError_t launch_step_v(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                          cudaStream_t s) {
  switch (variant) {
    case V_S32x16: return launch_split_t<S, 32, 8, 2, 2, true, DW>(f, fn, g, c, health, s);
    case V_S32x32: return launch_split_t<S, 32, 8, 4, 2, false, DW>(f, fn, g, c, health, s);
    case V_RP16x4:
      if constexpr (DW) return launch_step_t<S, 32, 4, 2, 4, false, false, DW>(f, fn, g, c, health, s);
      else return launch_rp_t<S, 16, 4>(f, fn, g, c, health, s);
    case V_RP8x4:
      if constexpr (DW) return launch_step_t<S, 32, 4, 2, 4, false, false, DW>(f, fn, g, c, health, s);
      else return launch_rp_t<S, 8, 4>(f, fn, g, c, health, s);
    case V_T32x4: return launch_step_t<S, 32, 4, 1, 4, false, false, DW>(f, fn, g, c, health, s);
    case V_T32x8: return launch_step_t<S, 32, 4, 2, 4, false, false, DW>(f, fn, g, c, health, s);
    case V_T32x16: return launch_step_t<S, 32, 8, 2, 2, false, true, DW>(f, fn, g, c, health, s);
    case V_T16x4: return launch_step_t<S, 16, 4, 1, 1, false, false, DW>(f, fn, g, c, health, s);
    case V_T64x8: return launch_step_t<S, 64, 4, 2, 2, false, true, DW>(f, fn, g, c, health, s);
    case V_T32x32:
      if constexpr (std::is_same<S, float>::value) return launch_step_t<S, 32, 4, 1, 6, false, true, DW>(f, fn, g, c, health, s);
      else return launch_step_t<S, 32, 8, 4, 2>(f, fn, g, c, health, s);
    case V_T32x24:
      // FP32 storage: a staged 32 x 8 tile at <= 85 registers for 3 CTAs per SM (24 warps); FP64
      // storage keeps the 32 x 24 tile of 128 threads
      if constexpr (std::is_same<S, float>::value) return launch_step_t<S, 32, 8, 1, 3, false, true, DW>(f, fn, g, c, health, s);
      else return launch_step_t<S, 32, 4, 6, 4>(f, fn, g, c, health, s);
    case V_T32x28:
      if constexpr (std::is_same<S, float>::value) return launch_step_t<S, 32, 8, 1, 4, false, true, DW>(f, fn, g, c, health, s);
      else return launch_step_t<S, 32, 4, 7, 4>(f, fn, g, c, health, s);
    default: return cudaErrorInvalidValue;
  }
}

// The tile variants for a grid whose whole y-periodic height fits in one tile (step_tile WRAPY):
// instantiated in their own translation units, fdlbm_step_wrap_*.cu.
template <typename S>
cudaError_t launch_step_wrap_v(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c,
                               unsigned* health, cudaStream_t s) {
  switch (variant) {
    case V_T32x4: return launch_step_t<S, 32, 4, 1, 4, true>(f, fn, g, c, health, s);
    case V_T32x8: return launch_step_t<S, 32, 4, 2, 4, true>(f, fn, g, c, health, s);
    case V_T32x16: return launch_step_t<S, 32, 8, 2, 2, true, true>(f, fn, g, c, health, s);
    case V_T16x4: return launch_step_t<S, 16, 4, 1, 1, true>(f, fn, g, c, health, s);
    case V_T64x8: return launch_step_t<S, 64, 4, 2, 2, true, true>(f, fn, g, c, health, s);
    case V_T32x32: return launch_step_t<S, 32, 8, 4, 2, true>(f, fn, g, c, health, s);
    case V_T32x24: return launch_step_t<S, 32, 4, 6, 4, true>(f, fn, g, c, health, s);
    case V_T32x28: return launch_step_t<S, 32, 4, 7, 4, true>(f, fn, g, c, health, s);
    default: return cudaErrorInvalidValue;
  }
}

inline dim3 grid2d(const Grid& g, dim3 b) { return dim3((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y); }

}  // namespace
}  // namespace fdlbm

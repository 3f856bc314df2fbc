// fdlbm_vn.cu -- von Neumann analysis of the FDLBM scheme (Sec. 4, Eqs. 18-20) on sm_103a.
//
// One warp per case. The 33 x 33 complex amplification matrix G lives in shared memory as
// double-double (re and im planes of (hi, lo) pairs, 34.8 KB), and every step runs in
// double-double arithmetic (fdlbm_dd.cuh):
//   1. G from the analytic chain rule of Eq. 20: row factors d f^eq_i / d(n, T, u_x, u_y) (lane
//      i), column factors d(n, T, u_x, u_y) / d f_j (lane j), and the diagonal symbol of Eq. 17.
//   2. Householder reduction to upper Hessenberg form (lanes over columns, then over rows).
//   3. Single-shift QR sweeps with Givens rotations restricted to the active block (eigenvalues
//      only). The rotation of row pair k is computed, the column rotation k-1 is applied right
//      after it (the two touch different data), so a sweep stores no rotations. Shifts are
//      Wilkinson's, in double-double: an FP64 shift stalls into linear convergence on the
//      near-double eigenvalues that coinciding stencil symbols produce. A 1 x 1 or 2 x 2 block
//      that splits off is solved directly.
// Scalar steps (a rotation's parameters, a shift) are computed by every lane alike, so no lane
// waits on another beyond __syncwarp.
//
// FP64 issues at ~2 instructions/clk/SM on this part, so the kernel is bound by the FP64 pipe;
// six single-warp CTAs share an SM (6 x 35 KB of shared memory).
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <string>

#include "../../include/fdlbm.h"
#include "fdlbm_dd.cuh"
#include "fdlbm_internal.h"

namespace fdlbm {
namespace {

using dd::cdd;
using dd::dd_t;

constexpr int N = Q;  // matrix order: one row/column per velocity

struct VnShared {
  double2 re[N * N];  // (hi, lo) of Re G[i][j] at i * N + j
  double2 im[N * N];
  double2 v[2 * 32];  // Householder vector: v[2l] real part, v[2l + 1] imaginary part
};

__device__ __forceinline__ cdd ldA(const VnShared& S, int i, int j) {
  const double2 a = S.re[i * N + j], b = S.im[i * N + j];
  return {{a.x, a.y}, {b.x, b.y}};
}
__device__ __forceinline__ void stA(VnShared& S, int i, int j, const cdd& z) {
  S.re[i * N + j] = make_double2(z.re.hi, z.re.lo);
  S.im[i * N + j] = make_double2(z.im.hi, z.im.lo);
}
__device__ __forceinline__ dd_t ldd(const double2& a) { return {a.x, a.y}; }
__device__ __forceinline__ double2 std2(const dd_t& a) { return make_double2(a.hi, a.lo); }

__device__ __forceinline__ dd_t warp_sum(dd_t x) {
  // xor butterfly; the double-double add is commutative bit for bit, so every lane ends with the
  // same sum
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const dd_t y = {__shfl_xor_sync(0xffffffffu, x.hi, off), __shfl_xor_sync(0xffffffffu, x.lo, off)};
    x = dd::add(x, y);
  }
  return x;
}

// Velocity q of Eq. 1 in double-double: q = 0 rest, q = 1 + 8k + d for speed k and direction d at
// angle (d + 1) * 45 degrees. Axis directions have components 0, +-v_k; diagonals +-v_k sqrt(1/2),
// with sqrt(1/2) carried to double-double accuracy.
__device__ void velocity_dd(int q, dd_t* vx, dd_t* vy) {
  *vx = dd::make(0.0);
  *vy = dd::make(0.0);
  if (q == 0) return;
  const int k = (q - 1) / 8, d = (q - 1) % 8;
  const double sp = speed(k);
  const int xs = (d == 0 || d == 6 || d == 7) ? 1 : (d == 2 || d == 3 || d == 4) ? -1 : 0;
  const int ys = (d == 0 || d == 1 || d == 2) ? 1 : (d == 4 || d == 5 || d == 6) ? -1 : 0;
  const dd_t mag = (d % 2 == 0) ? dd::mul(dd_t{0.7071067811865476, -4.833646656726457e-17}, sp) : dd::make(sp);
  if (xs) *vx = xs > 0 ? mag : dd::neg(mag);
  if (ys) *vy = ys > 0 ? mag : dd::neg(mag);
}

// Diagonal symbol of Eq. 17 along one axis (Eq. 18 with e^{i xi}):
//   line I    -(c/2)(e - 1/e)                         = -i c sin xi
//   line II   (c^2/2)(e - 2 + 1/e)                      = c^2 (cos xi - 1)
//   line III  c(1 - c^2)/12 (e^2 - 2e + 2/e - 1/e^2)    = i c (1 - c^2)/6 (sin 2xi - 2 sin xi)
//   line IV   lambda |k|(1 - |k|)/2 (e - 2 + 1/e)       = lambda |k|(1 - |k|)(cos xi - 1)
__device__ cdd symbol(dd_t c, dd_t sn, dd_t cs, dd_t kap, double lam, int flags) {
  const dd_t cm1 = dd::add(cs, -1.0);
  cdd d = {dd::make(0.0), dd::neg(dd::mul(c, sn))};
  if (!(flags & F_NO_LW)) d.re = dd::add(d.re, dd::mul(dd::sqr(c), cm1));
  if (!(flags & F_NO_DISP)) {
    const dd_t s2 = dd::scale2(dd::mul(sn, cs), 2.0);
    const dd_t w = dd::div(dd::mul(c, dd::sub(dd::make(1.0), dd::sqr(c))), 6.0);
    d.im = dd::add(d.im, dd::mul(w, dd::sub(s2, dd::scale2(sn, 2.0))));
  }
  if (!(flags & F_NO_VISC)) {
    const dd_t ak = kap.hi < 0.0 ? dd::neg(kap) : kap;
    d.re = dd::add(d.re, dd::mul(dd::mul(dd::mul(ak, dd::sub(dd::make(1.0), ak)), lam), cm1));
  }
  return d;
}

// Eigenvalues of the 2 x 2 block [a b; c d]: (a + d)/2 +- sqrt(((a - d)/2)^2 + b c).
__device__ void eig2(const cdd& a, const cdd& b, const cdd& c, const cdd& d, cdd* m1, cdd* m2) {
  const cdd h = {dd::scale2(dd::sub(a.re, d.re), 0.5), dd::scale2(dd::sub(a.im, d.im), 0.5)};
  const cdd disc = dd::csqrt(dd::cadd(dd::cmul(h, h), dd::cmul(b, c)));
  const cdd m = {dd::scale2(dd::add(a.re, d.re), 0.5), dd::scale2(dd::add(a.im, d.im), 0.5)};
  *m1 = dd::cadd(m, disc);
  *m2 = dd::csub(m, disc);
}
// Wilkinson shift: the eigenvalue of the trailing 2 x 2 block closer to d.
__device__ cdd wilkinson(const cdd& a, const cdd& b, const cdd& c, const cdd& d) {
  cdd m1, m2;
  eig2(a, b, c, d, &m1, &m2);
  const double e1 = hypot(m1.re.hi - d.re.hi, m1.im.hi - d.im.hi);
  const double e2 = hypot(m2.re.hi - d.re.hi, m2.im.hi - d.im.hi);
  return e1 <= e2 ? m1 : m2;
}
__device__ __forceinline__ double l1_hi(const cdd& z) { return fabs(z.re.hi) + fabs(z.im.hi); }

// Plane rotation of rows (k, k+1): U = [a b; -conj(b) conj(a)] with a = conj(x)/r, b = conj(y)/r,
// r = sqrt(|x|^2 + |y|^2). U is unitary, maps (x, y) to (r, 0), and needs one reciprocal
// square root. Applied from the left to rows k, k+1, and as U^H from the right to columns k, k+1.
struct Rot {
  cdd a, b;
};
__device__ Rot givens(const cdd& x, const cdd& y) {
  const dd_t r2 = dd::add(dd::cabs2(x), dd::cabs2(y));
  Rot g;
  if (r2.hi == 0.0) {
    g.a = {dd::make(1.0), dd::make(0.0)};
    g.b = {dd::make(0.0), dd::make(0.0)};
    return g;
  }
  const dd_t rinv = dd::rsqrt(r2);
  g.a = dd::cmul(dd::cconj(x), rinv);
  g.b = dd::cmul(dd::cconj(y), rinv);
  return g;
}
// One output element of a rotation, one lane each: lane parity picks the output row (left
// product: new_k = a X + b Y, new_k+1 = -conj(b) X + conj(a) Y) or column (right product by U^H:
// new_k = conj(a) P + conj(b) Q, new_k+1 = -b P + a Q). Both lanes of a pair read the same two
// inputs, so the warp reads everything before anyone writes.
__device__ __forceinline__ void rot_coeffs_left(const Rot& g, bool second, cdd* al, cdd* be) {
  if (!second) {
    *al = g.a;
    *be = g.b;
  } else {
    *al = dd::cconj(g.b);
    al->re = dd::neg(al->re);
    al->im = dd::neg(al->im);
    *be = dd::cconj(g.a);
  }
}
__device__ __forceinline__ void rot_coeffs_right(const Rot& g, bool second, cdd* al, cdd* be) {
  if (!second) {
    *al = dd::cconj(g.a);
    *be = dd::cconj(g.b);
  } else {
    *al = {dd::neg(g.b.re), dd::neg(g.b.im)};
    *be = g.a;
  }
}
// rows (k, k+1) over columns j0 .. j1
__device__ __forceinline__ void rotate_rows(VnShared& S, const Rot& g, int k, int j0, int j1, int lane) {
  cdd al, be;
  rot_coeffs_left(g, lane & 1, &al, &be);
  const int row = k + (lane & 1);
  for (int base = j0; base <= j1; base += 16) {
    const int j = base + (lane >> 1);
    const bool act = j <= j1;
    cdd X, Y;
    if (act) {
      X = ldA(S, k, j);
      Y = ldA(S, k + 1, j);
    }
    __syncwarp();
    if (act) {
      cdd out = dd::cadd(dd::cmul(al, X), dd::cmul(be, Y));
      if (row == k + 1 && j == k) out = cdd{dd::make(0.0), dd::make(0.0)};  // the zeroed entry, exactly
      stA(S, row, j, out);
    }
    __syncwarp();
  }
}
// columns (k, k+1) over rows i0 .. i1, by U^H from the right
__device__ __forceinline__ void rotate_cols(VnShared& S, const Rot& g, int k, int i0, int i1, int lane) {
  cdd al, be;
  rot_coeffs_right(g, lane & 1, &al, &be);
  const int col = k + (lane & 1);
  for (int base = i0; base <= i1; base += 16) {
    const int i = base + (lane >> 1);
    const bool act = i <= i1;
    cdd P, Qv;
    if (act) {
      P = ldA(S, i, k);
      Qv = ldA(S, i, k + 1);
    }
    __syncwarp();
    if (act) stA(S, i, col, dd::cadd(dd::cmul(P, al), dd::cmul(Qv, be)));
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32) k_vn(const fdlbm_vn_case* __restrict__ cases, double dx, double dy,
                                           double dt, double tau, double* __restrict__ max_abs,
                                           double* __restrict__ omega, double* __restrict__ Gout,
                                           int* __restrict__ status) {
  __shared__ VnShared S;
  const long long cid = blockIdx.x;
  const int lane = threadIdx.x;
  const fdlbm_vn_case cs = cases[cid];
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  const bool ok = isfinite(cs.rho) && isfinite(cs.ux) && isfinite(cs.uy) && isfinite(cs.T) && cs.rho > 0.0 &&
                  cs.T > 0.0 && fabs(cs.xi_x) <= 8.0 && fabs(cs.xi_y) <= 8.0 && cs.lambda >= 0.0 &&
                  isfinite(cs.lambda) && (cs.flags & ~(F_NO_LW | F_NO_DISP | F_NO_VISC)) == 0 &&
                  cs.reserved == 0;
  if (!ok) {
    for (int q = lane; q < 2 * N; q += 32)
      if (omega) omega[66 * cid + q] = nan;
    if (Gout)
      for (int q = lane; q < 2 * N * N; q += 32) Gout[2178 * cid + q] = nan;
    if (lane == 0) {
      max_abs[cid] = nan;
      if (status) status[cid] = FDLBM_VN_BAD_CASE;
    }
    return;
  }

  // ---------------------------------------------------------------- 1. G (Eqs. 10-13, 18, 20)
  const dd_t n = dd::make(cs.rho), T = dd::make(cs.T), ux = dd::make(cs.ux), uy = dd::make(cs.uy);
  const dd_t r = dd::div(dd::make(dt), dd::make(tau));
  const dd_t kx = dd::div(dd::make(dt), dd::make(dx)), ky = dd::div(dd::make(dt), dd::make(dy));
  // Eqs. 11-13: F_k(T) and dF_k/dT with the cyclic index {k+l}; F_0 = 1 - 8 sum F_k
  dd_t F[5], dF[5];
  {
    const dd_t T2 = dd::sqr(T), T3 = dd::mul(T2, T), T4 = dd::sqr(T2);
    dd_t sF = dd::make(0.0), sdF = dd::make(0.0);
    for (int k = 0; k < 4; ++k) {
      const dd_t vk2 = dd::two_prod(speed(k), speed(k));
      const dd_t a = dd::two_prod(speed((k + 1) % 4), speed((k + 1) % 4));
      const dd_t b = dd::two_prod(speed((k + 2) % 4), speed((k + 2) % 4));
      const dd_t c = dd::two_prod(speed((k + 3) % 4), speed((k + 3) % 4));
      const dd_t D = dd::mul(dd::mul(vk2, dd::sub(vk2, a)), dd::mul(dd::sub(vk2, b), dd::sub(vk2, c)));
      const dd_t s1 = dd::add(dd::add(a, b), c);
      const dd_t s2 = dd::add(dd::add(dd::mul(a, b), dd::mul(b, c)), dd::mul(c, a));
      const dd_t s3q = dd::scale2(dd::mul(dd::mul(a, b), c), 0.25);
      // 48 T^4 - 6 s1 T^3 + s2 T^2 - (s3/4) T   and its derivative in T
      dd_t num = dd::mul(T4, 48.0);
      num = dd::sub(num, dd::mul(dd::mul(s1, T3), 6.0));
      num = dd::add(num, dd::mul(s2, T2));
      num = dd::sub(num, dd::mul(s3q, T));
      dd_t dnum = dd::mul(T3, 192.0);
      dnum = dd::sub(dnum, dd::mul(dd::mul(s1, T2), 18.0));
      dnum = dd::add(dnum, dd::scale2(dd::mul(s2, T), 2.0));
      dnum = dd::sub(dnum, s3q);
      F[k + 1] = dd::div(num, D);
      dF[k + 1] = dd::div(dnum, D);
      sF = dd::add(sF, F[k + 1]);
      sdF = dd::add(sdF, dF[k + 1]);
    }
    F[0] = dd::sub(dd::make(1.0), dd::scale2(sF, 8.0));
    dF[0] = dd::neg(dd::scale2(sdF, 8.0));
  }
  dd_t sx, cx_, sy, cy_;
  dd::sincos_dd(cs.xi_x, &sx, &cx_);
  dd::sincos_dd(cs.xi_y, &sy, &cy_);
  const dd_t kapx = dd::mul(ux, kx), kapy = dd::mul(uy, ky);  // Eq. 15
  const dd_t Tinv = dd::rcp(T), ninv = dd::rcp(n);
  const dd_t b = dd::scale2(dd::mul(dd::add(dd::sqr(ux), dd::sqr(uy)), Tinv), 0.5);  // u^2 / (2 theta)
  const dd_t omb = dd::sub(dd::make(1.0), b);
  cdd diag[2];
  // Row factors R0..R3 and column factors C1..C3, staged in rows 0..6 of the imaginary plane
  // (all zero in G away from the diagonal, so it is free until the diagonal is written).
  for (int t = 0; t < 2; ++t) {
    const int q = lane + 32 * t;
    if (q >= N) break;
    dd_t vx, vy;
    velocity_dd(q, &vx, &vy);
    const dd_t s = dd::mul(dd::add(dd::mul(vx, ux), dd::mul(vy, uy)), Tinv);  // v.u / theta
    const dd_t s2h = dd::scale2(dd::sqr(s), 0.5), s3 = dd::div(dd::mul(dd::sqr(s), s), 6.0);
    const dd_t s4 = dd::div(dd::sqr(dd::sqr(s)), 24.0);
    // Eq. 10 bracket P(s, b) and its partial derivatives in s and b
    const dd_t P = dd::add(dd::add(dd::mul(omb, dd::add(dd::add(dd::make(1.0), s), s2h)),
                                   dd::scale2(dd::sqr(b), 0.5)), dd::add(s3, s4));
    const dd_t Ps = dd::add(dd::add(dd::mul(omb, dd::add(s, 1.0)), s2h), dd::div(dd::mul(dd::sqr(s), s), 6.0));
    const dd_t Pb = dd::sub(dd::sub(dd::add(b, -1.0), s), s2h);
    const int ring = q == 0 ? 0 : 1 + (q - 1) / 8;
    const dd_t Fk = F[ring], dFk = dF[ring];
    const dd_t rn = dd::mul(r, n);
    // r f^eq / n;  r df/dT = r n (F' P - F (P_s s + P_b b) / theta);  r df/du_a = r n F (P_s v_a + P_b u_a) / theta
    const dd_t R0 = dd::mul(r, dd::mul(Fk, P));
    const dd_t R1 = dd::mul(rn, dd::sub(dd::mul(dFk, P), dd::mul(dd::mul(Fk, Tinv), dd::add(dd::mul(Ps, s), dd::mul(Pb, b)))));
    const dd_t g = dd::mul(rn, dd::mul(Fk, Tinv));
    const dd_t R2 = dd::mul(g, dd::add(dd::mul(Ps, vx), dd::mul(Pb, ux)));
    const dd_t R3 = dd::mul(g, dd::add(dd::mul(Ps, vy), dd::mul(Pb, uy)));
    // dT/df_j = (|v_j - u|^2 / 2 - T) / n,  du_a/df_j = (v_ja - u_a) / n
    const dd_t wx = dd::sub(vx, ux), wy = dd::sub(vy, uy);
    const dd_t C1 = dd::mul(dd::sub(dd::scale2(dd::add(dd::sqr(wx), dd::sqr(wy)), 0.5), T), ninv);
    const dd_t C2 = dd::mul(wx, ninv), C3 = dd::mul(wy, ninv);
    S.im[0 * N + q] = std2(R0);
    S.im[1 * N + q] = std2(R1);
    S.im[2 * N + q] = std2(R2);
    S.im[3 * N + q] = std2(R3);
    S.im[4 * N + q] = std2(C1);
    S.im[5 * N + q] = std2(C2);
    S.im[6 * N + q] = std2(C3);
    // diagonal: (1 - r) + symbols along x and y
    const cdd dxs = symbol(dd::mul(vx, kx), sx, cx_, kapx, cs.lambda, cs.flags);
    const cdd dys = symbol(dd::mul(vy, ky), sy, cy_, kapy, cs.lambda, cs.flags);
    diag[t] = dd::cadd(dxs, dys);
    diag[t].re = dd::add(diag[t].re, dd::sub(dd::make(1.0), r));
  }
  __syncwarp();
  for (int j = lane; j < N; j += 32) {
    const dd_t C1 = ldd(S.im[4 * N + j]), C2 = ldd(S.im[5 * N + j]), C3 = ldd(S.im[6 * N + j]);
    for (int i = 0; i < N; ++i) {
      dd_t gij = ldd(S.im[0 * N + i]);  // Eq. 20
      gij = dd::add(gij, dd::mul(ldd(S.im[1 * N + i]), C1));
      gij = dd::add(gij, dd::mul(ldd(S.im[2 * N + i]), C2));
      gij = dd::add(gij, dd::mul(ldd(S.im[3 * N + i]), C3));
      S.re[i * N + j] = std2(gij);
    }
  }
  __syncwarp();
  for (int j = lane; j < N; j += 32)
    for (int i = 0; i < N; ++i) S.im[i * N + j] = make_double2(0.0, 0.0);
  for (int t = 0; t < 2; ++t) {
    const int q = lane + 32 * t;
    if (q >= N) break;
    dd_t re = dd::add(ldd(S.re[q * N + q]), diag[t].re);
    S.re[q * N + q] = std2(re);
    S.im[q * N + q] = std2(diag[t].im);
  }
  __syncwarp();
  if (Gout) {
    for (int e = lane; e < N * N; e += 32) {
      Gout[2178 * cid + 2 * e] = S.re[e].x;
      Gout[2178 * cid + 2 * e + 1] = S.im[e].x;
    }
  }

  // ---------------------------------------------------------------- 2. Hessenberg reduction
  for (int k = 0; k < N - 2; ++k) {
    const int m = N - 1 - k;  // rows k+1 .. N-1; m <= 32
    cdd xl = {dd::make(0.0), dd::make(0.0)};
    if (lane < m) xl = ldA(S, k + 1 + lane, k);
    const dd_t sig = warp_sum(lane >= 1 && lane < m ? dd::cabs2(xl) : dd::make(0.0));
    if (sig.hi == 0.0) continue;  // column already reduced (uniform across the warp)
    const cdd x0 = ldA(S, k + 1, k);
    const dd_t ax0 = dd::cabs2(x0);
    const dd_t nrm = dd::sqrt(dd::add(ax0, sig));
    cdd alpha;  // -(x0/|x0|) ||x||
    if (ax0.hi == 0.0) {
      alpha = {dd::neg(nrm), dd::make(0.0)};
    } else {
      const dd_t t = dd::mul(dd::rsqrt(ax0), nrm);
      alpha = {dd::neg(dd::mul(x0.re, t)), dd::neg(dd::mul(x0.im, t))};
    }
    const cdd v0 = dd::csub(x0, alpha);
    const dd_t beta = dd::scale2(dd::rcp(dd::add(dd::cabs2(v0), sig)), 2.0);  // 2 / (v^H v)
    if (lane < m) {
      const cdd vl = lane == 0 ? v0 : xl;
      S.v[2 * lane] = std2(vl.re);
      S.v[2 * lane + 1] = std2(vl.im);
    }
    __syncwarp();
    // left: columns k+1 .. N-1 (lane l -> column k+1+l), A -= v (beta v^H A)
    if (lane < m) {
      const int j = k + 1 + lane;
      cdd w = {dd::make(0.0), dd::make(0.0)};
      for (int i = 0; i < m; ++i) {
        const cdd vi = {ldd(S.v[2 * i]), ldd(S.v[2 * i + 1])};
        w = dd::cadd(w, dd::cmulc(vi, ldA(S, k + 1 + i, j)));
      }
      w = dd::cmul(w, beta);
      for (int i = 0; i < m; ++i) {
        const cdd vi = {ldd(S.v[2 * i]), ldd(S.v[2 * i + 1])};
        stA(S, k + 1 + i, j, dd::csub(ldA(S, k + 1 + i, j), dd::cmul(vi, w)));
      }
    }
    // column k becomes (alpha, 0, ..., 0) below the diagonal
    if (lane < m) stA(S, k + 1 + lane, k, lane == 0 ? alpha : cdd{dd::make(0.0), dd::make(0.0)});
    __syncwarp();
    // right: A -= (beta A v) v^H. Rows 0..31 one per lane; row 32 by the whole warp (lane j takes
    // column k+1+j, the dot product is a warp sum), so no lane runs a second pass alone.
    {
      const int i = lane;
      cdd w = {dd::make(0.0), dd::make(0.0)};
      for (int j = 0; j < m; ++j) {
        const cdd vj = {ldd(S.v[2 * j]), ldd(S.v[2 * j + 1])};
        w = dd::cadd(w, dd::cmul(ldA(S, i, k + 1 + j), vj));
      }
      w = dd::cmul(w, beta);
      for (int j = 0; j < m; ++j) {
        const cdd vj = {ldd(S.v[2 * j]), ldd(S.v[2 * j + 1])};
        stA(S, i, k + 1 + j, dd::csub(ldA(S, i, k + 1 + j), dd::cmul(w, dd::cconj(vj))));
      }
    }
    {
      cdd t = {dd::make(0.0), dd::make(0.0)}, vl = {dd::make(0.0), dd::make(0.0)};
      if (lane < m) {
        vl = {ldd(S.v[2 * lane]), ldd(S.v[2 * lane + 1])};
        t = dd::cmul(ldA(S, N - 1, k + 1 + lane), vl);
      }
      const cdd w = dd::cmul(cdd{warp_sum(t.re), warp_sum(t.im)}, beta);
      if (lane < m) stA(S, N - 1, k + 1 + lane, dd::csub(ldA(S, N - 1, k + 1 + lane), dd::cmul(w, dd::cconj(vl))));
    }
    __syncwarp();
  }

  // ---------------------------------------------------------------- 3. shifted QR
  double hnorm = 0.0;  // max |h_ij| (FP64 parts), the scale of the deflation floor
  for (int e = lane; e < N * N; e += 32) hnorm = fmax(hnorm, fabs(S.re[e].x) + fabs(S.im[e].x));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) hnorm = fmax(hnorm, __shfl_xor_sync(0xffffffffu, hnorm, off));
  const double eps = 4.930380657631324e-32;  // 2^-104
  const double floor_abs = eps * hnorm;
  dd_t maxabs2 = dd::make(0.0);
  int st = FDLBM_VN_OK, hi = N - 1, its = 0, sweeps = 0;
  while (hi >= 0) {
    // the largest l <= hi whose subdiagonal entry is negligible (0 if none), lane l-1 testing l
    int l;
    {
      const int lt = lane + 1;
      bool negl = false;
      if (lt <= hi) {
        const double sub = l1_hi(ldA(S, lt, lt - 1));
        const double tst = l1_hi(ldA(S, lt - 1, lt - 1)) + l1_hi(ldA(S, lt, lt));
        negl = sub <= eps * tst || sub <= floor_abs;
      }
      const unsigned m = __ballot_sync(0xffffffffu, negl);
      l = m ? 32 - __clz((int)m) : 0;
    }
    const int lo = l;
    if (lo >= hi - 1) {  // a 1 x 1 or 2 x 2 block splits off: its eigenvalues directly
      cdd z[2];
      int cnt = 1;
      if (lo == hi) {
        z[0] = ldA(S, hi, hi);
      } else {
        eig2(ldA(S, hi - 1, hi - 1), ldA(S, hi - 1, hi), ldA(S, hi, hi - 1), ldA(S, hi, hi), &z[0], &z[1]);
        cnt = 2;
      }
      for (int t = 0; t < cnt; ++t) {
        const dd_t a2 = dd::cabs2(z[t]);
        if (a2.hi > maxabs2.hi || (a2.hi == maxabs2.hi && a2.lo > maxabs2.lo)) maxabs2 = a2;
        if (omega && lane == 0) {
          omega[66 * cid + 2 * (hi - t)] = z[t].re.hi;
          omega[66 * cid + 2 * (hi - t) + 1] = z[t].im.hi;
        }
      }
      hi -= cnt;
      its = 0;
      continue;
    }
    if (++sweeps > 30 * N) {
      st = FDLBM_VN_NO_CONVERGENCE;
      break;
    }
    ++its;
    cdd mu;
    if (its % 10 == 0) {  // exceptional shift
      mu = ldA(S, hi, hi);
      mu.re = dd::add(mu.re, 0.75 * l1_hi(ldA(S, hi, hi - 1)));
    } else {
      mu = wilkinson(ldA(S, hi - 1, hi - 1), ldA(S, hi - 1, hi), ldA(S, hi, hi - 1), ldA(S, hi, hi));
    }
    __syncwarp();
    for (int q = lo + lane; q <= hi; q += 32) stA(S, q, q, dd::csub(ldA(S, q, q), mu));
    __syncwarp();
    Rot prev;
    for (int k = lo; k < hi; ++k) {
      const Rot g = givens(ldA(S, k, k), ldA(S, k + 1, k));
      __syncwarp();
      rotate_rows(S, g, k, k, hi, lane);                // left rotation of rows k, k+1
      if (k > lo) rotate_cols(S, prev, k - 1, lo, k, lane);  // right rotation k-1 over rows lo..k
      prev = g;
    }
    rotate_cols(S, prev, hi - 1, lo, hi, lane);
    for (int q = lo + lane; q <= hi; q += 32) stA(S, q, q, dd::cadd(ldA(S, q, q), mu));
    __syncwarp();
  }
  if (st != FDLBM_VN_OK) {
    if (omega)
      for (int q = lane; q <= hi; q += 32) {
        omega[66 * cid + 2 * q] = nan;
        omega[66 * cid + 2 * q + 1] = nan;
      }
  }
  if (lane == 0) {
    max_abs[cid] = st == FDLBM_VN_OK ? dd::sqrt(maxabs2).hi : nan;
    if (status) status[cid] = st;
  }
}

int vn_fail(int code, const std::string& msg) {
  set_thread_error(msg.c_str());
  return code;
}

}  // namespace
}  // namespace fdlbm

extern "C" int fdlbm_vn_spectrum(const fdlbm_vn_case* cases, long long n, double dx, double dy, double dt,
                                 double tau, double* max_abs, double* omega, double* G, int* status,
                                 void* cuda_stream) {
  using namespace fdlbm;
  if (n < 0 || n > INT_MAX) return vn_fail(FDLBM_E_ARG, "fdlbm_vn_spectrum: n must be in [0, 2^31 - 1]");
  const double p[4] = {dx, dy, dt, tau};
  for (double x : p)
    if (!(std::isfinite(x) && x > 0.0))
      return vn_fail(FDLBM_E_ARG, "fdlbm_vn_spectrum: dx, dy, dt and tau must be finite and positive");
  if (n == 0) return FDLBM_OK;
  if (!cases || !max_abs) return vn_fail(FDLBM_E_ARG, "fdlbm_vn_spectrum: cases and max_abs are required");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_vn<<<(unsigned)n, 32, 0, s>>>(cases, dx, dy, dt, tau, max_abs, omega, G, status);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vn_fail(FDLBM_E_CUDA, std::string("fdlbm_vn_spectrum: ") + cudaGetErrorString(e));
  return FDLBM_OK;
}

/*
 * fdlbm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU restatement of the finite-difference lattice Boltzmann
 * method of Gan, Xu, Zhang, Yu and Li, "Two-Dimensional Lattice Boltzmann Model
 * for Compressible Flows with High Mach Number" (arXiv 0801.4169): the
 * Watari-Tsutahara 33-velocity model (Sec. 2, Eq. 1), its equilibrium
 * (Eqs. 10-13), and the modified Lax-Wendroff update with dispersion and
 * pressure-switched artificial viscosity (Sec. 3, Eqs. 15-17).
 *
 * It exists to check the CUDA path. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it. It shares no code, header,
 * table or constant with the CUDA library, and the product path never calls it.
 *
 * Build with -O2 -ffp-contract=off (no FMA contraction, fixed summation order
 * over q = 0..32), single thread.
 *
 * Every step follows the paper's order and notation:
 *   moments n, u, T, P at every site (Eqs. 3-5) ->
 *   F_k(theta), F_0 (Eqs. 11-13) -> f_eq (Eq. 10) ->
 *   Eq. 17 summed over alpha = x, y, with the relaxation term counted once ->
 *   ghost fill (Sec. 5 boundary kinds).
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *   - Eq. 10: all five bracket terms sit inside nF_k[...] (the printed bracket
 *     closes early; the reading makes f_eq the 4th-order expansion of
 *     exp((v.u - u^2/2)/theta)).
 *   - Moments (Eqs. 3-5) are taken of f, not f_eq (they agree for the
 *     conserved moments because relaxation conserves them).
 *   - m = 1, so theta = T and rho = n; P = nT.
 *   - The alpha-terms add unsplit (Einstein sum in Eq. 14); everything is
 *     explicit at time t.
 *   - Boundary mechanics (not given in the paper): ghost ring of width 2;
 *     periodic wrap; zero-gradient copies the nearest interior node; Dirichlet
 *     ghosts hold f_eq of the prescribed state; a specular wall mirrors node
 *     -1-j onto node j with the velocity direction reflected.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 33
#define NG 2 /* ghost width */

/* Flags (match oracle/fdlbm.py). Dropping lines II/III/IV of Eq. 17 gives the
 * scheme variants compared in Sec. 4 (Fig. 2, Fig. 3). */
#define ORC_NO_LW 1          /* drop line II (Lax-Wendroff dissipation)      */
#define ORC_NO_DISP 2        /* drop line III (dispersion)                   */
#define ORC_NO_VISC 4        /* drop line IV (artificial viscosity)          */
#define ORC_SWITCH_CONST 8   /* theta_alphaI := lambda (von Neumann reading) */

/* boundary kinds */
#define BC_PERIODIC 0
#define BC_OUTFLOW 1
#define BC_DIRICHLET 2
#define BC_WALL 3
#define BC_HALO 4 /* ghosts written by the caller (a neighbouring sub-domain), never by the fill */

/* ---------------------------------------------------------------------- */
/* Sec. 2, Eq. 1: v_0 = 0; v_ki = v_k (cos(i pi/4), sin(i pi/4)), i = 1..8.  */
/* q = 0 is rest; q = 1 + 8(k-1) + (i-1).                                    */
/* Speeds (v1..v4) = (1, 1.92, 2.99, 4.49), the values of Sec. 4 (Fig. 2).   */
/* Direction components are written exactly (0, +-1, +-sqrt(1/2)).           */
/* ---------------------------------------------------------------------- */
static const double SPEED[5] = {0.0, 1.0, 1.92, 2.99, 4.49};

static void direction(int i, double* cx, double* cy) {
  const double s = sqrt(0.5);
  switch (i) {
    case 1: *cx = s;    *cy = s;    break;  /* 45 deg  */
    case 2: *cx = 0.0;  *cy = 1.0;  break;  /* 90 deg  */
    case 3: *cx = -s;   *cy = s;    break;  /* 135 deg */
    case 4: *cx = -1.0; *cy = 0.0;  break;  /* 180 deg */
    case 5: *cx = -s;   *cy = -s;   break;  /* 225 deg */
    case 6: *cx = 0.0;  *cy = -1.0; break;  /* 270 deg */
    case 7: *cx = s;    *cy = -s;   break;  /* 315 deg */
    default: *cx = 1.0; *cy = 0.0;  break;  /* i = 8: 360 deg */
  }
}

void orc_velocities(double* vx, double* vy) {
  vx[0] = 0.0;
  vy[0] = 0.0;
  for (int k = 1; k <= 4; ++k)
    for (int i = 1; i <= 8; ++i) {
      double cx, cy;
      direction(i, &cx, &cy);
      int q = 1 + 8 * (k - 1) + (i - 1);
      vx[q] = SPEED[k] * cx;
      vy[q] = SPEED[k] * cy;
    }
}

/* ---------------------------------------------------------------------- */
/* Eqs. 11-13: F_k(theta), k = 1..4, cyclic index {k+l}; F_0 = 1 - 8 sum F_k */
/* ---------------------------------------------------------------------- */
static int cyc(int k, int l) { /* Eq. 13 */
  return (k + l <= 4) ? k + l : k + l - 4;
}

void orc_weights(double theta, double* F) {
  double sumF = 0.0;
  for (int k = 1; k <= 4; ++k) {
    double vk2 = SPEED[k] * SPEED[k];
    double a = SPEED[cyc(k, 1)] * SPEED[cyc(k, 1)];
    double b = SPEED[cyc(k, 2)] * SPEED[cyc(k, 2)];
    double c = SPEED[cyc(k, 3)] * SPEED[cyc(k, 3)];
    double denom = vk2 * (vk2 - a) * (vk2 - b) * (vk2 - c);
    double t2 = theta * theta, t3 = t2 * theta, t4 = t3 * theta;
    double numer = 48.0 * t4 - 6.0 * (a + b + c) * t3 + (a * b + b * c + c * a) * t2 -
                   (a * b * c) / 4.0 * theta;
    F[k] = numer / denom;
    sumF += F[k];
  }
  F[0] = 1.0 - 8.0 * sumF; /* Eq. 12 */
}

/* ---------------------------------------------------------------------- */
/* Eq. 10: f_ki^eq = n F_k [ (1 - u^2/2th + u^4/8th^2)                       */
/*                           + (v.u/th)(1 - u^2/2th)                         */
/*                           + (v.u)^2/(2th^2) (1 - u^2/2th)                 */
/*                           + (v.u)^3/(6th^3) + (v.u)^4/(24th^4) ]          */
/* with theta = T/m, m = 1.                                                  */
/* ---------------------------------------------------------------------- */
void orc_feq(double n, double ux, double uy, double T, double* feq) {
  double vx[Q], vy[Q], F[5];
  orc_velocities(vx, vy);
  double theta = T;
  orc_weights(theta, F);
  double u2 = ux * ux + uy * uy;
  for (int q = 0; q < Q; ++q) {
    int k = (q == 0) ? 0 : 1 + (q - 1) / 8;
    double vu = vx[q] * ux + vy[q] * uy;
    double term0 = 1.0 - u2 / (2.0 * theta) + (u2 * u2) / (8.0 * theta * theta);
    double term1 = (vu / theta) * (1.0 - u2 / (2.0 * theta));
    double term2 = (vu * vu) / (2.0 * theta * theta) * (1.0 - u2 / (2.0 * theta));
    double term3 = (vu * vu * vu) / (6.0 * theta * theta * theta);
    double term4 = (vu * vu * vu * vu) / (24.0 * theta * theta * theta * theta);
    feq[q] = n * F[k] * (term0 + term1 + term2 + term3 + term4);
  }
}

/* ---------------------------------------------------------------------- */
/* Eqs. 3-5: n = sum f; n u = sum v f; P = nT = sum (1/2)(v-u)^2 f.          */
/* ---------------------------------------------------------------------- */
void orc_moments(const double* f, double* n_out, double* ux_out, double* uy_out, double* T_out) {
  double vx[Q], vy[Q];
  orc_velocities(vx, vy);
  double n = 0.0, jx = 0.0, jy = 0.0;
  for (int q = 0; q < Q; ++q) {
    n += f[q];
    jx += vx[q] * f[q];
    jy += vy[q] * f[q];
  }
  double ux = jx / n, uy = jy / n;
  double P = 0.0;
  for (int q = 0; q < Q; ++q) {
    double wx = vx[q] - ux, wy = vy[q] - uy;
    P += 0.5 * (wx * wx + wy * wy) * f[q];
  }
  *n_out = n;
  *ux_out = ux;
  *uy_out = uy;
  *T_out = P / n;
}

/* ---------------------------------------------------------------------- */
/* Simulation state                                                         */
/* ---------------------------------------------------------------------- */
typedef struct {
  int nx, ny;
  double dx, dy, dt, tau, lambda;
  int bc[4];            /* left, right, bottom, top */
  double bstate[4][4];  /* Dirichlet (rho, u, v, T) per side */
  int flags;
  long steps_done;
  /* Optional Dirichlet segment per side (Sec. 5.2.2, double Mach reflection): the ghosts of the
   * side whose coordinate along it, (i + 1/2) dx or (j + 1/2) dy, lies below (lower = 1) or at or
   * above (lower = 0) the split c0 + speed * t hold f_eq of seg_state at time t; the rest of the
   * side follows its boundary kind. */
  int seg_on[4], seg_lower[4];
  double seg_c0[4], seg_speed[4], seg_state[4][4];
  int sx, sy;           /* padded extents nx+4, ny+4 */
  double* f;            /* [Q][sy][sx] */
  double* fn;
  double *n, *ux, *uy, *T; /* [sy][sx] macros (cross-shaped region valid) */
} orc_sim;

#define FI(s, q, i, j) ((size_t)(q) * (s)->sy * (s)->sx + (size_t)((j) + NG) * (s)->sx + (size_t)((i) + NG))
#define MI(s, i, j) ((size_t)((j) + NG) * (s)->sx + (size_t)((i) + NG))

static int mirror_q(int q, int axis) {
  /* specular reflection of direction i: y-wall maps i -> 8-i, x-wall maps i -> 4-i (mod 8) */
  if (q == 0) return 0;
  int k = 1 + (q - 1) / 8, i = 1 + (q - 1) % 8;
  int j = (axis == 1) ? (8 - i) : (4 - i);
  j = ((j % 8) + 8) % 8;
  if (j == 0) j = 8;
  return 1 + 8 * (k - 1) + (j - 1);
}

static int posmod(int a, int n) { return ((a % n) + n) % n; }

/* 1 if the ghost at along-side coordinate index a (node i or j) of `side` lies in the side's
 * Dirichlet segment at time t. */
static int in_segment(const orc_sim* s, int side, int a, double t) {
  if (!s->seg_on[side]) return 0;
  const double c = ((double)a + 0.5) * (side < 2 ? s->dy : s->dx);
  const double split = s->seg_c0[side] + s->seg_speed[side] * t;
  return s->seg_lower[side] ? (c < split) : !(c < split);
}

/* Fill the ghost ring of buffer g at time t: x-ghost columns on interior rows first,
 * then y-ghost rows across the full padded width. */
static void fill_ghosts(orc_sim* s, double* g, double t) {
  double vx[Q], vy[Q];
  orc_velocities(vx, vy);
  (void)vx; (void)vy;
  double fe[4][Q], fseg[4][Q];
  for (int side = 0; side < 4; ++side) {
    if (s->bc[side] == BC_DIRICHLET)
      orc_feq(s->bstate[side][0], s->bstate[side][1], s->bstate[side][2], s->bstate[side][3], fe[side]);
    if (s->seg_on[side])
      orc_feq(s->seg_state[side][0], s->seg_state[side][1], s->seg_state[side][2], s->seg_state[side][3], fseg[side]);
  }
  int nx = s->nx, ny = s->ny;
#define G(q, i, j) g[(size_t)(q) * s->sy * s->sx + (size_t)((j) + NG) * s->sx + (size_t)((i) + NG)]
  for (int j = 0; j < ny; ++j) {
    for (int gi = -NG; gi < 0 && s->bc[0] != BC_HALO; ++gi) { /* left */
      if (in_segment(s, 0, j, t)) {
        for (int q = 0; q < Q; ++q) G(q, gi, j) = fseg[0][q];
        continue;
      }
      for (int q = 0; q < Q; ++q) {
        switch (s->bc[0]) {
          case BC_PERIODIC: G(q, gi, j) = G(q, posmod(gi, nx), j); break;
          case BC_OUTFLOW: G(q, gi, j) = G(q, 0, j); break;
          case BC_DIRICHLET: G(q, gi, j) = fe[0][q]; break;
          default: G(q, gi, j) = G(mirror_q(q, 0), -1 - gi, j); break;
        }
      }
    }
    for (int gi = nx; gi < nx + NG && s->bc[1] != BC_HALO; ++gi) { /* right */
      if (in_segment(s, 1, j, t)) {
        for (int q = 0; q < Q; ++q) G(q, gi, j) = fseg[1][q];
        continue;
      }
      for (int q = 0; q < Q; ++q) {
        switch (s->bc[1]) {
          case BC_PERIODIC: G(q, gi, j) = G(q, posmod(gi, nx), j); break;
          case BC_OUTFLOW: G(q, gi, j) = G(q, nx - 1, j); break;
          case BC_DIRICHLET: G(q, gi, j) = fe[1][q]; break;
          default: G(q, gi, j) = G(mirror_q(q, 0), 2 * nx - 1 - gi, j); break;
        }
      }
    }
  }
  for (int i = -NG; i < nx + NG; ++i) {
    for (int gj = -NG; gj < 0 && s->bc[2] != BC_HALO; ++gj) { /* bottom */
      if (in_segment(s, 2, i, t)) {
        for (int q = 0; q < Q; ++q) G(q, i, gj) = fseg[2][q];
        continue;
      }
      for (int q = 0; q < Q; ++q) {
        switch (s->bc[2]) {
          case BC_PERIODIC: G(q, i, gj) = G(q, i, posmod(gj, ny)); break;
          case BC_OUTFLOW: G(q, i, gj) = G(q, i, 0); break;
          case BC_DIRICHLET: G(q, i, gj) = fe[2][q]; break;
          default: G(q, i, gj) = G(mirror_q(q, 1), i, -1 - gj); break;
        }
      }
    }
    for (int gj = ny; gj < ny + NG && s->bc[3] != BC_HALO; ++gj) { /* top */
      if (in_segment(s, 3, i, t)) {
        for (int q = 0; q < Q; ++q) G(q, i, gj) = fseg[3][q];
        continue;
      }
      for (int q = 0; q < Q; ++q) {
        switch (s->bc[3]) {
          case BC_PERIODIC: G(q, i, gj) = G(q, i, posmod(gj, ny)); break;
          case BC_OUTFLOW: G(q, i, gj) = G(q, i, ny - 1); break;
          case BC_DIRICHLET: G(q, i, gj) = fe[3][q]; break;
          default: G(q, i, gj) = G(mirror_q(q, 1), i, 2 * ny - 1 - gj); break;
        }
      }
    }
  }
#undef G
}

orc_sim* orc_create(int nx, int ny, double dx, double dy, double dt, double tau, double lambda,
                    const int* bc, const double* bstate /* 4x4 */, int flags) {
  if (nx < 1 || ny < 1) return NULL;
  for (int side = 0; side < 4; ++side) {
    if (bc[side] < 0 || bc[side] > 4) return NULL;
    if (bc[side] == BC_WALL && ((side < 2 && nx < 2) || (side >= 2 && ny < 2))) return NULL;
  }
  if ((bc[0] == BC_PERIODIC) != (bc[1] == BC_PERIODIC)) return NULL;
  if ((bc[2] == BC_PERIODIC) != (bc[3] == BC_PERIODIC)) return NULL;
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->nx = nx; s->ny = ny; s->dx = dx; s->dy = dy; s->dt = dt; s->tau = tau; s->lambda = lambda;
  memcpy(s->bc, bc, 4 * sizeof(int));
  if (bstate) memcpy(s->bstate, bstate, 16 * sizeof(double));
  s->flags = flags;
  s->sx = nx + 2 * NG;
  s->sy = ny + 2 * NG;
  size_t nf = (size_t)Q * s->sx * s->sy, nm = (size_t)s->sx * s->sy;
  s->f = (double*)calloc(nf, sizeof(double));
  s->fn = (double*)calloc(nf, sizeof(double));
  s->n = (double*)calloc(nm, sizeof(double));
  s->ux = (double*)calloc(nm, sizeof(double));
  s->uy = (double*)calloc(nm, sizeof(double));
  s->T = (double*)calloc(nm, sizeof(double));
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  free(s->f); free(s->fn); free(s->n); free(s->ux); free(s->uy); free(s->T);
  free(s);
}

/* initial f = f_eq(initial macros) on the interior, then the ghost ring */
void orc_set_macro(orc_sim* s, const double* rho, const double* u, const double* v, const double* T) {
  double fe[Q];
  for (int j = 0; j < s->ny; ++j)
    for (int i = 0; i < s->nx; ++i) {
      size_t m = (size_t)j * s->nx + i;
      orc_feq(rho[m], u[m], v[m], T[m], fe);
      for (int q = 0; q < Q; ++q) s->f[FI(s, q, i, j)] = fe[q];
    }
  s->steps_done = 0;
  fill_ghosts(s, s->f, 0.0);
}

/* A Dirichlet segment on `side` (see orc_sim); takes effect at the next ghost fill. */
int orc_set_segment(orc_sim* s, int side, double c0, double speed, int lower, const double* state) {
  if (side < 0 || side > 3) return -1;
  s->seg_on[side] = 1;
  s->seg_c0[side] = c0;
  s->seg_speed[side] = speed;
  s->seg_lower[side] = lower ? 1 : 0;
  for (int a = 0; a < 4; ++a) s->seg_state[side][a] = state[a];
  return 0;
}

/* raw f access, interior only, layout [q][j][i] (for perturbation tests) */
void orc_set_f(orc_sim* s, const double* f) {
  for (int q = 0; q < Q; ++q)
    for (int j = 0; j < s->ny; ++j)
      for (int i = 0; i < s->nx; ++i)
        s->f[FI(s, q, i, j)] = f[((size_t)q * s->ny + j) * s->nx + i];
  fill_ghosts(s, s->f, (double)s->steps_done * s->dt);
}

void orc_get_f(const orc_sim* s, double* f) {
  for (int q = 0; q < Q; ++q)
    for (int j = 0; j < s->ny; ++j)
      for (int i = 0; i < s->nx; ++i)
        f[((size_t)q * s->ny + j) * s->nx + i] = s->f[FI(s, q, i, j)];
}

/* full padded buffer (ghosts included), layout [q][j+2][i+2], written as given (no ghost fill):
 * a sub-domain's halo rows come from its neighbour */
void orc_set_f_padded(orc_sim* s, const double* f) {
  memcpy(s->f, f, (size_t)Q * s->sx * s->sy * sizeof(double));
}

/* full padded buffer (ghosts included), layout [q][j+2][i+2] */
void orc_get_f_padded(const orc_sim* s, double* f) {
  memcpy(f, s->f, (size_t)Q * s->sx * s->sy * sizeof(double));
}

static int site_needed(const orc_sim* s, int i, int j) {
  /* cross-shaped region: interior plus one ghost layer beside each edge (no corners) */
  int in_x = (i >= 0 && i < s->nx), in_y = (j >= 0 && j < s->ny);
  if (in_x && in_y) return 1;
  if (in_y && (i == -1 || i == s->nx)) return 1;
  if (in_x && (j == -1 || j == s->ny)) return 1;
  return 0;
}

/* One time step. Returns 0, or -4 if a needed site has non-finite moments or P <= 0. */
static int step_once(orc_sim* s) {
  double vx[Q], vy[Q];
  orc_velocities(vx, vy);
  int nx = s->nx, ny = s->ny;
  /* (1) moments, Eqs. 3-5 */
  double fq[Q];
  for (int j = -1; j <= ny; ++j)
    for (int i = -1; i <= nx; ++i) {
      if (!site_needed(s, i, j)) continue;
      for (int q = 0; q < Q; ++q) fq[q] = s->f[FI(s, q, i, j)];
      double n, ux, uy, T;
      orc_moments(fq, &n, &ux, &uy, &T);
      if (!isfinite(n) || !isfinite(ux) || !isfinite(uy) || !isfinite(T) || !(n > 0.0) || !(T > 0.0))
        return -4;
      size_t m = MI(s, i, j);
      s->n[m] = n; s->ux[m] = ux; s->uy[m] = uy; s->T[m] = T;
    }
  const double r = s->dt / s->tau;
  const double dr[2] = {s->dx, s->dy};
  double feq[Q];
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t m = MI(s, i, j);
      /* (2) equilibrium at the node, Eqs. 10-13 */
      orc_feq(s->n[m], s->ux[m], s->uy[m], s->T[m], feq);
      /* (3) switch theta_alphaI (Eq. 16) and kappa_alpha (Eq. 15) */
      double sw[2], kap[2];
      for (int a = 0; a < 2; ++a) {
        int di = (a == 0) ? 1 : 0, dj = (a == 0) ? 0 : 1;
        double Pp = s->n[MI(s, i + di, j + dj)] * s->T[MI(s, i + di, j + dj)];
        double P0 = s->n[m] * s->T[m];
        double Pm = s->n[MI(s, i - di, j - dj)] * s->T[MI(s, i - di, j - dj)];
        if (s->flags & ORC_SWITCH_CONST)
          sw[a] = s->lambda;
        else
          sw[a] = s->lambda * fabs((Pp - 2.0 * P0 + Pm) / (Pp + 2.0 * P0 + Pm));
        double ua = (a == 0) ? s->ux[m] : s->uy[m];
        kap[a] = ua * s->dt / dr[a];
      }
      /* (4) Eq. 17 for every velocity, summed over alpha = x, y */
      for (int q = 0; q < Q; ++q) {
        double f0 = s->f[FI(s, q, i, j)];
        double acc = f0 - r * (f0 - feq[q]);
        for (int a = 0; a < 2; ++a) {
          int di = (a == 0) ? 1 : 0, dj = (a == 0) ? 0 : 1;
          double fp1 = s->f[FI(s, q, i + di, j + dj)];
          double fm1 = s->f[FI(s, q, i - di, j - dj)];
          double fp2 = s->f[FI(s, q, i + 2 * di, j + 2 * dj)];
          double fm2 = s->f[FI(s, q, i - 2 * di, j - 2 * dj)];
          double va = (a == 0) ? vx[q] : vy[q];
          double c = va * s->dt / dr[a]; /* Eq. 15 */
          acc -= c / 2.0 * (fp1 - fm1);                                    /* line I  */
          if (!(s->flags & ORC_NO_LW))
            acc += c * c / 2.0 * (fp1 - 2.0 * f0 + fm1);                   /* line II */
          if (!(s->flags & ORC_NO_DISP))
            acc += c * (1.0 - c * c) / 12.0 * (fp2 - 2.0 * fp1 + 2.0 * fm1 - fm2); /* line III */
          if (!(s->flags & ORC_NO_VISC))
            acc += sw[a] * fabs(kap[a]) * (1.0 - fabs(kap[a])) / 2.0 * (fp1 - 2.0 * f0 + fm1); /* line IV */
        }
        s->fn[FI(s, q, i, j)] = acc;
      }
    }
  /* (5) ghost ring of the new field (at time (steps + 1) dt), then swap */
  fill_ghosts(s, s->fn, (double)(s->steps_done + 1) * s->dt);
  double* t = s->f;
  s->f = s->fn;
  s->fn = t;
  s->steps_done += 1;
  return 0;
}

int orc_step(orc_sim* s, long nsteps) {
  for (long k = 0; k < nsteps; ++k) {
    int rc = step_once(s);
    if (rc) return rc;
  }
  return 0;
}

long orc_steps_done(const orc_sim* s) { return s->steps_done; }

/* macros of the current f on the interior, x fastest */
void orc_get_macro(const orc_sim* s, double* rho, double* u, double* v, double* T) {
  double fq[Q];
  for (int j = 0; j < s->ny; ++j)
    for (int i = 0; i < s->nx; ++i) {
      for (int q = 0; q < Q; ++q) fq[q] = s->f[FI(s, q, i, j)];
      size_t m = (size_t)j * s->nx + i;
      orc_moments(fq, &rho[m], &u[m], &v[m], &T[m]);
    }
}

// fdlbm_capi.cu -- C ABI of include/fdlbm.h: handle life cycle, memory, checkpoints, and the
// launch sequence of each call. All numerical work runs in the kernels of fdlbm_step.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "../../include/fdlbm.h"
#include "fdlbm_internal.h"

using namespace fdlbm;



namespace {

thread_local std::string g_create_err;

}  // namespace

namespace fdlbm {
void set_thread_error(const char* msg) { g_create_err = msg; }
}  // namespace fdlbm

namespace {

int fail(fdlbm_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_fail(fdlbm_ctx* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (h) h->sticky = FDLBM_E_CUDA;
  return fail(h, FDLBM_E_CUDA, m);
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace fdlbm {

bool valid_cfg(const fdlbm_config* c, std::string* why) {
  if (!c) { *why = "config is NULL"; return false; }
  if (c->nx < 1 || c->ny < 1) { *why = "nx and ny must be >= 1"; return false; }
  if ((long long)c->nx * c->ny > (1LL << 31)) { *why = "nx*ny too large"; return false; }
  if (!(c->dx > 0) || !(c->dy > 0) || !(c->dt > 0) || !(c->tau > 0)) { *why = "dx, dy, dt, tau must be > 0"; return false; }
  if (!(c->lambda >= 0) || !std::isfinite(c->lambda)) { *why = "lambda must be finite and >= 0"; return false; }
  if (c->prec < FDLBM_FP64 || c->prec > FDLBM_FP64_STRICT) {
    *why = "prec must be FDLBM_FP64, FDLBM_FP32_STORE, FDLBM_FNEQ32, FDLBM_FP32_STORE_DW or FDLBM_FP64_STRICT";
    return false;
  }
  if (c->flags & ~15) { *why = "unknown flag bits"; return false; }
  for (int s = 0; s < 4; ++s)
    if (c->bc[s] < 0 || c->bc[s] > FDLBM_BC_HALO) { *why = "boundary kind out of range"; return false; }
  if ((c->bc[0] == FDLBM_BC_PERIODIC) != (c->bc[1] == FDLBM_BC_PERIODIC)) { *why = "periodic x needs both left and right periodic"; return false; }
  if ((c->bc[2] == FDLBM_BC_PERIODIC) != (c->bc[3] == FDLBM_BC_PERIODIC)) { *why = "periodic y needs both bottom and top periodic"; return false; }
  if ((c->bc[0] == FDLBM_BC_WALL || c->bc[1] == FDLBM_BC_WALL) && c->nx < 2) { *why = "a wall in x needs nx >= 2"; return false; }
  if ((c->bc[2] == FDLBM_BC_WALL || c->bc[3] == FDLBM_BC_WALL) && c->ny < 2) { *why = "a wall in y needs ny >= 2"; return false; }
  return true;
}

Layout layout_of(const fdlbm_config* c) {
  Layout L;
  L.g.nx = c->nx;
  L.g.ny = c->ny;
  L.g.pitch = (int)round_up((size_t)c->nx + 2 * NG, 32);
  L.g.rows = c->ny + 2 * NG;
  L.g.plane = (long long)L.g.pitch * L.g.rows;
  for (int s = 0; s < 4; ++s) L.g.bc[s] = c->bc[s];
  L.g.flags = c->flags;
  L.esize = f64_storage(c->prec) ? 8 : 4;
  L.fbytes = round_up((size_t)Q * L.g.plane * L.esize, 256);
  L.g.aux_off = 0;
  if (c->prec == FDLBM_FNEQ32) {  // 33 FP32 planes of g, then 4 FP64 planes n, ux, uy, T
    L.g.aux_off = (long long)L.fbytes;
    L.fbytes = round_up(L.fbytes + (size_t)4 * L.g.plane * sizeof(double), 256);
  }
  L.health_off = 2 * L.fbytes;
  L.stage_off = L.health_off + 256;
  L.mom_off = L.stage_off + round_up((size_t)4 * c->nx * c->ny * sizeof(double), 256);
  // moment buffer of the split step: 4 FP64 planes + P in the storage precision (the strict step
  // always goes through it)
  L.mom_bytes = ((long long)c->nx * c->ny > 65536 && c->prec != FDLBM_FNEQ32) || c->prec == FDLBM_FP64_STRICT
                    ? round_up((size_t)L.g.plane * (4 * sizeof(double) + L.esize), 256) : 0;
  L.total = L.mom_off + L.mom_bytes;
  L.g.mom = nullptr;  // set to the handle's buffer once its memory is known
  return L;
}

// Host-side constants of Eqs. 11 and 17 (FP64).
Coeffs make_coeffs(const fdlbm_config* cfg) {
  Coeffs c;
  std::memset(&c, 0, sizeof(c));
  const double v[4] = {speed(0), speed(1), speed(2), speed(3)};  // speeds v_1..v_4 (Sec. 4)
  for (int k = 0; k < 4; ++k) {
    // Eq. 11 with the cyclic index of Eq. 13
    const double vk2 = v[k] * v[k];
    const double a = v[(k + 1) % 4] * v[(k + 1) % 4];
    const double b = v[(k + 2) % 4] * v[(k + 2) % 4];
    const double cc = v[(k + 3) % 4] * v[(k + 3) % 4];
    const double D = vk2 * (vk2 - a) * (vk2 - b) * (vk2 - cc);
    c.Fh[k][3] = 48.0 / D;
    c.Fh[k][2] = -6.0 * (a + b + cc) / D;
    c.Fh[k][1] = (a * b + b * cc + cc * a) / D;
    c.Fh[k][0] = -(a * b * cc) / (4.0 * D);
    c.v[k] = v[k];
    c.v2[k] = vk2;
    c.v3_6[k] = vk2 * v[k] / 6.0;
    c.v4_24[k] = vk2 * vk2 / 24.0;
    c.v2h[k] = 0.5 * vk2;
  }
  const double kk[2] = {cfg->dt / cfg->dx, cfg->dt / cfg->dy};
  const double s = std::sqrt(0.5);
  const bool lw = !(cfg->flags & FDLBM_NO_LW), disp = !(cfg->flags & FDLBM_NO_DISP);
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 4; ++k)
      for (int l = 0; l < 2; ++l) {
        const double cc = v[k] * (l == 0 ? 1.0 : s) * kk[a];  // Eq. 15, positive direction
        const double c2h = lw ? 0.5 * cc * cc : 0.0;
        const double d = disp ? cc * (1.0 - cc * cc) / 12.0 : 0.0;
        c.W1[a][k][l] = -0.5 * cc + c2h - 2.0 * d;
        c.Wm1[a][k][l] = 0.5 * cc + c2h + 2.0 * d;
        c.D[a][k][l] = d;
        c.fW1[a][k][l] = (float)c.W1[a][k][l];
        c.fWm1[a][k][l] = (float)c.Wm1[a][k][l];
        c.fD[a][k][l] = (float)c.D[a][k][l];
      }
  for (int k = 0; k < 4; ++k) {
    const double cx = v[k] * kk[0], cy = v[k] * kk[1];
    c.C2[k][0] = lw ? cx * cx : 0.0;
    c.C2[k][1] = lw ? cy * cy : 0.0;
    c.C2[k][2] = lw ? 0.5 * (cx * cx + cy * cy) : 0.0;
    for (int l = 0; l < 3; ++l) c.fC2[k][l] = (float)c.C2[k][l];
  }
  c.r = cfg->dt / cfg->tau;
  c.fr = (float)c.r;
  c.kx = kk[0];
  c.ky = kk[1];
  c.lam = cfg->lambda;
  c.fkx = (float)c.kx;
  c.fky = (float)c.ky;
  c.flam = (float)c.lam;
  auto split = [](double x, float* out) {
    const float hi = (float)x;
    out[0] = hi;
    out[1] = (float)(x - (double)hi);
  };
  for (int k = 0; k < 4; ++k) {
    split(c.v[k], c.dv[k]);
    split(c.v2h[k], c.dv2h[k]);
    split(c.v3_6[k], c.dv3_6[k]);
    split(c.v4_24[k], c.dv4_24[k]);
    for (int i = 0; i < 4; ++i) split(c.Fh[k][i], c.dFh[k][i]);
  }
  split(c.r, c.dr);
  split(s, c.dkS);
  c.sdt = cfg->dt;
  c.stau = cfg->tau;
  c.sdr[0] = cfg->dx;
  c.sdr[1] = cfg->dy;
  return c;
}

int default_variant(const fdlbm_config* c) {
  const long long sites = (long long)c->nx * c->ny;
  if (c->prec == FDLBM_FNEQ32) return c->ny <= 4 ? V_T32x4 : V_T32x8;  // its own kernel (fdlbm_fneq.cu)
  if (c->prec == FDLBM_FP32_STORE_DW) return V_TMA32x8;  // fastest at every size measured (tiny grids: 32 x 8)
  // Small grids are latency-bound: four lanes per node win up to a few thousand sites (400 x 4:
  // 16 us per step against 32 us for the tiles), and lose by 1.3x at 16 000 sites, where the
  // tiles have reached their latency floor while the ring-parallel launch is throughput-bound.
  if (sites <= 6144) return V_RP8x4;
  // 4-row tubes (autotuned on a GB300, FP64 and FP32 storage): a 32 x 16 tile, whose phase 1
  // takes one round, is fastest up to ~16 000 sites, 16 x 4 up to ~32 000, then 32 x 4.
  if (c->ny <= 4) return sites <= 16000 ? V_T32x16 : sites <= 32000 ? V_T16x4 : V_T32x4;
  if (sites < 200000) return V_T32x8;
  return V_T32x16;
}

}  // namespace fdlbm

namespace {

// Collect a finished health copy, if any, into the sticky status.
void poll_health(fdlbm_ctx* h, bool wait) {
  if (!h->ev_pending) return;
  cudaError_t q = wait ? cudaEventSynchronize(h->ev) : cudaEventQuery(h->ev);
  if (q == cudaErrorNotReady) return;
  h->ev_pending = false;
  if (q != cudaSuccess) {
    cuda_fail(h, q, "device work of an earlier call failed");
    return;
  }
  h->health |= *h->h_health;
  if ((h->health & H_NUMERIC) && h->sticky == FDLBM_OK) {
    h->sticky = FDLBM_E_NUMERIC;
    h->err = "a node had non-finite moments, n <= 0 or T <= 0 (step count at detection unknown; <= steps_done)";
  }
  if ((h->health & H_TIMEOUT) && h->sticky == FDLBM_OK) {
    h->sticky = FDLBM_E_TIMEOUT;
    h->err = "a tile's tensor copy did not complete within the kernel's wait limit; that step wrote nothing there";
  }
}

int enqueue_health_copy(fdlbm_ctx* h) {
  cudaError_t e = cudaMemcpyAsync(h->h_health, h->d_health, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "health copy");
  e = cudaEventRecord(h->ev, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "event record");
  h->ev_pending = true;
  return FDLBM_OK;
}

bool any_segment(const fdlbm_ctx* h) { return h->seg_on[0] || h->seg_on[1] || h->seg_on[2] || h->seg_on[3]; }

// V_GRP8x4 applies (else its steps are launched one by one as V_RP8x4).
bool graph_ok(const fdlbm_ctx* h) {
  return (h->cfg.prec == FDLBM_FP64 || h->cfg.prec == FDLBM_FP32_STORE) && !any_segment(h);
}

// The executable graph of kGraphSteps ring-parallel steps starting from buffer `start`, captured on
// the handle's private stream the first time it is needed. The launches' arguments (buffers, grid,
// coefficients, health word) are fixed for the handle's life, so a graph stays valid until
// fdlbm_destroy. Capture launches nothing; a replay runs on the handle's stream.
int graph_exec(fdlbm_ctx* h, int start, cudaGraphExec_t* out) {
  if (h->gexec[start]) {
    *out = h->gexec[start];
    return FDLBM_OK;
  }
  cudaError_t e = cudaSuccess;
  if (!h->cap_stream) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(h, e, "capture stream");
  e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(h, e, "begin capture");
  int c = start;
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k, c = 1 - c)
    le = launch_step(h->cfg.prec, V_RP8x4, h->f[c], h->f[1 - c], h->grid, h->coeffs, h->d_health, h->cap_stream);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(h->cap_stream, &graph);  // ends the capture whatever happened inside
  if (le != cudaSuccess) e = le;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "step graph");
  h->gexec[start] = exec;
  *out = exec;
  return FDLBM_OK;
}

// The Dirichlet segments of every side at the time of step `steps_at` (t = steps_at * dt), in
// buffer buf.
int apply_segments(fdlbm_ctx* h, void* buf, long steps_at) {
  const double t = (double)steps_at * h->cfg.dt;
  for (int side = 0; side < 4; ++side) {
    if (!h->seg_on[side]) continue;
    Segment sg;
    sg.side = side;
    sg.lower = h->seg_lower[side];
    sg.base_dirichlet = h->cfg.bc[side] == FDLBM_BC_DIRICHLET;
    sg.split = h->seg_c0[side] + h->seg_speed[side] * t;
    for (int a = 0; a < 4; ++a) {
      sg.seg[a] = h->seg_state[side][a];
      sg.base[a] = h->bstate[side][a];
    }
    cudaError_t e = h->cfg.prec == FDLBM_FNEQ32
                        ? launch_segment_fneq(buf, h->grid, sg, h->cfg.dx, h->cfg.dy, h->stream)
                        : launch_segment(h->cfg.prec, buf, h->grid, h->coeffs, sg, h->cfg.dx, h->cfg.dy, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "segment launch");
  }
  return FDLBM_OK;
}

// Dirichlet ghosts of both buffers (and the segments, at the time of step steps_at).
int fill_ghosts_dirichlet(fdlbm_ctx* h, long steps_at) {
  for (int b = 0; b < 2; ++b) {
    cudaError_t e = h->cfg.prec == FDLBM_FNEQ32 ? launch_dirichlet_fneq(h->f[b], h->grid, h->bstate, h->stream)
                                                : launch_dirichlet(h->cfg.prec, h->f[b], h->grid, h->coeffs, h->bstate,
                                                                   h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "dirichlet launch");
    int rc = apply_segments(h, h->f[b], steps_at);
    if (rc) return rc;
  }
  return FDLBM_OK;
}

int init_from_device_macros(fdlbm_ctx* h, const double* rho, const double* u, const double* v, const double* T) {
  poll_health(h, true);
  cudaError_t e = cudaMemsetAsync(h->d_health, 0, sizeof(unsigned), h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "health reset");
  // The current buffer gets f_eq with its ghost ring. The other one needs only its Dirichlet ghosts
  // and segments (fill_ghosts_dirichlet writes both buffers'): the first step writes its interior
  // and every ghost an interior node owns, halo ghosts come from the caller, and ghost corners are
  // never read.
  e = h->cfg.prec == FDLBM_FNEQ32 ? launch_init_fneq(h->f[0], h->grid, h->coeffs, rho, u, v, T, h->stream)
                                  : launch_init(h->cfg.prec, h->f[0], h->grid, h->coeffs, rho, u, v, T, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "init launch");
  int rc = fill_ghosts_dirichlet(h, 0);
  if (rc) return rc;
  h->cur = 0;
  h->steps = 0;
  h->health = 0;
  *h->h_health = 0;
  h->sticky = FDLBM_OK;
  h->initialised = true;
  return FDLBM_OK;
}

int ensure_fstage(fdlbm_ctx* h, size_t ndoubles) {
  if (h->d_fstage && h->fstage_cap >= ndoubles) return FDLBM_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "staging sync");
  if (h->d_fstage) cudaFree(h->d_fstage);
  h->d_fstage = nullptr;
  h->fstage_cap = 0;
  e = cudaMalloc(&h->d_fstage, ndoubles * sizeof(double));
  if (e != cudaSuccess) {
    h->d_fstage = nullptr;
    cudaGetLastError();
    return fail(h, FDLBM_E_OOM, "cannot allocate the f staging buffer");
  }
  h->fstage_cap = ndoubles;
  return FDLBM_OK;
}

size_t full_f_doubles(const fdlbm_ctx* h) { return (size_t)Q * h->cfg.nx * h->cfg.ny; }

struct CkptHeader {
  char magic[8];
  int version, nx, ny, prec, flags, bc[4], pitch, rows;
  double dx, dy, dt, tau, lambda;
  double bstate[4][4];
  long long steps;
  unsigned health;
  unsigned long long fbytes;
};

}  // namespace

extern "C" {

size_t fdlbm_device_bytes(const fdlbm_config* cfg) {
  std::string why;
  if (!valid_cfg(cfg, &why)) return 0;
  return layout_of(cfg).total;
}

int fdlbm_create_ex(fdlbm_t* out, const fdlbm_config* cfg, void* device_mem, size_t device_bytes, void* cuda_stream) {
  if (!out) return fail(nullptr, FDLBM_E_ARG, "out is NULL");
  *out = nullptr;
  std::string why;
  if (!valid_cfg(cfg, &why)) return fail(nullptr, FDLBM_E_ARG, why);
  Layout L = layout_of(cfg);
  if (device_mem && (device_bytes < L.total || ((uintptr_t)device_mem & 255)))
    return fail(nullptr, FDLBM_E_OOM, "caller device memory smaller than fdlbm_device_bytes() or not 256-byte aligned");
  fdlbm_ctx* h = new (std::nothrow) fdlbm_ctx();
  if (!h) return fail(nullptr, FDLBM_E_OOM, "host allocation failed");
  h->cfg = *cfg;
  h->grid = L.g;
  h->coeffs = make_coeffs(cfg);
  h->esize = L.esize;
  h->fbytes = L.fbytes;
  h->total = L.total;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->variant = default_variant(cfg);
  for (int s = 0; s < 4; ++s) {
    h->bstate[s][0] = 1.0;
    h->bstate[s][1] = 0.0;
    h->bstate[s][2] = 0.0;
    h->bstate[s][3] = 1.0;
  }
  cudaError_t e;
  if (device_mem) {
    h->mem = static_cast<unsigned char*>(device_mem);
  } else {
    e = cudaMalloc(&h->mem, L.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return fail(nullptr, FDLBM_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->owns_mem = true;
  }
  h->f[0] = h->mem;
  h->f[1] = h->mem + L.fbytes;
  h->d_health = reinterpret_cast<unsigned*>(h->mem + L.health_off);
  h->d_bar = reinterpret_cast<unsigned*>(h->mem + L.health_off + 64);
  h->d_stage = reinterpret_cast<double*>(h->mem + L.stage_off);
  h->grid.mom = L.mom_bytes ? static_cast<void*>(h->mem + L.mom_off) : nullptr;
  e = cudaMallocHost(&h->h_health, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->mem, 0, 2 * L.fbytes + 256, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    std::string m = std::string("create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    fdlbm_destroy(h);
    return fail(nullptr, FDLBM_E_CUDA, m);
  }
  *h->h_health = 0;
  *out = h;
  return FDLBM_OK;
}

int fdlbm_create(fdlbm_t* out, int nx, int ny, double dx, double dy, double dt, double tau, double lambda,
                 const int bc[4], int prec, void* cuda_stream) {
  if (!bc) return fail(nullptr, FDLBM_E_ARG, "bc is NULL");
  fdlbm_config c;
  std::memset(&c, 0, sizeof(c));
  c.nx = nx;
  c.ny = ny;
  c.dx = dx;
  c.dy = dy;
  c.dt = dt;
  c.tau = tau;
  c.lambda = lambda;
  for (int s = 0; s < 4; ++s) c.bc[s] = bc[s];
  c.prec = prec;
  c.flags = 0;
  return fdlbm_create_ex(out, &c, nullptr, 0, cuda_stream);
}

int fdlbm_set_boundary_state(fdlbm_t h, int side, double rho, double u, double v, double T) {
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (side < 0 || side > 3) return fail(h, FDLBM_E_ARG, "side out of range");
  if (!(rho > 0) || !(T > 0) || !std::isfinite(u) || !std::isfinite(v) || !std::isfinite(rho) || !std::isfinite(T))
    return fail(h, FDLBM_E_ARG, "boundary state needs finite rho > 0, T > 0");
  h->bstate[side][0] = rho;
  h->bstate[side][1] = u;
  h->bstate[side][2] = v;
  h->bstate[side][3] = T;
  if (h->cfg.bc[side] == FDLBM_BC_DIRICHLET && h->initialised) return fill_ghosts_dirichlet(h, h->steps);
  return FDLBM_OK;
}

int fdlbm_set_boundary_segment(fdlbm_t h, int side, double c0, double speed, int lower, double rho, double u,
                               double v, double T) {
  if (h && h->batch) return fail(h, FDLBM_E_STATE, "the solve is a member of a batch (remove it first)");
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (side < 0 || side > 3) return fail(h, FDLBM_E_ARG, "side out of range");
  if (h->cfg.bc[side] == FDLBM_BC_PERIODIC || h->cfg.bc[side] == FDLBM_BC_HALO)
    return fail(h, FDLBM_E_ARG, "a periodic or halo side takes no segment");
  if (!std::isfinite(c0) || !std::isfinite(speed)) return fail(h, FDLBM_E_ARG, "c0 and speed must be finite");
  if (!(rho > 0) || !(T > 0) || !std::isfinite(u) || !std::isfinite(v) || !std::isfinite(rho) || !std::isfinite(T))
    return fail(h, FDLBM_E_ARG, "segment state needs finite rho > 0, T > 0");
  h->seg_on[side] = true;
  h->seg_lower[side] = lower ? 1 : 0;
  h->seg_c0[side] = c0;
  h->seg_speed[side] = speed;
  h->seg_state[side][0] = rho;
  h->seg_state[side][1] = u;
  h->seg_state[side][2] = v;
  h->seg_state[side][3] = T;
  if (h->initialised) return fill_ghosts_dirichlet(h, h->steps);
  return FDLBM_OK;
}

int fdlbm_clear_boundary_segment(fdlbm_t h, int side) {
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (side < 0 || side > 3) return fail(h, FDLBM_E_ARG, "side out of range");
  h->seg_on[side] = false;
  return FDLBM_OK;
}

int fdlbm_set_macro_device(fdlbm_t h, const double* rho, const double* u, const double* v, const double* T) {
  if (h && h->batch) return fail(h, FDLBM_E_STATE, "the solve is a member of a batch (step it with fdlbm_batch_step, or remove it first)");
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (!rho || !u || !v || !T) return fail(h, FDLBM_E_ARG, "NULL macro array");
  return init_from_device_macros(h, rho, u, v, T);
}

int fdlbm_set_macro(fdlbm_t h, const double* rho, const double* u, const double* v, const double* T) {
  if (h && h->batch) return fail(h, FDLBM_E_STATE, "the solve is a member of a batch (step it with fdlbm_batch_step, or remove it first)");
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (!rho || !u || !v || !T) return fail(h, FDLBM_E_ARG, "NULL macro array");
  const size_t n = (size_t)h->cfg.nx * h->cfg.ny;
  const double* src[4] = {rho, u, v, T};
  poll_health(h, true);
  for (int a = 0; a < 4; ++a) {
    cudaError_t e = cudaMemcpyAsync(h->d_stage + a * n, src[a], n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_macro copy");
  }
  int rc = init_from_device_macros(h, h->d_stage, h->d_stage + n, h->d_stage + 2 * n, h->d_stage + 3 * n);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(h->stream);  // caller's host arrays may go away on return
  if (e != cudaSuccess) return cuda_fail(h, e, "set_macro");
  return FDLBM_OK;
}

int fdlbm_step(fdlbm_t h, long nsteps) {
  if (h && h->batch) return fail(h, FDLBM_E_STATE, "the solve is a member of a batch (step it with fdlbm_batch_step, or remove it first)");
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (nsteps < 0) return fail(h, FDLBM_E_ARG, "nsteps < 0");
  if (!h->initialised) return fail(h, FDLBM_E_STATE, "fdlbm_step before fdlbm_set_macro / fdlbm_load");
  poll_health(h, false);
  if (h->sticky) return h->sticky;
  if (variant_persistent(h->variant) && !any_segment(h) &&
      (h->cfg.prec == FDLBM_FP64 || h->cfg.prec == FDLBM_FP32_STORE)) {
    for (long done = 0; done < nsteps;) {
      const int k = (int)(nsteps - done < kPersistMaxSteps ? nsteps - done : kPersistMaxSteps);
      cudaError_t e = launch_steps_persist(h->cfg.prec, h->variant, h->f[h->cur], h->f[1 - h->cur], k, h->grid,
                                           h->coeffs, h->d_health, h->d_bar, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "persistent step launch");
      if (k & 1) h->cur = 1 - h->cur;
      h->steps += k;
      done += k;
    }
    if (nsteps > 0) return enqueue_health_copy(h);
    return FDLBM_OK;
  }
  long left = nsteps;
  if (variant_graph(h->variant) && graph_ok(h)) {
    for (; left >= kGraphSteps; left -= kGraphSteps) {
      cudaGraphExec_t ge = nullptr;
      const int rc = graph_exec(h, h->cur, &ge);
      if (rc) return rc;
      const cudaError_t e = cudaGraphLaunch(ge, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "step graph launch");
      h->steps += kGraphSteps;  // an even count: the state is back in buffer cur
    }
  }
  for (long s = 0; s < left; ++s) {
    cudaError_t e = launch_step(h->cfg.prec, h->variant, h->f[h->cur], h->f[1 - h->cur], h->grid, h->coeffs,
                                h->d_health, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
    h->cur = 1 - h->cur;
    h->steps += 1;
    if (any_segment(h)) {
      const int rc = apply_segments(h, h->f[h->cur], h->steps);
      if (rc) return rc;
    }
  }
  // health bits accumulate on the device, so a newer copy supersedes a pending one
  if (nsteps > 0) return enqueue_health_copy(h);
  return FDLBM_OK;
}

int fdlbm_sync(fdlbm_t h) {
  if (h && h->batch) {
    cudaError_t fe = batch_fence(h->batch);
    if (fe != cudaSuccess) return cuda_fail(h, fe, "batch fence");
  }
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (h->initialised) {
    int rc = enqueue_health_copy(h);
    if (rc) return rc;
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sync");
  poll_health(h, true);
  return h->sticky;
}

int fdlbm_get_macro_device(fdlbm_t h, double* rho, double* u, double* v, double* T) {
  if (h && h->batch) {
    cudaError_t fe = batch_fence(h->batch);
    if (fe != cudaSuccess) return cuda_fail(h, fe, "batch fence");
  }
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (!rho || !u || !v || !T) return fail(h, FDLBM_E_ARG, "NULL macro array");
  if (!h->initialised) return fail(h, FDLBM_E_STATE, "no state yet");
  cudaError_t e = h->cfg.prec == FDLBM_FNEQ32 ? launch_macro_fneq(h->f[h->cur], h->grid, rho, u, v, T, h->stream)
                                              : launch_macro(h->cfg.prec, h->f[h->cur], h->grid, rho, u, v, T, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "macro launch");
  return FDLBM_OK;
}

int fdlbm_get_macro(fdlbm_t h, double* rho, double* u, double* v, double* T) {
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (!rho || !u || !v || !T) return fail(h, FDLBM_E_ARG, "NULL macro array");
  if (!h->initialised) return fail(h, FDLBM_E_STATE, "no state yet");
  const size_t n = (size_t)h->cfg.nx * h->cfg.ny;
  int rc = fdlbm_get_macro_device(h, h->d_stage, h->d_stage + n, h->d_stage + 2 * n, h->d_stage + 3 * n);
  if (rc) return rc;
  double* dst[4] = {rho, u, v, T};
  for (int a = 0; a < 4; ++a) {
    cudaError_t e = cudaMemcpyAsync(dst[a], h->d_stage + a * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_macro copy");
  }
  return fdlbm_sync(h);
}

int fdlbm_get_f(fdlbm_t h, double* f) {
  if (h && h->batch) {
    cudaError_t fe = batch_fence(h->batch);
    if (fe != cudaSuccess) return cuda_fail(h, fe, "batch fence");
  }
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (!f) return fail(h, FDLBM_E_ARG, "f is NULL");
  if (!h->initialised) return fail(h, FDLBM_E_STATE, "no state yet");
  int rc = ensure_fstage(h, full_f_doubles(h));
  if (rc) return rc;
  cudaError_t e = h->cfg.prec == FDLBM_FNEQ32
                      ? launch_get_region_fneq(h->f[h->cur], h->grid, h->coeffs, 0, 0, h->cfg.nx, h->cfg.ny,
                                               h->d_fstage, h->stream)
                      : launch_get_f(h->cfg.prec, h->f[h->cur], h->grid, h->d_fstage, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_f launch");
  e = cudaMemcpyAsync(f, h->d_fstage, (size_t)Q * h->cfg.nx * h->cfg.ny * sizeof(double), cudaMemcpyDeviceToHost,
                      h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_f copy");
  return fdlbm_sync(h);
}

int fdlbm_get_f_region(fdlbm_t h, int x0, int y0, int w, int hgt, double* f) {
  if (h && h->batch) {
    cudaError_t fe = batch_fence(h->batch);
    if (fe != cudaSuccess) return cuda_fail(h, fe, "batch fence");
  }
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (!f) return fail(h, FDLBM_E_ARG, "f is NULL");
  if (!h->initialised) return fail(h, FDLBM_E_STATE, "no state yet");
  if (w < 1 || hgt < 1 || x0 < -NG || y0 < -NG || (long long)x0 + w > (long long)h->cfg.nx + NG ||
      (long long)y0 + hgt > (long long)h->cfg.ny + NG)
    return fail(h, FDLBM_E_ARG, "region outside the padded grid [-2, n+2)");
  const size_t nd = (size_t)Q * w * hgt;
  int rc = ensure_fstage(h, nd);
  if (rc) return rc;
  cudaError_t e = h->cfg.prec == FDLBM_FNEQ32
                      ? launch_get_region_fneq(h->f[h->cur], h->grid, h->coeffs, x0, y0, w, hgt, h->d_fstage, h->stream)
                      : launch_get_region(h->cfg.prec, h->f[h->cur], h->grid, x0, y0, w, hgt, h->d_fstage, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_f_region launch");
  e = cudaMemcpyAsync(f, h->d_fstage, nd * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_f_region copy");
  return fdlbm_sync(h);
}

int fdlbm_set_f(fdlbm_t h, const double* f) {
  if (h && h->batch) return fail(h, FDLBM_E_STATE, "the solve is a member of a batch (step it with fdlbm_batch_step, or remove it first)");
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (!f) return fail(h, FDLBM_E_ARG, "f is NULL");
  int rc = ensure_fstage(h, full_f_doubles(h));
  if (rc) return rc;
  poll_health(h, true);
  cudaError_t e = cudaMemcpyAsync(h->d_fstage, f, (size_t)Q * h->cfg.nx * h->cfg.ny * sizeof(double),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_f copy");
  if (!h->initialised) {
    e = cudaMemsetAsync(h->mem, 0, 2 * h->fbytes, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_f clear");
  }
  for (int b = 0; b < 2; ++b) {
    e = h->cfg.prec == FDLBM_FNEQ32 ? launch_set_f_fneq(h->f[b], h->grid, h->coeffs, h->d_fstage, h->stream)
                                    : launch_set_f(h->cfg.prec, h->f[b], h->grid, h->d_fstage, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_f launch");
  }
  rc = fill_ghosts_dirichlet(h, h->steps);
  if (rc) return rc;
  e = cudaMemsetAsync(h->d_health, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_f");
  h->initialised = true;
  h->health = 0;
  h->sticky = FDLBM_OK;
  return FDLBM_OK;
}

int fdlbm_save(fdlbm_t h, const char* path) {
  if (h && h->batch) {
    cudaError_t fe = batch_fence(h->batch);
    if (fe != cudaSuccess) return cuda_fail(h, fe, "batch fence");
  }
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (!path) return fail(h, FDLBM_E_ARG, "path is NULL");
  if (!h->initialised) return fail(h, FDLBM_E_STATE, "no state yet");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "save sync");
  poll_health(h, true);
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "FDLBMCK1", 8);
  hd.version = 1;
  hd.nx = h->cfg.nx;
  hd.ny = h->cfg.ny;
  hd.prec = h->cfg.prec;
  hd.flags = h->cfg.flags;
  for (int s = 0; s < 4; ++s) hd.bc[s] = h->cfg.bc[s];
  hd.pitch = h->grid.pitch;
  hd.rows = h->grid.rows;
  hd.dx = h->cfg.dx;
  hd.dy = h->cfg.dy;
  hd.dt = h->cfg.dt;
  hd.tau = h->cfg.tau;
  hd.lambda = h->cfg.lambda;
  std::memcpy(hd.bstate, h->bstate, sizeof(hd.bstate));
  hd.steps = h->steps;
  hd.health = h->health;
  hd.fbytes = h->fbytes;
  void* host = std::malloc(h->fbytes);
  if (!host) return fail(h, FDLBM_E_OOM, "host buffer for checkpoint");
  e = cudaMemcpy(host, h->f[h->cur], h->fbytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    std::free(host);
    return cuda_fail(h, e, "save copy");
  }
  FILE* fp = std::fopen(path, "wb");
  bool ok = fp && std::fwrite(&hd, sizeof(hd), 1, fp) == 1 && std::fwrite(host, 1, h->fbytes, fp) == h->fbytes;
  if (fp) ok = (std::fclose(fp) == 0) && ok;
  std::free(host);
  if (!ok) return fail(h, FDLBM_E_IO, std::string("cannot write ") + path);
  return FDLBM_OK;
}

int fdlbm_load(fdlbm_t h, const char* path) {
  if (h && h->batch) return fail(h, FDLBM_E_STATE, "the solve is a member of a batch (step it with fdlbm_batch_step, or remove it first)");
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (!path) return fail(h, FDLBM_E_ARG, "path is NULL");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(h, FDLBM_E_IO, std::string("cannot open ") + path);
  CkptHeader hd;
  bool ok = std::fread(&hd, sizeof(hd), 1, fp) == 1 && std::memcmp(hd.magic, "FDLBMCK1", 8) == 0 && hd.version == 1;
  ok = ok && hd.nx == h->cfg.nx && hd.ny == h->cfg.ny && hd.prec == h->cfg.prec && hd.flags == h->cfg.flags &&
       hd.pitch == h->grid.pitch && hd.rows == h->grid.rows && hd.fbytes == h->fbytes && hd.dx == h->cfg.dx &&
       hd.dy == h->cfg.dy && hd.dt == h->cfg.dt && hd.tau == h->cfg.tau && hd.lambda == h->cfg.lambda;
  for (int s = 0; s < 4 && ok; ++s) ok = hd.bc[s] == h->cfg.bc[s];
  if (!ok) {
    std::fclose(fp);
    return fail(h, FDLBM_E_IO, "checkpoint does not match this handle's configuration");
  }
  void* host = std::malloc(h->fbytes);
  if (!host) {
    std::fclose(fp);
    return fail(h, FDLBM_E_OOM, "host buffer for checkpoint");
  }
  ok = std::fread(host, 1, h->fbytes, fp) == h->fbytes;
  std::fclose(fp);
  if (!ok) {
    std::free(host);
    return fail(h, FDLBM_E_IO, "truncated checkpoint");
  }
  poll_health(h, true);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(h->f[0], host, h->fbytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->f[1], host, h->fbytes, cudaMemcpyHostToDevice);
  std::free(host);
  if (e != cudaSuccess) return cuda_fail(h, e, "load copy");
  std::memcpy(h->bstate, hd.bstate, sizeof(h->bstate));
  h->cur = 0;
  h->steps = hd.steps;
  h->health = hd.health;
  *h->h_health = 0;
  e = cudaMemsetAsync(h->d_health, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "load");
  h->initialised = true;
  h->sticky = (h->health & H_NUMERIC) ? FDLBM_E_NUMERIC : FDLBM_OK;
  return FDLBM_OK;
}

int fdlbm_variant_count(void) { return V_COUNT; }

int fdlbm_set_variant(fdlbm_t h, int variant) {
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (variant < 0 || variant >= V_COUNT) return fail(h, FDLBM_E_ARG, "variant out of range");
  if (variant_needs_mom(variant) && !h->grid.mom)
    return fail(h, FDLBM_E_ARG, "the split variants need a moment buffer, which grids of up to 65536 sites do not have");
  h->variant = variant;
  return FDLBM_OK;
}

int fdlbm_get_variant(fdlbm_t h) {
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  return h->variant;
}

int fdlbm_autotune(fdlbm_t h, int trial_steps, float* times_ms) {
  if (h && h->batch) return fail(h, FDLBM_E_STATE, "the solve is a member of a batch (step it with fdlbm_batch_step, or remove it first)");
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  if (trial_steps < 1) return fail(h, FDLBM_E_ARG, "trial_steps must be >= 1");
  if (!h->initialised) return fail(h, FDLBM_E_STATE, "autotune needs a state (set_macro first)");
  if (h->cfg.prec == FDLBM_FP64_STRICT) {  // one kernel pair: nothing to choose
    if (times_ms)
      for (int v = 0; v < V_COUNT; ++v) times_ms[v] = 0.f;
    return FDLBM_OK;
  }
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune events");
  int best = h->variant;
  float best_ms = 1e30f;
  // On small grids the trials advance the state, from a snapshot of the current buffer and health
  // word restored after each variant: the persistent variants (timed there only, where they can
  // win) over their launch, the one-step variants by alternating the buffers as fdlbm_step does.
  const bool small = (long long)h->cfg.nx * h->cfg.ny <= 262144;
  const bool persist_ok = (h->cfg.prec == FDLBM_FP64 || h->cfg.prec == FDLBM_FP32_STORE) && !any_segment(h) && small;
  // Small grids step in tens of microseconds: a few trial steps would weigh the persistent launch's
  // fixed start-up against back-to-back one-step launches, so every variant is timed over at least
  // kSmallGridTrialSteps steps there (a few milliseconds in all).
  const int tsteps = small && trial_steps < kSmallGridTrialSteps ? kSmallGridTrialSteps : trial_steps;
  unsigned char* snap = nullptr;
  if (small) {
    e = cudaMalloc(&snap, h->fbytes + 256);
    if (e == cudaSuccess) e = cudaMemcpyAsync(snap, h->f[h->cur], h->fbytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(snap + h->fbytes, h->d_health, sizeof(unsigned), cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) {
      if (snap) cudaFree(snap);
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return cuda_fail(h, e, "autotune snapshot");
    }
  }
  for (int v = 0; v < V_COUNT && e == cudaSuccess; ++v) {
    if ((variant_needs_mom(v) && !h->grid.mom) || ((variant_persistent(v) || variant_graph(v)) && !persist_ok)) {
      if (times_ms) times_ms[v] = 0.f;  // not available here
      continue;
    }
    if (variant_graph(v)) {  // replays from the current buffer (each ends there), then the snapshot
      const int replays = tsteps > kGraphSteps ? tsteps / kGraphSteps : 1;
      cudaGraphExec_t ge = nullptr;
      const int rc = graph_exec(h, h->cur, &ge);
      if (rc) {
        e = cudaErrorUnknown;
        break;
      }
      e = cudaGraphLaunch(ge, h->stream);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
      for (int r = 0; r < replays && e == cudaSuccess; ++r) e = cudaGraphLaunch(ge, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->f[h->cur], snap, h->fbytes, cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_health, snap + h->fbytes, sizeof(unsigned), cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      ms /= (float)replays * kGraphSteps;
      if (times_ms) times_ms[v] = ms;
      if (e == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = v;
      }
      continue;
    }
    if (variant_persistent(v)) {
      e = launch_steps_persist(h->cfg.prec, v, h->f[h->cur], h->f[1 - h->cur], tsteps, h->grid, h->coeffs,
                               h->d_health, h->d_bar, h->stream);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
      if (e == cudaSuccess)
        e = launch_steps_persist(h->cfg.prec, v, h->f[h->cur], h->f[1 - h->cur], tsteps, h->grid, h->coeffs,
                                 h->d_health, h->d_bar, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->f[h->cur], snap, h->fbytes, cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_health, snap + h->fbytes, sizeof(unsigned), cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      ms /= tsteps;
      if (times_ms) times_ms[v] = ms;
      if (e == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = v;
      }
      continue;
    }
    // warm-up launch, then the timed ones. With the snapshot (small grids) they step like
    // fdlbm_step, alternating the buffers, and the state is restored after: relaunching one buffer
    // pair with the same arguments times a 400 x 4 step at 14.3 us against its 16.4 us in a long
    // call. Without it (large grids, whose steps take milliseconds) every launch maps
    // f[cur] -> f[1-cur] and the state is not advanced.
    e = launch_step(h->cfg.prec, v, h->f[h->cur], h->f[1 - h->cur], h->grid, h->coeffs, h->d_health, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
    for (int t = 0; t < tsteps && e == cudaSuccess; ++t) {
      const int src = snap && (t & 1) ? 1 - h->cur : h->cur;
      e = launch_step(h->cfg.prec, v, h->f[src], h->f[1 - src], h->grid, h->coeffs, h->d_health, h->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
    if (snap && e == cudaSuccess) e = cudaMemcpyAsync(h->f[h->cur], snap, h->fbytes, cudaMemcpyDeviceToDevice, h->stream);
    if (snap && e == cudaSuccess)
      e = cudaMemcpyAsync(h->d_health, snap + h->fbytes, sizeof(unsigned), cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    ms /= tsteps;
    if (times_ms) times_ms[v] = ms;
    if (e == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  if (snap) {  // whatever happened above, the state goes back to the snapshot
    cudaError_t e2 = cudaMemcpyAsync(h->f[h->cur], snap, h->fbytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e2 == cudaSuccess)
      e2 = cudaMemcpyAsync(h->d_health, snap + h->fbytes, sizeof(unsigned), cudaMemcpyDeviceToDevice, h->stream);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(h->stream);
    cudaFree(snap);
    if (e == cudaSuccess) e = e2;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  h->variant = best;
  return FDLBM_OK;
}

long fdlbm_steps_done(fdlbm_t h) { return h ? h->steps : -1; }

int fdlbm_current_buffer(fdlbm_t h) {
  if (!h) return fail(nullptr, FDLBM_E_ARG, "handle is NULL");
  return h->cur;
}

unsigned fdlbm_health(fdlbm_t h) {
  if (!h) return 0;
  fdlbm_sync(h);
  return h->health;
}

int fdlbm_destroy(fdlbm_t h) {
  if (!h) return FDLBM_OK;
  if (h->batch) fdlbm_batch_remove(h->batch, h);
  if (h->stream || h->mem) cudaStreamSynchronize(h->stream);
  if (h->owns_mem && h->mem) cudaFree(h->mem);
  if (h->d_fstage) cudaFree(h->d_fstage);
  if (h->h_health) cudaFreeHost(h->h_health);
  if (h->ev) cudaEventDestroy(h->ev);
  for (int b = 0; b < 2; ++b)
    if (h->gexec[b]) cudaGraphExecDestroy(h->gexec[b]);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
  return FDLBM_OK;
}

const char* fdlbm_last_error(fdlbm_t h) {
  if (!h) return g_create_err.c_str();
  return h->err.c_str();
}

const char* fdlbm_version(void) { return "fdlbm-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// fdlbm_internal.h -- types shared by the host (C ABI) and device (kernels) halves of the
// CUDA library. Not part of the public ABI (include/fdlbm.h is).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/fdlbm.h"

struct fdlbm_batch_ctx;

namespace fdlbm {

constexpr int Q = 33;   // Watari-Tsutahara velocity count: rest + 4 speeds x 8 directions (Eq. 1)
constexpr int NG = 2;   // ghost ring width: Eq. 17 reaches I +- 2 along each axis

// Speeds v_1..v_4 of the four rings (the values of Sec. 4, used for every problem). They have two
// decimals, so 100 v_k is an integer (the fixed-point moment sums weight by it exactly); v_k is
// that integer over 100, correctly rounded, which is the FP64 value of the decimal.
__host__ __device__ constexpr int speed_c(int k) { return k == 0 ? 100 : k == 1 ? 192 : k == 2 ? 299 : 449; }
__host__ __device__ constexpr double speed(int k) { return speed_c(k) / 100.0; }

// Scheme flags (same values as enum fdlbm_flags).
constexpr int F_NO_LW = 1, F_NO_DISP = 2, F_NO_VISC = 4, F_SWITCH_CONST = 8;
// Boundary kinds (same values as enum fdlbm_bc).
constexpr int BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_DIRICHLET = 2, BC_WALL = 3, BC_HALO = 4;
// Health bits (same values as enum fdlbm_health_bits).
constexpr unsigned H_NUMERIC = 1u, H_KAPPA = 2u, H_TIMEOUT = 4u;

// Layout of one distribution buffer: SoA planes f[q][row][col] with row = j + 2, col = i + 2
// (ghost ring of width 2 stored in place), row pitch padded to 32 elements so every row starts
// on a 128-byte (FP32) or 256-byte (FP64) boundary.
struct Grid {
  int nx, ny;
  int pitch;        // elements per row, multiple of 32, >= nx + 4
  int rows;         // ny + 4
  long long plane;  // pitch * rows (elements per velocity plane)
  int bc[4];        // left, right, bottom, top
  int flags;
  // Moment buffer of the split step (V_S* variants), or null: planes n, ux, uy, T (FP64) and P
  // (storage precision) over the padded grid, indexed like f. Only grids above 65 536 sites and
  // FDLBM_FP64_STRICT solves (whose step always goes through it) have one.
  void* mom;
  // FDLBM_FNEQ32 only: byte offset, within one state buffer, of its 4 FP64 planes n, ux, uy, T
  // (after the 33 FP32 planes of g = f - f_eq); 0 for the other precisions.
  long long aux_off;
};

// Per-solve constants computed once on the host in FP64 and passed by value (kernel parameter
// space), so every thread reads them as uniform operands.
struct Coeffs {
  // Eq. 11 in Horner form: F_k(th) = th*(h[k][0] + th*(h[k][1] + th*(h[k][2] + th*h[k][3]))).
  double Fh[4][4];
  double v[4];        // speeds v_1..v_4
  double v2[4];       // v_k^2
  double v3_6[4];     // v_k^3 / 6
  double v4_24[4];    // v_k^4 / 24
  double v2h[4];      // v_k^2 / 2
  // Eq. 17 stencil weights without line IV, for axis a (0 = x, 1 = y), ring k, class c (0 = the
  // two axis-aligned directions, |c| = v_k dt/dr_a; 1 = the four diagonals, |c| = v_k dt/(sqrt2 dr_a)),
  // for the direction with positive c. The negative direction swaps W1/Wm1 and negates D.
  double W1[2][4][2];   // coefficient of f_{I+1}: -c/2 + c^2/2 - 2d
  double Wm1[2][4][2];  // coefficient of f_{I-1}: +c/2 + c^2/2 + 2d
  double D[2][4][2];    // coefficient of (f_{I+2} - f_{I-2}): d = c(1 - c^2)/12
  double C2[4][3];      // centre weight of line II summed over alpha: class 0 = x-axis dirs,
                        // 1 = y-axis dirs, 2 = diagonals
  double r;             // dt / tau
  double kx, ky;        // dt/dx, dt/dy  (kappa_alpha = u_alpha * k_alpha, Eq. 15)
  double lam;           // lambda of Eq. 16
  // FP32 copies used by the FP32-storage stencil
  float fW1[2][4][2], fWm1[2][4][2], fD[2][4][2], fC2[4][3];
  float fr, fkx, fky, flam;
  // Double-word FP32 (hi + lo) copies of the ring constants v_k, v_k^2/2, v_k^3/6, v_k^4/24 for
  // FDLBM_FP32_STORE_DW (hi = the FP32 rounding, lo = the rounding of the remainder)
  float dv[4][2], dv2h[4][2], dv3_6[4][2], dv4_24[4][2];
  // ... and of the F_k polynomials' coefficients, dt/tau and sqrt(1/2)
  float dFh[4][4][2], dr[2], dkS[2];
  // The raw dt, tau, dx, dy: FDLBM_FP64_STRICT forms every ratio itself, in its own order.
  double sdt, stau, sdr[2];
};

// FP64 storage (FDLBM_FP64 and FDLBM_FP64_STRICT share the layout and the copy kernels).
inline bool f64_storage(int prec) { return prec == FDLBM_FP64 || prec == FDLBM_FP64_STRICT; }

// One member of a batch (device-resident descriptor table, sorted by tile0).
struct BatchMember {
  Grid g;
  void* f[2];                // the member's ping-pong buffers
  unsigned* health;          // the member's health word
  long long tile0;           // first block index of the member in the batched launch
  int tiles_x;               // tiles along x (the tile shape is the batch's variant)
  int cur0;                  // buffer holding the state at batch step 0 (parity)
};

// Tile shape (width, height) of a launch variant.
inline void variant_tile(int v, int* tw, int* th) {
  static const int W[8] = {32, 32, 32, 16, 64, 32, 32, 32}, H[8] = {4, 8, 16, 4, 8, 32, 24, 28};
  *tw = W[v];
  *th = H[v];
}

// Launch configuration of the fused step: tile of TW x TH nodes per CTA, registers capped at 128
// per thread (2-4 CTAs per SM). Phase 1 computes the moments of the tile and its 1-node ring,
// (TW+2)(TH+2) - 4 nodes, in rounds of one node per thread. 32 x 24 and 32 x 28 on 128 threads
// fill 98-99 % of their rounds (32 x 16 on 256 threads: 79 %); which shape is fastest depends on
// the precision and the grid, and the autotuner measures it.
// V_RP* are the ring-parallel variants (four lanes per node) for small grids; batches use the
// tile variants only (V_TILE_COUNT).
// V_S* split the step in two launches: k_moments writes every node's moments once to the grid's
// moment buffer, and the update pass stages them for its tile and ring instead of recomputing
// them. Same functions, so the results are bitwise those of the fused variants.
// V_TMA32x8 (FP32 storage): the 32 x 8 tile with its 36 x 12 x 33 box brought into shared memory
// by one tensor copy (fdlbm_step_tma.cu); the other precisions run the 32 x 8 tile for it.
// V_PRP8x4, V_PT32x16 (FP64 and FP32 storage): persistent -- one cooperative launch runs all the
// steps of a call (up to kPersistMaxSteps), the CTAs meeting at a grid barrier between steps, with
// the tile bodies of V_RP8x4 and V_T32x16 (fdlbm_step_persist.cu). One-step paths (the no-alloc
// entry point, other precisions, solves with boundary segments) run those one-step variants.
// V_GRP8x4 (FP64 and FP32 storage): the ring-parallel 8 x 4 step replayed from CUDA graphs of
// kGraphSteps launches, captured once per starting buffer; the steps of a call beyond a multiple of
// kGraphSteps, and every other path, launch V_RP8x4 one by one.
enum StepVariant {
  V_T32x4 = 0, V_T32x8 = 1, V_T32x16 = 2, V_T16x4 = 3, V_T64x8 = 4, V_T32x32 = 5, V_T32x24 = 6,
  V_T32x28 = 7, V_TILE_COUNT = 8, V_RP16x4 = 8, V_RP8x4 = 9, V_S32x16 = 10, V_S32x32 = 11, V_TMA32x8 = 12,
  V_PRP8x4 = 13, V_PT32x16 = 14, V_GRP8x4 = 15, V_COUNT = 16
};
inline bool variant_needs_mom(int v) { return v == V_S32x16 || v == V_S32x32; }
inline bool variant_persistent(int v) { return v == V_PRP8x4 || v == V_PT32x16; }
inline bool variant_graph(int v) { return v == V_GRP8x4; }
inline int variant_one_step(int v) {
  return v == V_PRP8x4 || v == V_GRP8x4 ? V_RP8x4 : v == V_PT32x16 ? V_T32x16 : v;
}
constexpr int kPersistMaxSteps = 4096;
constexpr int kGraphSteps = 32;  // launches per captured graph (even: a replay ends in its first buffer)
// fdlbm_autotune times every variant over at least this many steps on grids of up to 262144 sites.
constexpr int kSmallGridTrialSteps = 32;

// Kernel launchers (fdlbm_aux.cu, fdlbm_step_f32.cu, fdlbm_step_f64.cu, fdlbm_fneq.cu). All return
// cudaGetLastError() of the launch. prec is enum fdlbm_prec.
cudaError_t launch_step_f64(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                            cudaStream_t s);
cudaError_t launch_step_f32(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                            cudaStream_t s);
// The tile variants (< V_TILE_COUNT) for a y-periodic grid with ny <= the tile height
// (fdlbm_step_wrap_f32.cu, fdlbm_step_wrap_f64.cu); launch_step picks them.
cudaError_t launch_step_wrap_f64(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c,
                                 unsigned* health, cudaStream_t s);
cudaError_t launch_step_wrap_f32(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c,
                                 unsigned* health, cudaStream_t s);
// FDLBM_FP32_STORE_DW (fdlbm_step_f32dw.cu): the FP32-storage step with the per-ring equilibrium
// constants and pairs in double-word FP32. Tile and split variants; the ring-parallel ones map to
// the 32 x 8 tile.
cudaError_t launch_step_f32dw(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                              cudaStream_t s);
cudaError_t launch_batch_f64(int variant, const BatchMember* mem, int nmem, long long tiles, unsigned long long step,
                             const Coeffs& c, cudaStream_t s);
cudaError_t launch_batch_f32(int variant, const BatchMember* mem, int nmem, long long tiles, unsigned long long step,
                             const Coeffs& c, cudaStream_t s);
cudaError_t launch_gather_health(const BatchMember* mem, int nmem, unsigned* out, cudaStream_t s);
// FDLBM_FNEQ32 (fdlbm_fneq.cu): the step, and the read-out / set-up kernels of that layout.
cudaError_t launch_step_fneq(int variant, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                             cudaStream_t s);
cudaError_t launch_batch_fneq(int variant, const BatchMember* mem, int nmem, long long tiles, unsigned long long step,
                              const Coeffs& c, cudaStream_t s);  // V_T32x4 or V_T32x8 only
cudaError_t prepare_batch_fneq(int variant);  // opt-in to its shared memory, outside stream capture
cudaError_t launch_init_fneq(void* f, const Grid& g, const Coeffs& c, const double* rho, const double* u,
                             const double* v, const double* T, cudaStream_t s);
cudaError_t launch_dirichlet_fneq(void* f, const Grid& g, const double bstate[4][4], cudaStream_t s);
cudaError_t launch_macro_fneq(const void* f, const Grid& g, double* rho, double* u, double* v, double* T,
                              cudaStream_t s);
cudaError_t launch_get_region_fneq(const void* f, const Grid& g, const Coeffs& c, int x0, int y0, int w, int h,
                                   double* out, cudaStream_t s);
cudaError_t launch_set_f_fneq(void* f, const Grid& g, const Coeffs& c, const double* in, cudaStream_t s);
// V_TMA32x8 for FP32 storage (fdlbm_step_tma.cu); dw: the double-word equilibrium.
cudaError_t launch_step_tma(bool dw, const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                            cudaStream_t s);
// nsteps steps of a persistent variant in one launch (FP64 or FP32 storage): f0 -> f1 -> f0 ...,
// the result in f1 after an odd count. bar: two zeroed-per-launch words of device memory.
cudaError_t launch_steps_persist(int prec, int variant, void* f0, void* f1, int nsteps, const Grid& g,
                                 const Coeffs& c, unsigned* health, unsigned* bar, cudaStream_t s);
// FDLBM_FP64_STRICT (fdlbm_strict.cu): the step (moments into the grid's moment buffer, then the
// update) and the kernels that write f_eq (initial condition, Dirichlet ghosts, segments) or read
// the moments, all in the canonical operation order.
cudaError_t launch_step_strict(const void* f, void* fn, const Grid& g, const Coeffs& c, unsigned* health,
                               cudaStream_t s);
cudaError_t launch_init_strict(void* f, const Grid& g, const double* rho, const double* u, const double* v,
                               const double* T, cudaStream_t s);
cudaError_t launch_dirichlet_strict(void* f, const Grid& g, const double bstate[4][4], cudaStream_t s);
cudaError_t launch_macro_strict(const void* f, const Grid& g, double* rho, double* u, double* v, double* T,
                                cudaStream_t s);
cudaError_t launch_step(int prec, int variant, const void* f, void* fn, const Grid& g, const Coeffs& c,
                        unsigned* health, cudaStream_t s);
cudaError_t launch_init(int prec, void* f, const Grid& g, const Coeffs& c, const double* rho, const double* u,
                        const double* v, const double* T, cudaStream_t s);
cudaError_t launch_dirichlet(int prec, void* f, const Grid& g, const Coeffs& c, const double bstate[4][4],
                             cudaStream_t s);
cudaError_t launch_macro(int prec, const void* f, const Grid& g, double* rho, double* u, double* v, double* T,
                         cudaStream_t s);
cudaError_t launch_get_f(int prec, const void* f, const Grid& g, double* out, cudaStream_t s);
cudaError_t launch_get_region(int prec, const void* f, const Grid& g, int x0, int y0, int w, int h, double* out,
                              cudaStream_t s);
cudaError_t launch_set_f(int prec, void* f, const Grid& g, const double* in, cudaStream_t s);
// A side's Dirichlet segment at one time (fdlbm_set_boundary_segment): the ghosts of `side` whose
// coordinate along it lies below (lower) or at/above `split` get f_eq of seg; with base_dirichlet
// the others get f_eq of base (the side's own Dirichlet state).
struct Segment {
  int side, lower, base_dirichlet;
  double split;
  double seg[4], base[4];
};
cudaError_t launch_segment(int prec, void* f, const Grid& g, const Coeffs& c, const Segment& sg, double dx, double dy,
                           cudaStream_t s);
cudaError_t launch_segment_fneq(void* f, const Grid& g, const Segment& sg, double dx, double dy, cudaStream_t s);
cudaError_t launch_segment_strict(void* f, const Grid& g, const Segment& sg, double dx, double dy, cudaStream_t s);

// Host helpers shared by the C ABI files (fdlbm_capi.cu).
struct Layout {
  Grid g;
  size_t esize, fbytes, health_off, stage_off, mom_off, mom_bytes, total;
};
bool valid_cfg(const fdlbm_config* c, std::string* why);
Layout layout_of(const fdlbm_config* c);
Coeffs make_coeffs(const fdlbm_config* cfg);
int default_variant(const fdlbm_config* c);
void set_thread_error(const char* msg);  // message returned by fdlbm_last_error(NULL)
cudaError_t batch_fence(struct ::fdlbm_batch_ctx* b);  // wait for a batch's stream (fdlbm_batch.cu)

}  // namespace fdlbm

// A solve handle (opaque in the C ABI). Shared by the C ABI files.
struct fdlbm_ctx {
  fdlbm_config cfg;
  fdlbm::Grid grid;
  fdlbm::Coeffs coeffs;
  size_t esize = 8;
  size_t fbytes = 0;       // one distribution buffer (padded)
  size_t total = 0;        // bytes of device memory in use
  unsigned char* mem = nullptr;
  bool owns_mem = false;
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  unsigned* d_health = nullptr;
  unsigned* d_bar = nullptr;   // the persistent variants' grid barrier (2 words beside the health word)
  double* d_stage = nullptr;   // 4 * nx * ny doubles for host-pointer macro calls
  double* d_fstage = nullptr;  // staging for get_f / set_f / get_f_region (allocated on first use)
  size_t fstage_cap = 0;       // doubles
  unsigned* h_health = nullptr;  // pinned
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;            // private stream the step graphs are captured on
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // V_GRP8x4: kGraphSteps steps from buffer 0 / 1
  cudaEvent_t ev = nullptr;
  bool ev_pending = false;
  bool initialised = false;
  long steps = 0;
  int sticky = FDLBM_OK;
  unsigned health = 0;
  int variant = fdlbm::V_T32x8;
  double bstate[4][4];
  // Dirichlet segments per side (fdlbm_set_boundary_segment)
  bool seg_on[4] = {false, false, false, false};
  int seg_lower[4] = {0, 0, 0, 0};
  double seg_c0[4] = {0, 0, 0, 0}, seg_speed[4] = {0, 0, 0, 0}, seg_state[4][4] = {};
  std::string err;
  struct fdlbm_batch_ctx* batch = nullptr;  // the batch this solve is a member of, if any
};



/*
 * fdlbm.h -- C ABI of the GB300-native finite-difference lattice Boltzmann
 * solver for compressible flow with high Mach number (Gan, Xu, Zhang, Yu, Li,
 * arXiv 0801.4169).
 *
 * One handle is one 2-D solve on one GPU: a distribution f_ki(x, y) over the
 * Watari-Tsutahara 33-velocity set (Sec. 2, Eq. 1; speeds v_1..v_4 =
 * 1, 1.92, 2.99, 4.49 as in Sec. 4) on an nx x ny node grid with a ghost ring of
 * width 2. Each step applies, at every node, the moments of Eqs. 3-5, the
 * equilibrium of Eqs. 10-13, and the modified Lax-Wendroff update with
 * dispersion and pressure-switched artificial viscosity of Eqs. 15-17 (the
 * alpha = x, y terms summed, relaxation counted once), followed by the
 * boundary fill of the ghost ring.
 *
 * Conventions for every call:
 *  - All physical arguments and results are FP64, whatever the storage
 *    precision. Macroscopic arrays hold nx*ny values, x fastest
 *    (index j*nx + i for node i along x, j along y). rho = n (m = 1),
 *    u, v are the x/y velocity, T the temperature (theta = T), p = rho*T.
 *  - Host pointers are owned by the caller and are not retained after the call
 *    returns. "_device" variants take device pointers that must stay valid
 *    until the handle's stream has passed the call.
 *  - Every call returns FDLBM_OK (0) or a negative fdlbm_status.
 *    fdlbm_last_error(h) then describes the failure.
 *  - Errors are sticky. After FDLBM_E_NUMERIC or FDLBM_E_CUDA, fdlbm_step
 *    refuses to run. fdlbm_get_macro, fdlbm_save and fdlbm_destroy still work,
 *    and fdlbm_set_macro / fdlbm_load clear the error.
 *  - A handle is not thread safe; different handles may be used from
 *    different threads.
 *
 * Numerical readings of points the paper leaves open:
 *  - Eq. 10: all five bracket terms sit inside nF_k[...].
 *  - gamma = 2 (2-D, e_int = nT).
 *  - Moments are taken of f.
 *  - The scheme is explicit at time t.
 *  - Boundary mechanics, which the paper does not give, are set out at
 *    enum fdlbm_bc.
 */
#ifndef FDLBM_H
#define FDLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdlbm_ctx* fdlbm_t;

enum fdlbm_status {
  FDLBM_OK = 0,
  FDLBM_E_ARG = -1,     /* invalid argument (sizes, kinds, NULL pointers, wrong handle state) */
  FDLBM_E_OOM = -2,     /* device or pinned-host allocation failed, or caller memory too small */
  FDLBM_E_CUDA = -3,    /* a CUDA runtime call failed; message in fdlbm_last_error */
  FDLBM_E_NUMERIC = -4, /* a node had non-finite moments, n <= 0 or T <= 0 (P <= 0, Eq. 16 undefined) */
  FDLBM_E_TIMEOUT = -5, /* a bounded device or host wait gave up */
  FDLBM_E_STATE = -6,   /* call not valid in the handle's state (e.g. step before set_macro) */
  FDLBM_E_IO = -7       /* checkpoint file could not be written/read or does not match the handle */
};

/* Boundary kinds per side (Sec. 5.2 names reflecting, supersonic-outflow and
 * Dirichlet boundaries; the paper gives no mechanics). Ghost ring of width 2:
 *  PERIODIC  ghost node g copies interior node g mod n (both sides of an axis must be periodic);
 *  OUTFLOW   zero gradient: both ghost layers copy the nearest interior node;
 *  DIRICHLET ghosts hold f_eq of the state given by fdlbm_set_boundary_state (default rho=1,u=v=0,T=1);
 *  WALL      specular reflection: ghost node -1-j mirrors node j with the normal
 *            velocity component reversed (needs n >= 2 along that axis).
 *  HALO      the side borders another sub-domain of a larger grid: no call of the library writes
 *            its ghosts; the caller copies the neighbour's two edge rows (or columns) of the
 *            current state into them between steps (paper_0801_4169_gb300/halo.py). */
enum fdlbm_bc { FDLBM_BC_PERIODIC = 0, FDLBM_BC_OUTFLOW = 1, FDLBM_BC_DIRICHLET = 2, FDLBM_BC_WALL = 3,
                FDLBM_BC_HALO = 4 };

enum fdlbm_side { FDLBM_LEFT = 0, FDLBM_RIGHT = 1, FDLBM_BOTTOM = 2, FDLBM_TOP = 3 };

/* Storage / arithmetic precision.
 *  FP64        f stored in FP64; moments, f_eq and the stencil in FP64.
 *  FP32_STORE  f stored and differenced in FP32; moments (Eqs. 3-5), weights and
 *              f_eq (Eqs. 10-13) evaluated in FP64. Its rounding error is about
 *              kappa * 2^-24 * n per step, kappa = sum |f_eq| / n, which destroys the
 *              temperature at high Mach number (kappa ~ 1e4 - 1e9).
 *  FNEQ32      f stored as its departure from the local equilibrium: per node the macros
 *              (n, u, v, T) in FP64 and g = f - f_eq(n, u, v, T) (Eq. 10) in FP32. Each step
 *              rebuilds f = f_eq + g in FP64 over the tile and its halo, applies Eq. 17 in
 *              FP64, takes the new moments (Eqs. 3-5) in FP64 and stores the new g. The
 *              rounding error is then 2^-24 |g| instead of 2^-24 |f|: small where the flow is
 *              near equilibrium, at any Mach number. 164 bytes per node and buffer, against
 *              264 (FP64) and 132 (FP32_STORE); about 1.6x the FP64 path's FP64 work.
 *              fdlbm_get_macro returns the stored macros; fdlbm_get_f returns f_eq + g;
 *              fdlbm_set_f stores the FP64 moments of the given f and its departure from their
 *              equilibrium. Batches of FNEQ32 solves take the 32x4 or 32x8 tile variant. */
enum fdlbm_prec { FDLBM_FP64 = 0, FDLBM_FP32_STORE = 1, FDLBM_FNEQ32 = 2, FDLBM_FP32_STORE_DW = 3,
                  FDLBM_FP64_STRICT = 4 };
/*  FP32_STORE_DW  a labelled variant of FP32_STORE ("f32-store/df32-feq"): the same storage and exact
 *              fixed-point moments finished in FP64, but the equilibrium (Eqs. 10-13: 1/T, the
 *              projections, A0, A1, F_k(theta), the per-ring constants and the 16 opposite-direction
 *              pairs) is evaluated in double-word FP32 (Dekker products, Knuth sums, compensated
 *              Horner) on the FP32 pipe instead of the FP64 one. Each f_eq is within about 2^-40 of its FP64 value before it is
 *              rounded to FP32 storage, so results differ from FP32_STORE by rare last-bit roundings.
 *              Not FP64 arithmetic; not accepted by fdlbm_batch_add.
 *  FP64_STRICT FP64 storage and arithmetic in one canonical order: every value of Eqs. 3-5
 *              (moments summed over q = 0..32 in turn), 10-13 (F_k as the quotient of Eq. 11's
 *              polynomial by its denominator, f_eq as n F_k times its five terms added left to right)
 *              and 17 (relaxation, then lines I-IV for x and then y) is formed one IEEE-754 FP64
 *              operation at a time, with no fused multiply-add, no reassociation and true divisions.
 *              Any IEEE FP64 program taking the same operations in the same order (the order is
 *              spelled out in csrc/fdlbm_strict.cu) gets the same bits; FDLBM_FP64 agrees with it to
 *              rounding (1e-12 relative on smooth flows). It is the slow reference-grade path: 8-9x
 *              the FP64 path's time per step (0.10 GLUPS). One kernel pair: the tile variants do not apply
 *              (fdlbm_set_variant is accepted and ignored; fdlbm_autotune times nothing). Not
 *              accepted by fdlbm_batch_add or fdlbm_step_noalloc (its step needs the handle's
 *              moment buffer). */

/* Scheme variants of Sec. 4 (Fig. 2, Fig. 3): drop line II, III or IV of Eq. 17,
 * or hold the switch theta_alphaI of Eq. 16 at lambda. Default 0 = full Eq. 17. */
enum fdlbm_flags {
  FDLBM_NO_LW = 1,
  FDLBM_NO_DISP = 2,
  FDLBM_NO_VISC = 4,
  FDLBM_SWITCH_CONST = 8
};

/* Health bits reported by fdlbm_health. */
enum fdlbm_health_bits {
  FDLBM_HEALTH_NUMERIC = 1, /* non-finite moment, n <= 0 or T <= 0 seen (=> FDLBM_E_NUMERIC) */
  FDLBM_HEALTH_KAPPA = 2,   /* |kappa_alpha| = |u_alpha| dt/dr_alpha > 1 seen (Eq. 15); informational */
  FDLBM_HEALTH_TIMEOUT = 4  /* a kernel's bounded wait (tile copy, grid barrier) gave up (=> FDLBM_E_TIMEOUT) */
};

/* Problem description (Eqs. 15-17 parameters). dx, dy, dt, tau > 0; lambda >= 0. */
typedef struct {
  int nx, ny;          /* interior nodes, >= 1 each */
  double dx, dy;       /* mesh spacing Delta r_alpha */
  double dt;           /* time step Delta t */
  double tau;          /* BGK relaxation time (Eq. 2) */
  double lambda;       /* artificial-viscosity amplitude (Eq. 16) */
  int bc[4];           /* enum fdlbm_bc for left, right, bottom, top */
  int prec;            /* enum fdlbm_prec */
  int flags;           /* enum fdlbm_flags */
} fdlbm_config;

/* Device bytes a handle needs for cfg (two f buffers, staging for the macro
 * arrays of the host-pointer calls, and a health word). 0 if cfg is invalid. */
size_t fdlbm_device_bytes(const fdlbm_config* cfg);

/* Create a solve. device_mem: NULL to let the library cudaMalloc, or caller
 * device memory of at least fdlbm_device_bytes(cfg) bytes, 256-byte aligned,
 * that outlives the handle (e.g. a PyTorch tensor). cuda_stream: a
 * cudaStream_t, or NULL for the legacy default stream; all device work of the
 * handle is ordered on it. The state is undefined until fdlbm_set_macro. */
int fdlbm_create_ex(fdlbm_t* out, const fdlbm_config* cfg, void* device_mem, size_t device_bytes,
                    void* cuda_stream);

/* Convenience form of fdlbm_create_ex with flags = 0 and library-owned memory. */
int fdlbm_create(fdlbm_t* out, int nx, int ny, double dx, double dy, double dt, double tau,
                 double lambda, const int bc[4], int prec, void* cuda_stream);

/* Prescribed state (rho, u, v, T) of a DIRICHLET side (enum fdlbm_side); its
 * ghosts become f_eq of that state (Eq. 10). Enqueued on the stream. */
int fdlbm_set_boundary_state(fdlbm_t h, int side, double rho, double u, double v, double T);

/* A Dirichlet segment on one side, for boundaries that change along a side or in time (the
 * double Mach reflection of Sec. 5.2.2: the post-shock state on the bottom before the wall starts
 * at x = 0.08, and on the top left of the moving shock, x <= g(t)). The paper gives no mechanics;
 * this one is a reading. At time t = steps * dt, the side's ghosts (both layers, at the interior's
 * columns or rows) whose coordinate along the side, (i + 1/2) dx for bottom/top or (j + 1/2) dy
 * for left/right, lies below the split c0 + speed * t (lower != 0), or at or above it (lower == 0),
 * hold f_eq of (rho, u, v, T). The rest of the side keeps its kind: a DIRICHLET side its own
 * state, a WALL or OUTFLOW side the ghost copies its interior nodes write. One segment per side;
 * a new call replaces it. fdlbm_step applies it after every step, with the time of the new state.
 * FDLBM_E_ARG for a periodic side, a non-finite c0 or speed, or a state without rho > 0, T > 0.
 * Solves with segments are stepped alone: fdlbm_batch_add refuses them, and fdlbm_step_noalloc
 * (which takes no handle) knows nothing of them. */
int fdlbm_set_boundary_segment(fdlbm_t h, int side, double c0, double speed, int lower, double rho, double u,
                               double v, double T);
int fdlbm_clear_boundary_segment(fdlbm_t h, int side);

/* Initial condition: f = f_eq(rho, u, v, T) at every node (Eq. 10), ghost ring
 * filled per boundary kind. Host arrays of nx*ny doubles; copied before
 * return. Resets the step count and clears a sticky error. */
int fdlbm_set_macro(fdlbm_t h, const double* rho, const double* u, const double* v, const double* T);

/* As fdlbm_set_macro with device arrays; asynchronous on the handle's stream. */
int fdlbm_set_macro_device(fdlbm_t h, const double* rho, const double* u, const double* v,
                           const double* T);

/* Advance nsteps >= 0 time steps (Eq. 17), asynchronously on the stream.
 * Returns a sticky error found by an earlier step, else FDLBM_OK; numerical
 * failure inside these steps is reported by a later call (fdlbm_sync,
 * fdlbm_get_macro, or the next fdlbm_step once the device has passed it).
 * Not for stream capture: each call ends by copying the health word to the host and recording
 * an event on the stream, which the next call polls; captured into a CUDA graph, that event is
 * not a recorded one, and the next call reports FDLBM_E_CUDA. Batches replay their steps from
 * graphs of their own (fdlbm_batch_step). */
int fdlbm_step(fdlbm_t h, long nsteps);

/* Wait for the handle's stream and return its status (FDLBM_E_NUMERIC if a
 * step saw a bad node). */
int fdlbm_sync(fdlbm_t h);

/* Moments (Eqs. 3-5) of the current f at every node into caller host arrays
 * of nx*ny doubles. Synchronises the stream. Works after a sticky error (then
 * it returns that error after filling the arrays). */
int fdlbm_get_macro(fdlbm_t h, double* rho, double* u, double* v, double* T);

/* As fdlbm_get_macro into device arrays; asynchronous, no status check. */
int fdlbm_get_macro_device(fdlbm_t h, double* rho, double* u, double* v, double* T);

/* Raw distribution of the interior, converted to FP64, layout [q][j][i]
 * (33*nx*ny doubles, q = 0 rest, q = 1 + 8(k-1) + (i-1) for speed k and
 * direction angle i*pi/4). Host arrays; synchronises. */
int fdlbm_get_f(fdlbm_t h, double* f);

/* Raw distribution of the node window [x0, x0+w) x [y0, y0+hgt), converted to FP64, layout
 * [q][j][i] (33*w*hgt doubles). The window may reach into the ghost ring
 * (-2 <= x0, x0+w <= nx+2, same for y); ghost corners hold unspecified values. Host array;
 * synchronises. FDLBM_E_ARG if the window leaves that range or is empty. */
int fdlbm_get_f_region(fdlbm_t h, int x0, int y0, int w, int hgt, double* f);

/* Set the raw interior distribution (same layout; rounded to the storage
 * precision) and refill the ghost ring. Host array; synchronises. */
int fdlbm_set_f(fdlbm_t h, const double* f);

/* Checkpoint: write / read the current f (storage precision, bit exact), the
 * step count, the boundary states and the configuration to a file. fdlbm_load
 * requires a handle with the same configuration and returns FDLBM_E_IO otherwise.
 * Boundary segments (fdlbm_set_boundary_segment) are not part of a checkpoint: the
 * saved ghosts hold their values at the saved time, and the loading handle's own
 * segments apply from its next step on. */
int fdlbm_save(fdlbm_t h, const char* path);
int fdlbm_load(fdlbm_t h, const char* path);

/* Launch variants of the fused step (CTA tile shapes). Every variant gives bitwise identical
 * results: a node's arithmetic does not depend on the tiling. FDLBM_FNEQ32 has its own kernel and
 * maps the variants onto its tile shapes (32x4, 32x8 at two register caps, 16x16, 64x4). Variant
 * 12 is, for FP32 storage, the 32x8 tile whose 36x12x33 box of f (tile, halo, all planes)
 * arrives in shared memory by one tensor-memory-accelerator copy; other precisions run the plain
 * 32x8 tile for it. Variants 13 and 14 (FP64 and FP32 storage) are persistent: one cooperative
 * launch runs all the steps of an fdlbm_step call (up to 4096 per launch), the CTAs meeting at a
 * grid barrier between steps, with the tile bodies of variants 9 (ring-parallel 8x4) and 2 (32x16).
 * That removes the per-step launch cost, 3% of a 1600-site step (small grids wait on the FP64 pipe
 * of their few warps, not on launches); the autotuner times them on small grids. A solve with boundary
 * segments, other precisions and fdlbm_step_noalloc run the one-step variants 9 and 2 for them. A
 * barrier wait that gives up (bounded at about 2^22 polls) sets FDLBM_HEALTH_TIMEOUT. Variant 15
 * (FP64 and FP32 storage) launches variant 9's step from CUDA graphs of 32 steps, captured the
 * first time they are needed (one per starting buffer, on a stream of the handle's own) and
 * replayed on the handle's stream; a call's steps beyond a multiple of 32, solves with boundary
 * segments and other precisions launch variant 9 step by step. */
int fdlbm_variant_count(void);
int fdlbm_set_variant(fdlbm_t h, int variant);  /* FDLBM_E_ARG if out of range */
int fdlbm_get_variant(fdlbm_t h);               /* current variant, or a negative status */

/* Autotuner: time every variant over trial_steps steps on the current state and keep the
 * fastest. The state is not advanced. On grids of up to 262144 sites every variant is timed over at
 * least 32 steps that alternate the buffers as fdlbm_step does (steps of tens of microseconds, where
 * launching and the persistent variants' start-up count), from a copy of the state and health word
 * that is restored after each variant (device memory for the copy: one state buffer). On larger
 * grids each trial launch reads the current buffer and writes the other, which the next real step
 * overwrites. times_ms (may be NULL) receives fdlbm_variant_count() mean times per step in
 * milliseconds. Synchronises the stream.
 * FDLBM_FP64_STRICT has one kernel pair: nothing is timed and times_ms gets zeros. */
int fdlbm_autotune(fdlbm_t h, int trial_steps, float* times_ms);

/* Which of the handle's two state buffers holds the current state (0: the first, at offset 0 of
 * its device memory; 1: the second, fbytes further on, fbytes = 33 * pitch * (ny + 4) * element
 * size rounded up to 256 bytes; FDLBM_FNEQ32 adds its 4 FP64 planes, see enum fdlbm_prec). Waits
 * for nothing: a caller that reads the buffer orders its reads after the handle's stream. */
int fdlbm_current_buffer(fdlbm_t h);

/* Steps taken since the last set_macro/load (+ the loaded count). */
long fdlbm_steps_done(fdlbm_t h);

/* Diagnostic: the FP64 operation rate this GPU sustains at its present clocks, measured with one
 * kernel of 8 CTAs of 256 threads per SM, each thread running 8 independent fused multiply-add
 * chains for iters rounds (one FMA = one operation, the unit of the step kernels' DADD + DFMA +
 * DMUL counts), timed with CUDA events after a warm-up launch on cuda_stream (NULL: the legacy
 * default stream). *ops_per_s receives the rate. Synchronous; allocates 8 bytes of device
 * memory. FDLBM_E_ARG for a NULL pointer or iters < 1. */
int fdlbm_fp64_rate(int iters, double* ops_per_s, void* cuda_stream);

/* Self-test of the bounded wait that the tensor-copy step (variant 12) uses for its tile: one CTA
 * on the current device initialises an mbarrier for one arrival, arrives on it (arrive != 0) or
 * not, and waits at most iters polls. *completed = 1 and FDLBM_OK if the wait saw the arrival;
 * *completed = 0 and FDLBM_E_TIMEOUT if it gave up (as it must without an arrival). Allocates
 * 4 bytes of device memory; synchronous. FDLBM_E_ARG for a NULL pointer or iters < 1. */
int fdlbm_selftest_wait(int arrive, int iters, int* completed);

/* Self-test of the grid barrier of the persistent variants: one cooperative launch of one CTA per SM
 * meets `rounds` times at the barrier, each wait bounded by iters polls; with skip != 0 the second
 * CTA never arrives. *completed = 1 and FDLBM_OK if every wait completed; *completed = 0 and
 * FDLBM_E_TIMEOUT if a wait gave up (as it must with skip). Synchronous; allocates 12 bytes of device
 * memory. FDLBM_E_ARG for a NULL pointer, iters < 1 or rounds < 1. */
int fdlbm_selftest_grid_barrier(int skip, int iters, int rounds, int* completed);

/* Health bits (enum fdlbm_health_bits) accumulated since set_macro; synchronises. */
unsigned fdlbm_health(fdlbm_t h);

/* ---------------------------------------------------------------------------------------------
 * Batches: many solves advanced together, one kernel launch per time step over all members'
 * tiles (replayed from a CUDA graph), for serving many small solves at once. Members keep their
 * own buffers, grids, boundary kinds and states; they must share dx, dy, dt, tau, lambda, flags
 * and the storage precision. A member's result is bitwise the same as when it is stepped alone
 * with fdlbm_step (the per-node arithmetic is identical).
 *
 * While a solve is a member: fdlbm_step, fdlbm_set_macro(_device), fdlbm_set_f, fdlbm_load and
 * fdlbm_autotune on it return FDLBM_E_STATE; read-out calls (get_macro, get_f, get_f_region,
 * save, sync, health) first wait for the batch's stream. fdlbm_destroy removes it from its batch.
 * ------------------------------------------------------------------------------------------- */
typedef struct fdlbm_batch_ctx* fdlbm_batch_t;

/* cuda_stream: the batch's stream, or NULL for a stream the batch creates (graphs cannot be
 * captured on the legacy default stream). */
int fdlbm_batch_create(fdlbm_batch_t* out, void* cuda_stream);

/* Add an initialised solve (synchronises the solve's own stream first). FDLBM_E_ARG if its
 * scheme constants differ from the batch's, FDLBM_E_STATE if it is in a batch already, has no
 * state, or carries a sticky error. */
int fdlbm_batch_add(fdlbm_batch_t b, fdlbm_t h);

/* Remove a member (synchronises the batch's stream). The solve keeps its state and step count. */
int fdlbm_batch_remove(fdlbm_batch_t b, fdlbm_t h);

/* Number of members, or a negative status. */
int fdlbm_batch_size(fdlbm_batch_t b);

/* Advance every member nsteps time steps (Eq. 17), asynchronously on the batch's stream.
 * FDLBM_E_STATE if a member carries a sticky error (remove it first). */
int fdlbm_batch_step(fdlbm_batch_t b, long nsteps);

/* Wait for the batch and collect each member's health bits into its status: a member that saw
 * a bad node (FDLBM_HEALTH_NUMERIC) gets the sticky FDLBM_E_NUMERIC. health (may be NULL)
 * receives fdlbm_batch_size() words in member order (order of addition, removals closing the
 * gaps). Returns the number of members carrying a sticky error (>= 0), or a negative status. */
int fdlbm_batch_sync(fdlbm_batch_t b, unsigned* health);

/* Launch variant of the batched step (as fdlbm_set_variant); the autotuner times every variant
 * on the members' current states without advancing them. */
int fdlbm_batch_set_variant(fdlbm_batch_t b, int variant);
int fdlbm_batch_autotune(fdlbm_batch_t b, int trial_steps, float* times_ms);

/* Release the batch (its members stay valid, detached). NULL-safe. */
int fdlbm_batch_destroy(fdlbm_batch_t b);

/* Message describing the last failure on b (NULL: as fdlbm_last_error(NULL)). Never NULL. */
const char* fdlbm_batch_last_error(fdlbm_batch_t b);

/* ---------------------------------------------------------------------------------------------
 * Serving: a continuous-batching runtime. A worker thread owns all device work. Clients submit
 * solves from any thread, then poll, wait and collect results. Each round the worker:
 *  - admits queued requests in submission order while the HBM budget and slots allow;
 *  - advances every admitted solve by the same number of steps, one batch per group of solves
 *    sharing scheme constants and precision;
 *  - retires finished solves (moments read back to host memory) and failed ones.
 * A numerical failure of an FP32-storage solve is reported; it is never re-run in FP64.
 * Time to solution runs from submission to retirement.
 * ------------------------------------------------------------------------------------------- */
typedef struct fdlbm_server_ctx* fdlbm_server_t;

enum fdlbm_req_status { FDLBM_REQ_QUEUED = 0, FDLBM_REQ_ACTIVE = 1, FDLBM_REQ_DONE = 2, FDLBM_REQ_FAILED = 3,
                        FDLBM_REQ_CANCELLED = 4 };

/* FDLBM_ENGINE_GPU runs the solves in batches (one launch per step per group).
 * FDLBM_ENGINE_GPU_SEPARATE runs the same scheduler but steps every solve with its own launches
 * (the unbatched baseline). FDLBM_ENGINE_SIMULATED runs the scheduler with no device work: each
 * step sleeps 1 ns per site, and results are filled with the step count. It is for testing the
 * scheduling policy on machines without a GPU. */
enum fdlbm_engine { FDLBM_ENGINE_GPU = 0, FDLBM_ENGINE_SIMULATED = 1, FDLBM_ENGINE_GPU_SEPARATE = 2 };

typedef struct {
  fdlbm_config cfg;                 /* the solve (as fdlbm_create_ex) */
  double bstate[4][4];              /* Dirichlet states (rho, u, v, T) per side */
  const double *rho, *u, *v, *T;    /* initial macros, nx*ny each, x fastest; copied by submit */
  long steps;                       /* time steps to run (>= 0) */
  long sim_fail_step;               /* simulated engine only: fail on reaching this step (0: never) */
} fdlbm_request;

typedef struct {
  long long submitted, done, failed, queued, rounds;
  int max_active;                   /* most solves on the device at once */
  size_t max_bytes;                 /* most device bytes in use at once (<= budget) */
  double p50_s, p99_s, mean_s;      /* time to solution of finished requests */
  double wall_s;                    /* first submission to last retirement */
  double aggregate_glups;           /* site updates of all solves / wall_s */
} fdlbm_server_stats_t;

/* budget_bytes: device memory the admitted solves may hold together (fdlbm_device_bytes each);
 * max_slots: most solves at once; round_steps: most steps per round; cuda_stream: the server's
 * stream or NULL (one is created). The GPU engine uses the device current at the call. */
int fdlbm_server_create(fdlbm_server_t* out, size_t budget_bytes, int max_slots, long round_steps, int engine,
                        void* cuda_stream);
/* Thread-safe. Copies the request's arrays; *id identifies it. A request larger than the budget
 * fails at once (status FDLBM_REQ_FAILED). */
int fdlbm_server_submit(fdlbm_server_t s, const fdlbm_request* req, long long* id);
int fdlbm_server_poll(fdlbm_server_t s, long long id, int* status);
/* Wait until the request is DONE, FAILED or CANCELLED (timeout_s < 0: no limit). FDLBM_E_TIMEOUT
 * if the time ran out first. */
int fdlbm_server_wait(fdlbm_server_t s, long long id, double timeout_s, int* status);
/* Collect a finished request's moments (any array may be NULL) and its time to solution, and
 * release it. A failed request returns its error code (FDLBM_E_NUMERIC for a numerical failure,
 * FDLBM_E_OOM if it exceeds the budget or could not be allocated) and is released;
 * FDLBM_E_STATE if it is still queued or active. */
int fdlbm_server_result(fdlbm_server_t s, long long id, double* rho, double* u, double* v, double* T,
                        double* seconds_to_solution);
int fdlbm_server_stats(fdlbm_server_t s, fdlbm_server_stats_t* st);
/* Stop the worker after its current round; queued and active requests become CANCELLED.
 * NULL-safe. */
int fdlbm_server_destroy(fdlbm_server_t s);
/* Message of the last failure on s (valid until the next call on s). */
const char* fdlbm_server_last_error(fdlbm_server_t s);

/* Largest nsteps one fdlbm_step_noalloc call accepts (its static scratch holds one word per step). */
#define FDLBM_NOALLOC_MAX_STEPS 4096

/* The fused step for callers that cannot allocate device memory. The paper has no counterpart;
 * this is a service of the library.
 *
 * Who needs it: a caller whose device memory all belongs to another allocator (a framework's
 * caching pool, a fixed arena set up at start-up), or whose path must not call cudaMalloc
 * (which can synchronise the device or fail under a memory cap). Such a caller owns both state
 * buffers and passes them in. The call allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine. The step's only scratch, one health word per step, is a
 * file-scope __device__ array of FDLBM_NOALLOC_MAX_STEPS words (16 KiB), which every GPU that
 * loads the library holds until the process exits.
 *
 * cfg      the problem (as for fdlbm_create_ex).
 * f_a      the current state, in the layout the handle calls use: 33 planes f[q][j+2][i+2] of
 *          (ny+4) rows x pitch elements, pitch = (nx+4) rounded up to a multiple of 32, in the
 *          storage precision of cfg->prec (FDLBM_FNEQ32: 33 FP32 planes of g, then, from the next
 *          256-byte boundary, 4 FP64 planes n, u, v, T of the same shape). Device memory,
 *          256-byte aligned. Its ghost ring must be filled (e.g. it was produced by a handle, or
 *          copied from one).
 * f_b      the second buffer of the pair, same size and alignment, with the same Dirichlet
 *          ghosts as f_a (steps rewrite every other ghost).
 * nsteps   0..FDLBM_NOALLOC_MAX_STEPS; larger values return FDLBM_E_ARG. Steps alternate
 *          f_a -> f_b -> f_a ...; the result is in f_a if nsteps is even, in f_b if odd.
 * first_bad_step  may be NULL; receives the index of the first step whose input held a node with
 *          non-finite moments, n <= 0 or T <= 0 (then FDLBM_E_NUMERIC is returned), else -1.
 * cuda_stream  a cudaStream_t or NULL; the call synchronises it before returning.
 *
 * The first call on a device looks up the scratch array's device address (cudaGetSymbolAddress)
 * with that device current, and later calls reuse it; make that first call before any stream
 * capture. cudaDeviceReset unloads the library's device code and may place the array elsewhere
 * when it is loaded again, so the remembered address is then stale: do not call
 * fdlbm_step_noalloc in a process after it has reset the device. Every call on a
 * device shares the one array and clears the words it uses at its start: calls that overlap on
 * the GPU (different streams or threads) race on it. Errors: FDLBM_E_ARG (invalid cfg, NULL or
 * misaligned buffers, nsteps out of range), FDLBM_E_NUMERIC, FDLBM_E_CUDA; the message is in
 * fdlbm_last_error(NULL). */
int fdlbm_step_noalloc(const fdlbm_config* cfg, void* f_a, void* f_b, long nsteps, long* first_bad_step,
                       void* cuda_stream);

/* ---- von Neumann analysis (Sec. 4, Eqs. 18-20) ----------------------------------------------
 *
 * A small Fourier perturbation of a uniform equilibrium (rho, u1, u2, T) on a periodic grid is
 * amplified each step by the 33 x 33 matrix
 *   G = (1 - dt/tau) I + (dt/tau) d f^eq/d f + diag(symbol of Eq. 17, lines I-IV)   (Eq. 18),
 * with the equilibrium Jacobian taken through rho, T and u (Eq. 20). The scheme is stable at that
 * state when max |omega| <= 1 over the wave numbers. Readings: the switch theta_alphaI of Eq. 16,
 * quadratic in the perturbation, is held at lambda (as the lambda dependence of Sec. 4 requires).
 * The speeds are the solver's, and dx, dy, dt, tau are shared by all cases of a call.
 *
 * Precision: G and its eigenvalues are computed in double-double arithmetic (~106 bits). At the
 * high-Mach states of Sec. 4 the entries of G carry the cancellation of the 4th-order f^eq, and
 * the eigenvalues move by O(1) under an FP64 rounding of G. At (2, 30, 0, 1) FP64 results are off
 * by up to 0.05, while double-double ones agree with 50-digit arithmetic to ~1e-15. */
typedef struct {
  double rho, ux, uy, T; /* uniform equilibrium state: rho > 0, T > 0 */
  double xi_x, xi_y;     /* k_x dx and k_y dy in radians, |xi| <= 8 */
  double lambda;         /* artificial-viscosity switch held at lambda (>= 0) */
  int flags;             /* FDLBM_NO_LW | FDLBM_NO_DISP | FDLBM_NO_VISC drop lines II-IV of Eq. 17 */
  int reserved;          /* must be 0 */
} fdlbm_vn_case;

/* Per-case status written by fdlbm_vn_spectrum. */
enum fdlbm_vn_status {
  FDLBM_VN_OK = 0,
  FDLBM_VN_BAD_CASE = 1,      /* rho or T not positive, a non-finite field, |xi| > 8, lambda < 0,
                                 unknown flags or reserved != 0: outputs are NaN */
  FDLBM_VN_NO_CONVERGENCE = 2 /* the QR iteration exceeded 30 sweeps per eigenvalue: the
                                 eigenvalues not found are NaN, max_abs is NaN */
};

/* Eigenvalues of G for n cases, one warp per case.
 *
 * cases    n fdlbm_vn_case records, device memory.
 * n        number of cases, 0 <= n <= 2^31 - 1.
 * dx, dy, dt, tau   grid spacings, time step, relaxation time (all > 0, finite).
 * max_abs  n doubles, device memory: max_q |omega_q| per case (the curves of Figs. 2, 4-6 are
 *          its maximum over the wave numbers).
 * omega    NULL, or 66 n doubles, device memory: the 33 eigenvalues of case c as (re, im) pairs
 *          at omega[66 c + 2 q], in no particular order.
 * G        NULL, or 2178 n doubles, device memory: G of case c, row-major (re, im) pairs at
 *          G[2178 c + 66 i + 2 j], rounded to FP64 (for checking; costs device bandwidth only).
 * status   NULL, or n ints, device memory: enum fdlbm_vn_status per case.
 * cuda_stream  a cudaStream_t or NULL. The call is asynchronous: outputs are valid once the
 *          stream has passed it. All buffers are caller-owned and must stay valid until then.
 *
 * Returns FDLBM_OK, FDLBM_E_ARG (invalid scalar argument or NULL required buffer; nothing is
 * launched) or FDLBM_E_CUDA (launch failure); the message is in fdlbm_last_error(NULL). */
int fdlbm_vn_spectrum(const fdlbm_vn_case* cases, long long n, double dx, double dy, double dt, double tau,
                      double* max_abs, double* omega, double* G, int* status, void* cuda_stream);

/* Release the handle and the memory it owns. NULL-safe. */
int fdlbm_destroy(fdlbm_t h);

/* Message describing the last failure on h, or, for h == NULL, the last
 * failure of fdlbm_create* on the calling thread. Never NULL. */
const char* fdlbm_last_error(fdlbm_t h);

/* Library version string. */
const char* fdlbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDLBM_H */

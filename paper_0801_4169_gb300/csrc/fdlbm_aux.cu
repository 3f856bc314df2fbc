// fdlbm_aux.cu -- launchers of the step dispatch and of the auxiliary kernels (initial condition,
// Dirichlet ghosts, moments out, raw f copies); templates in fdlbm_kernels.cuh.
#include "fdlbm_kernels.cuh"

namespace fdlbm {

namespace {

// Ghost node t of a side's two layers next to the interior (t < 2 len, len = ny for left/right,
// nx for top/bottom): its coordinates and its index along the side.
__device__ __forceinline__ void side_ghost(const Grid& g, int side, int t, int& gx, int& gy, int& along) {
  const int len = side < 2 ? g.ny : g.nx;
  along = t % len;
  const int layer = t / len;  // 0: next to the interior, 1: outer
  if (side == 0) { gx = -1 - layer; gy = along; }
  else if (side == 1) { gx = g.nx + layer; gy = along; }
  else if (side == 2) { gx = along; gy = -1 - layer; }
  else { gx = along; gy = g.ny + layer; }
}

template <typename S>
__global__ void k_segment(S* __restrict__ f, Grid g, Coeffs c, Segment sg, double d) {
  const int len = sg.side < 2 ? g.ny : g.nx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * len) return;
  int gx, gy, along;
  side_ghost(g, sg.side, t, gx, gy, along);
  const double pos = ((double)along + 0.5) * d;
  const bool in = sg.lower ? (pos < sg.split) : !(pos < sg.split);
  if (!in && !sg.base_dirichlet) return;
  const double* st = in ? sg.seg : sg.base;
  GhostOwn none;
  none.mx = 0;
  none.my = 0;
  write_feq<S>(f, g, c, gx, gy, none, st[0], st[1], st[2], st[3]);
}

}  // namespace

cudaError_t launch_segment(int prec, void* f, const Grid& g, const Coeffs& c, const Segment& sg, double dx, double dy,
                           cudaStream_t s) {
  const int len = sg.side < 2 ? g.ny : g.nx;
  const double d = sg.side < 2 ? dy : dx;
  dim3 b(128), grid((2 * len + 127) / 128);
  if (prec == FDLBM_FP64_STRICT) return launch_segment_strict(f, g, sg, dx, dy, s);
  if (prec == 0)
    k_segment<double><<<grid, b, 0, s>>>(static_cast<double*>(f), g, c, sg, d);
  else
    k_segment<float><<<grid, b, 0, s>>>(static_cast<float*>(f), g, c, sg, d);
  return cudaGetLastError();
}

cudaError_t launch_step(int prec, int variant, const void* f, void* fn, const Grid& g, const Coeffs& c,
                        unsigned* health, cudaStream_t s) {
  variant = variant_one_step(variant);  // one step of a persistent or graph-replayed variant: its tile body
  if (prec == FDLBM_FNEQ32) return launch_step_fneq(variant, f, fn, g, c, health, s);
  if (prec == FDLBM_FP64_STRICT) return launch_step_strict(f, fn, g, c, health, s);  // one kernel pair
  if (variant == V_TMA32x8) {
    if (prec == FDLBM_FP32_STORE || prec == FDLBM_FP32_STORE_DW)
      return launch_step_tma(prec == FDLBM_FP32_STORE_DW, f, fn, g, c, health, s);
    variant = V_T32x8;  // FP64 storage: the box would take 114 KB
  }
  if (prec == FDLBM_FP32_STORE_DW) return launch_step_f32dw(variant, f, fn, g, c, health, s);
  // a tile that holds a y-periodic grid's whole height reuses the interior rows' moments for its
  // ghost rows (same values, bit for bit)
  if (variant >= 0 && variant < V_TILE_COUNT && g.bc[2] == BC_PERIODIC && g.bc[3] == BC_PERIODIC) {
    int tw, th;
    variant_tile(variant, &tw, &th);
    if (g.ny <= th)
      return prec == 0 ? launch_step_wrap_f64(variant, f, fn, g, c, health, s)
                       : launch_step_wrap_f32(variant, f, fn, g, c, health, s);
  }
  return prec == 0 ? launch_step_f64(variant, f, fn, g, c, health, s)
                   : launch_step_f32(variant, f, fn, g, c, health, s);
}

cudaError_t launch_gather_health(const BatchMember* mem, int nmem, unsigned* out, cudaStream_t s) {
  k_gather_health<<<(nmem + 127) / 128, 128, 0, s>>>(mem, nmem, out);
  return cudaGetLastError();
}

cudaError_t launch_init(int prec, void* f, const Grid& g, const Coeffs& c, const double* rho, const double* u,
                        const double* v, const double* T, cudaStream_t s) {
  if (prec == FDLBM_FP64_STRICT) return launch_init_strict(f, g, rho, u, v, T, s);
  dim3 b(32, 4);
  if (prec == 0)
    k_init<double><<<grid2d(g, b), b, 0, s>>>(static_cast<double*>(f), g, c, rho, u, v, T);
  else
    k_init<float><<<grid2d(g, b), b, 0, s>>>(static_cast<float*>(f), g, c, rho, u, v, T);
  return cudaGetLastError();
}

cudaError_t launch_dirichlet(int prec, void* f, const Grid& g, const Coeffs& c, const double bstate[4][4],
                             cudaStream_t s) {
  if (prec == FDLBM_FP64_STRICT) return launch_dirichlet_strict(f, g, bstate, s);
  BState bs;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) bs.s[i][j] = bstate[i][j];
  const int len = 2 * (g.nx > g.ny ? g.nx : g.ny);
  dim3 b(128), grid((len + 127) / 128, 4);
  if (prec == 0)
    k_dirichlet<double><<<grid, b, 0, s>>>(static_cast<double*>(f), g, c, bs);
  else
    k_dirichlet<float><<<grid, b, 0, s>>>(static_cast<float*>(f), g, c, bs);
  return cudaGetLastError();
}

cudaError_t launch_macro(int prec, const void* f, const Grid& g, double* rho, double* u, double* v, double* T,
                         cudaStream_t s) {
  if (prec == FDLBM_FP64_STRICT) return launch_macro_strict(f, g, rho, u, v, T, s);
  dim3 b(32, 4);
  Coeffs c{};
  const double sp[4] = {1.0, 1.92, 2.99, 4.49};
  for (int k = 0; k < 4; ++k) {
    c.v[k] = sp[k];
    c.v2[k] = sp[k] * sp[k];
  }
  if (prec == 0)
    k_macro<double><<<grid2d(g, b), b, 0, s>>>(static_cast<const double*>(f), g, c, rho, u, v, T);
  else
    k_macro<float><<<grid2d(g, b), b, 0, s>>>(static_cast<const float*>(f), g, c, rho, u, v, T);
  return cudaGetLastError();
}

cudaError_t launch_get_f(int prec, const void* f, const Grid& g, double* out, cudaStream_t s) {
  dim3 b(32, 4);
  if (f64_storage(prec))
    k_get_f<double><<<grid2d(g, b), b, 0, s>>>(static_cast<const double*>(f), g, out);
  else
    k_get_f<float><<<grid2d(g, b), b, 0, s>>>(static_cast<const float*>(f), g, out);
  return cudaGetLastError();
}

cudaError_t launch_get_region(int prec, const void* f, const Grid& g, int x0, int y0, int w, int h, double* out,
                              cudaStream_t s) {
  dim3 b(32, 4), grid((w + 31) / 32, (h + 3) / 4);
  if (f64_storage(prec))
    k_get_region<double><<<grid, b, 0, s>>>(static_cast<const double*>(f), g, x0, y0, w, h, out);
  else
    k_get_region<float><<<grid, b, 0, s>>>(static_cast<const float*>(f), g, x0, y0, w, h, out);
  return cudaGetLastError();
}

cudaError_t launch_set_f(int prec, void* f, const Grid& g, const double* in, cudaStream_t s) {
  dim3 b(32, 4);
  if (f64_storage(prec))
    k_set_f<double><<<grid2d(g, b), b, 0, s>>>(static_cast<double*>(f), g, in);
  else
    k_set_f<float><<<grid2d(g, b), b, 0, s>>>(static_cast<float*>(f), g, in);
  return cudaGetLastError();
}

}  // namespace fdlbm

// fdlbm_batch.cu -- batches of solves advanced together: one launch per time step over every
// member's tiles (k_step_batch), replayed from a CUDA graph. Members keep their own buffers,
// grids, boundary kinds and states; they share the scheme constants (dx, dy, dt, tau, lambda,
// flags) and the storage precision. A node's arithmetic is the same as in the single-solve
// kernel, so a member's result does not depend on the other members.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fdlbm.h"
#include "fdlbm_internal.h"

using namespace fdlbm;

struct fdlbm_batch_ctx {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<fdlbm_ctx*> members;
  std::vector<int> cur0;               // per member: buffer holding its state at batch step 0 (parity)
  bool have_scheme = false;
  fdlbm_config scheme;                 // scheme constants shared by the members
  Coeffs coeffs;
  int variant = V_T32x8;
  bool variant_set = false;            // set explicitly or by the autotuner; else from the members
  bool dirty = true;                   // descriptor table / graph out of date
  BatchMember* d_table = nullptr;
  size_t table_cap = 0;
  unsigned* d_gather = nullptr;
  unsigned* h_gather = nullptr;        // pinned
  size_t gather_cap = 0;
  long long tiles = 0;
  unsigned long long t = 0;            // batch step counter
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;                 // even
  std::vector<BatchMember> host_table;
  std::string err;
};

namespace {

int bfail(fdlbm_batch_ctx* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  else set_thread_error(msg.c_str());
  return code;
}

int bcuda(fdlbm_batch_ctx* b, cudaError_t e, const char* what) {
  return bfail(b, FDLBM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool same_scheme(const fdlbm_config& a, const fdlbm_config& b) {
  return a.dx == b.dx && a.dy == b.dy && a.dt == b.dt && a.tau == b.tau && a.lambda == b.lambda &&
         a.flags == b.flags && a.prec == b.prec;
}

void drop_graph(fdlbm_batch_ctx* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

cudaError_t launch_one(fdlbm_batch_ctx* b, unsigned long long step) {
  const int n = (int)b->members.size();
  if (b->scheme.prec == FDLBM_FNEQ32)
    return launch_batch_fneq(b->variant, b->d_table, n, b->tiles, step, b->coeffs, b->stream);
  return b->scheme.prec == FDLBM_FP64 ? launch_batch_f64(b->variant, b->d_table, n, b->tiles, step, b->coeffs, b->stream)
                                      : launch_batch_f32(b->variant, b->d_table, n, b->tiles, step, b->coeffs, b->stream);
}

// FNEQ32 batches have two tile shapes (launch_batch_fneq).
bool variant_ok(const fdlbm_batch_ctx* b, int v) {
  if (v < 0 || v >= V_TILE_COUNT) return false;
  return b->scheme.prec != FDLBM_FNEQ32 || v == V_T32x4 || v == V_T32x8;
}

// Rebuild the device descriptor table (members sorted by insertion; tile0 is a prefix sum).
int rebuild(fdlbm_batch_ctx* b) {
  drop_graph(b);
  const size_t n = b->members.size();
  if (!b->variant_set && n) {  // tile height from the tallest member (thin shock tubes: 4 rows)
    int ny = 0;
    for (fdlbm_ctx* h : b->members) ny = std::max(ny, h->cfg.ny);
    b->variant = ny <= 4 ? V_T32x4 : ny <= 8 || b->scheme.prec == FDLBM_FNEQ32 ? V_T32x8 : V_T32x16;
  }
  if (n && !variant_ok(b, b->variant)) b->variant = V_T32x8;  // an FNEQ32 batch given another shape
  if (n && b->scheme.prec == FDLBM_FNEQ32) {
    const cudaError_t pe = prepare_batch_fneq(b->variant);
    if (pe != cudaSuccess) return bcuda(b, pe, "batch kernel set-up");
  }
  b->host_table.resize(n);
  int tw, th;
  variant_tile(b->variant, &tw, &th);
  long long tile0 = 0;
  for (size_t i = 0; i < n; ++i) {
    fdlbm_ctx* h = b->members[i];
    BatchMember& m = b->host_table[i];
    m.g = h->grid;
    m.f[0] = h->f[0];
    m.f[1] = h->f[1];
    m.health = h->d_health;
    m.tile0 = tile0;
    m.tiles_x = (h->cfg.nx + tw - 1) / tw;
    m.cur0 = b->cur0[i];
    tile0 += (long long)m.tiles_x * ((h->cfg.ny + th - 1) / th);
  }
  b->tiles = tile0;
  cudaError_t e = cudaSuccess;
  if (n > b->table_cap) {
    if (b->d_table) cudaFree(b->d_table);
    b->d_table = nullptr;
    b->table_cap = 0;
    const size_t cap = std::max<size_t>(n, 2 * b->table_cap + 16);
    e = cudaMalloc(&b->d_table, cap * sizeof(BatchMember));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, FDLBM_E_OOM, "cannot allocate the batch descriptor table");
    }
    b->table_cap = cap;
  }
  if (n > b->gather_cap) {
    if (b->d_gather) cudaFree(b->d_gather);
    if (b->h_gather) cudaFreeHost(b->h_gather);
    b->d_gather = nullptr;
    b->h_gather = nullptr;
    b->gather_cap = 0;
    const size_t cap = std::max<size_t>(n, 64);
    e = cudaMalloc(&b->d_gather, cap * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_gather, cap * sizeof(unsigned));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, FDLBM_E_OOM, "cannot allocate the batch health buffers");
    }
    b->gather_cap = cap;
  }
  if (n) {
    e = cudaMemcpyAsync(b->d_table, b->host_table.data(), n * sizeof(BatchMember), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host_table may change after return
    if (e != cudaSuccess) return bcuda(b, e, "batch table upload");
  }
  b->dirty = false;
  return FDLBM_OK;
}

// Capture graph_steps (even) launches with relative step arguments 0..G-1; replayed only when the
// batch counter is even, so member parities stay (cur0 + t) & 1.
int capture(fdlbm_batch_ctx* b, int G) {
  drop_graph(b);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  for (int i = 0; i < G && e == cudaSuccess; ++i) e = launch_one(b, (unsigned long long)i);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    cudaGetLastError();
    return bcuda(b, e, "batch graph capture");
  }
  b->graph_steps = G;
  return FDLBM_OK;
}

}  // namespace

namespace fdlbm {
cudaError_t batch_fence(fdlbm_batch_ctx* b) { return b ? cudaStreamSynchronize(b->stream) : cudaSuccess; }
}  // namespace fdlbm

extern "C" {

int fdlbm_batch_create(fdlbm_batch_t* out, void* cuda_stream) {
  if (!out) return bfail(nullptr, FDLBM_E_ARG, "out is NULL");
  *out = nullptr;
  fdlbm_batch_ctx* b = new (std::nothrow) fdlbm_batch_ctx();
  if (!b) return bfail(nullptr, FDLBM_E_OOM, "host allocation failed");
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  if (!b->stream) {  // graphs cannot be captured on the legacy default stream
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return bfail(nullptr, FDLBM_E_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    b->own_stream = true;
  }
  *out = b;
  return FDLBM_OK;
}

int fdlbm_batch_add(fdlbm_batch_t b, fdlbm_t h) {
  if (!b || !h) return bfail(b, FDLBM_E_ARG, "batch or handle is NULL");
  if (h->batch) return bfail(b, FDLBM_E_STATE, "the solve is already in a batch");
  if (!h->initialised) return bfail(b, FDLBM_E_STATE, "the solve has no state (set_macro first)");
  if (h->sticky) return bfail(b, h->sticky, "the solve carries a sticky error");
  if (h->cfg.prec == FDLBM_FP32_STORE_DW || h->cfg.prec == FDLBM_FP64_STRICT)
    return bfail(b, FDLBM_E_ARG, "FDLBM_FP32_STORE_DW and FDLBM_FP64_STRICT solves are stepped alone (fdlbm_step)");
  if (h->seg_on[0] || h->seg_on[1] || h->seg_on[2] || h->seg_on[3])
    return bfail(b, FDLBM_E_ARG, "a solve with boundary segments is stepped alone (fdlbm_step)");
  if (b->have_scheme && !same_scheme(b->scheme, h->cfg))
    return bfail(b, FDLBM_E_ARG, "members of a batch share dx, dy, dt, tau, lambda, flags and precision");
  cudaError_t e = cudaStreamSynchronize(h->stream);  // the solve's own queued work completes first
  if (e != cudaSuccess) return bcuda(b, e, "member sync");
  if (!b->have_scheme) {
    b->scheme = h->cfg;
    b->coeffs = h->coeffs;
    b->have_scheme = true;
  }
  b->members.push_back(h);
  b->cur0.push_back((int)((h->cur + 2 - (int)(b->t & 1ull)) & 1));
  h->batch = b;
  b->dirty = true;
  return FDLBM_OK;
}

int fdlbm_batch_remove(fdlbm_batch_t b, fdlbm_t h) {
  if (!b || !h) return bfail(b, FDLBM_E_ARG, "batch or handle is NULL");
  auto it = std::find(b->members.begin(), b->members.end(), h);
  if (it == b->members.end()) return bfail(b, FDLBM_E_ARG, "the solve is not a member of this batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch sync");
  const size_t i = it - b->members.begin();
  b->members.erase(it);
  b->cur0.erase(b->cur0.begin() + i);
  h->batch = nullptr;
  b->dirty = true;
  if (b->members.empty()) b->have_scheme = false;
  return FDLBM_OK;
}

int fdlbm_batch_size(fdlbm_batch_t b) {
  if (!b) return bfail(nullptr, FDLBM_E_ARG, "batch is NULL");
  return (int)b->members.size();
}

int fdlbm_batch_step(fdlbm_batch_t b, long nsteps) {
  if (!b) return bfail(nullptr, FDLBM_E_ARG, "batch is NULL");
  if (nsteps < 0) return bfail(b, FDLBM_E_ARG, "nsteps < 0");
  if (b->members.empty() || nsteps == 0) return FDLBM_OK;
  for (fdlbm_ctx* h : b->members)
    if (h->sticky) return bfail(b, FDLBM_E_STATE, "a member carries a sticky error; remove it first");
  if (b->dirty) {
    int rc = rebuild(b);
    if (rc) return rc;
  }
  cudaError_t e = cudaSuccess;
  long left = nsteps;
  // odd counter: one plain launch restores the even parity the graph was captured for
  if (b->t & 1ull) {
    e = launch_one(b, b->t);
    if (e != cudaSuccess) return bcuda(b, e, "batch launch");
    b->t += 1;
    --left;
  }
  const int G = 16;
  if (left >= G) {
    if (!b->graph) {
      int rc = capture(b, G);
      if (rc) return rc;
    }
    while (left >= G) {
      e = cudaGraphLaunch(b->graph, b->stream);
      if (e != cudaSuccess) return bcuda(b, e, "batch graph launch");
      b->t += G;
      left -= G;
    }
  }
  while (left > 0) {
    e = launch_one(b, b->t);
    if (e != cudaSuccess) return bcuda(b, e, "batch launch");
    b->t += 1;
    --left;
  }
  for (fdlbm_ctx* h : b->members) {
    h->steps += nsteps;
    h->cur = (int)((h->cur + nsteps) & 1);
  }
  return FDLBM_OK;
}

int fdlbm_batch_sync(fdlbm_batch_t b, unsigned* health) {
  if (!b) return bfail(nullptr, FDLBM_E_ARG, "batch is NULL");
  if (b->members.empty()) return FDLBM_OK;
  if (b->dirty) {
    int rc = rebuild(b);
    if (rc) return rc;
  }
  const int n = (int)b->members.size();
  cudaError_t e = launch_gather_health(b->d_table, n, b->d_gather, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_gather, b->d_gather, n * sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch sync");
  int failed = 0;
  for (int i = 0; i < n; ++i) {
    fdlbm_ctx* h = b->members[i];
    h->health |= b->h_gather[i];
    if (health) health[i] = h->health;
    if ((h->health & H_NUMERIC) && h->sticky == FDLBM_OK) {
      h->sticky = FDLBM_E_NUMERIC;
      h->err = "a node had non-finite moments, n <= 0 or T <= 0 (seen in a batched step)";
    }
    if (h->sticky) ++failed;
  }
  return failed;
}

int fdlbm_batch_set_variant(fdlbm_batch_t b, int variant) {
  if (!b) return bfail(nullptr, FDLBM_E_ARG, "batch is NULL");
  if (variant < 0 || variant >= V_TILE_COUNT) return bfail(b, FDLBM_E_ARG, "variant out of range for a batch");
  if (b->have_scheme && !variant_ok(b, variant))
    return bfail(b, FDLBM_E_ARG, "batches of FDLBM_FNEQ32 solves take the 32x4 or 32x8 tile variant");
  b->variant_set = true;
  if (variant != b->variant) {
    b->variant = variant;
    b->dirty = true;
  }
  return FDLBM_OK;
}

int fdlbm_batch_autotune(fdlbm_batch_t b, int trial_steps, float* times_ms) {
  if (!b) return bfail(nullptr, FDLBM_E_ARG, "batch is NULL");
  if (trial_steps < 1) return bfail(b, FDLBM_E_ARG, "trial_steps must be >= 1");
  if (b->members.empty()) return bfail(b, FDLBM_E_STATE, "empty batch");
  cudaEvent_t a0, a1;
  cudaError_t e = cudaEventCreate(&a0);
  if (e == cudaSuccess) e = cudaEventCreate(&a1);
  if (e != cudaSuccess) return bcuda(b, e, "autotune events");
  int best = b->variant;
  float best_ms = 1e30f;
  for (int v = 0; v < V_COUNT && e == cudaSuccess; ++v) {
    if (!variant_ok(b, v)) {  // ring-parallel variants are single-solve only; FNEQ32 has two shapes
      if (times_ms) times_ms[v] = 0.f;
      continue;
    }
    b->variant = v;
    b->variant_set = true;
    int rc = rebuild(b);
    if (rc) {
      cudaEventDestroy(a0);
      cudaEventDestroy(a1);
      return rc;
    }
    // every trial launch maps the current buffers to the other ones at the same step index, so
    // the members' states are not advanced
    e = launch_one(b, b->t);
    if (e == cudaSuccess) e = cudaEventRecord(a0, b->stream);
    for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = launch_one(b, b->t);
    if (e == cudaSuccess) e = cudaEventRecord(a1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(a1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a0, a1);
    ms /= trial_steps;
    if (times_ms) times_ms[v] = ms;
    if (e == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(a0);
  cudaEventDestroy(a1);
  if (e != cudaSuccess) return bcuda(b, e, "batch autotune");
  b->variant = best;
  b->variant_set = true;
  b->dirty = true;
  return FDLBM_OK;
}

int fdlbm_batch_destroy(fdlbm_batch_t b) {
  if (!b) return FDLBM_OK;
  cudaStreamSynchronize(b->stream);
  for (fdlbm_ctx* h : b->members) h->batch = nullptr;
  drop_graph(b);
  if (b->d_table) cudaFree(b->d_table);
  if (b->d_gather) cudaFree(b->d_gather);
  if (b->h_gather) cudaFreeHost(b->h_gather);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return FDLBM_OK;
}

const char* fdlbm_batch_last_error(fdlbm_batch_t b) {
  if (!b) return fdlbm_last_error(nullptr);
  return b->err.c_str();
}

}  // extern "C"

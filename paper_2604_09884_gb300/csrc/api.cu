// C-ABI entry points (include/inrct.h): argument checks, workspace carving and
// the composition of Algorithm 1 (Sec. 3) with an Adam update.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "filter.cuh"
#include "mlp.cuh"
#include "projector.cuh"

namespace inrct {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Stage profile of grad_step: one event per mark per step, recorded on the
// step's stream while active.
struct Profile {
  std::mutex mu;
  bool on = false;
  int max_steps = 0, step = -1;
  std::vector<cudaEvent_t> ev;  // [max_steps][kNumMarks]
  std::vector<unsigned char> hit;
};
static Profile g_prof;

// Set while a batched step is being recorded into a CUDA graph: no profile marks then.
static thread_local bool g_capturing = false;

void prof_mark(int mark, cudaStream_t st) {
  if (g_capturing) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!g_prof.on || g_prof.step < 0 || g_prof.step >= g_prof.max_steps) return;
  const size_t i = (size_t)g_prof.step * kNumMarks + mark;
  if (cudaEventRecord(g_prof.ev[i], st) == cudaSuccess) g_prof.hit[i] = 1;
}

static void prof_step_begin() {
  if (g_capturing) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (g_prof.on) ++g_prof.step;
}

static bool use_tc(const inrct_mlp* mlp) { return mlp->prec == INRCT_BF16; }

static size_t eval_ws(const inrct_mlp* mlp, const Net& n) {
  return use_tc(mlp) ? tc_eval_ws_bytes(n) : simt_eval_ws_bytes(n);
}

static size_t vjp_ws(const inrct_mlp* mlp, const Net& n, int64_t n_idx) {
  return use_tc(mlp) ? tc_vjp_ws_bytes(n, n_idx) : simt_vjp_ws_bytes(n, n_idx);
}

static int check_tc(const inrct_mlp* mlp, const Net& n) {
  if (!use_tc(mlp)) return INRCT_OK;
  char why[256];
  if (!tc_supported(n, why, sizeof(why))) {
    set_error("BF16 tensor-core path: %s", why);
    return INRCT_ERR_UNSUPPORTED;
  }
  return INRCT_OK;
}

static int eval_dispatch(const inrct_mlp* mlp, const Net& n, const float* theta, int N, int64_t npts,
                         float* image, void* ws, size_t ws_bytes, cudaStream_t st,
                         const void* prepared = nullptr) {
  return use_tc(mlp) ? tc_eval(n, theta, N, npts, image, ws, ws_bytes, st, prepared)
                     : simt_eval(n, theta, N, npts, image, ws, ws_bytes, st);
}

static int vjp_dispatch(const inrct_mlp* mlp, const Net& n, const float* theta, int N,
                        const int32_t* idx, int64_t n_idx, const float* v, double scale,
                        double* g64, float* g32, double* value, void* ws, size_t ws_bytes, cudaStream_t st,
                        const void* prepared = nullptr) {
  return use_tc(mlp) ? tc_vjp(n, theta, N, idx, n_idx, v, scale, g64, g32, value, ws, ws_bytes, st, prepared)
                     : simt_vjp(n, theta, N, idx, n_idx, v, scale, g64, g32, value, ws, ws_bytes, st);
}

}  // namespace inrct

using namespace inrct;

extern "C" {

const char* inrct_last_error(void) { return g_err; }

int64_t inrct_num_params(const inrct_mlp* mlp) {
  Net n;
  if (make_net(mlp, nullptr, &n) != INRCT_OK) return 0;
  return n.p;
}

int64_t inrct_num_rays(const inrct_geom* geom) { return num_rays(geom); }

size_t inrct_project_ws_bytes(const inrct_geom* geom, const inrct_grid* grid) {
  return project_ws_bytes(geom, grid);
}

int project(const inrct_geom* geom, const inrct_grid* grid, const float* image, float* sino,
            const float* y, float* resid, double* loss_out, void* ws, size_t ws_bytes,
            cudaStream_t stream) {
  clear_error();
  return project_impl(geom, grid, image, sino, y, resid, loss_out, ws, ws_bytes, stream);
}

int project_noalloc(const inrct_geom* geom, const inrct_grid* grid, const float* image, float* sino,
                    const float* y, float* resid, double* loss_out, cudaStream_t stream) {
  clear_error();
  return project_noalloc_impl(geom, grid, image, sino, y, resid, loss_out, stream);
}

size_t inrct_backproject_ws_bytes(const inrct_geom* geom, const inrct_grid* grid) {
  return backproject_ws_bytes(geom, grid);
}

int backproject(const inrct_geom* geom, const inrct_grid* grid, const float* sino, float* image,
                void* ws, size_t ws_bytes, cudaStream_t stream) {
  clear_error();
  return backproject_impl(geom, grid, sino, image, ws, ws_bytes, stream);
}

size_t inrct_check_index_ws_bytes(const inrct_grid* grid) {
  if (!grid || grid->N <= 0 || grid->N > 4096 || (grid->d != 2 && grid->d != 3)) return 0;
  return check_index_ws_bytes(grid_points(grid));
}

int inrct_check_index_set(const inrct_grid* grid, const int32_t* idx, int64_t n_idx, long long* counts, void* ws,
                          size_t ws_bytes, cudaStream_t stream) {
  clear_error();
  INRCT_REQUIRE(grid && grid->N > 0 && grid->N <= 4096 && (grid->d == 2 || grid->d == 3), "invalid grid");
  INRCT_REQUIRE(grid->fov == 0 || grid->fov == 1, "grid fov=%d must be 0 or 1", grid->fov);
  INRCT_REQUIRE(counts && (idx || n_idx == 0) && n_idx >= 0, "idx and counts must not be NULL");
  return check_index_set(idx, n_idx, grid_points(grid), grid->N, grid->fov, ws, ws_bytes, counts, stream);
}

size_t inrct_tune_ws_bytes(const inrct_geom* geom, const inrct_grid* grid) { return tune_ws_bytes(geom, grid); }

int inrct_tune(const inrct_geom* geom, const inrct_grid* grid, void* ws, size_t ws_bytes, cudaStream_t stream) {
  clear_error();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (g_capturing || (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)) {
    set_error("inrct_tune: the stream is being captured");
    return INRCT_ERR_INVALID_ARG;
  }
  return tune_impl(geom, grid, ws, ws_bytes, stream, nullptr);
}

int inrct_tune_plan(const inrct_geom* geom, const inrct_grid* grid, int* seg, int* bp_splits, int* zc,
                    int* tuned) {
  clear_error();
  INRCT_TRY(check_geom(geom, grid));
  INRCT_REQUIRE(seg && bp_splits && zc && tuned, "output pointers must not be NULL");
  ProjPlan p;
  *tuned = plan_lookup(geom, grid, &p) ? 1 : 0;
  *seg = p.seg;
  *bp_splits = p.bp_splits;
  *zc = p.zc;
  return INRCT_OK;
}

int inrct_tune_set(const inrct_geom* geom, const inrct_grid* grid, int seg, int bp_splits, int zc) {
  clear_error();
  ProjPlan p;
  p.seg = seg;
  p.bp_splits = bp_splits;
  p.zc = zc;
  return plan_set(geom, grid, p);
}

int inrct_tune_reset(void) {
  clear_error();
  plan_reset();
  return INRCT_OK;
}

size_t inrct_ramp_ws_bytes(const inrct_geom* geom, const inrct_grid* grid) {
  if (check_geom(geom, grid) != INRCT_OK) return 0;
  return ramp_ws_bytes(geom);
}

int ramp_filter(const inrct_geom* geom, const inrct_grid* grid, const float* r, float* out,
                double* loss_out, void* ws, size_t ws_bytes, cudaStream_t stream) {
  clear_error();
  return ramp_filter_impl(geom, grid, r, out, loss_out, ws, ws_bytes, stream);
}

size_t inrct_eval_ws_bytes(const inrct_mlp* mlp, const inrct_grid* grid) {
  Net n;
  if (!grid || make_net(mlp, grid, &n) != INRCT_OK) return 0;
  return eval_ws(mlp, n);
}

int inr_eval_grid(const inrct_mlp* mlp, const float* theta, const inrct_grid* grid, float* image,
                  void* ws, size_t ws_bytes, cudaStream_t stream) {
  clear_error();
  INRCT_REQUIRE(grid && grid->N > 0 && grid->N <= 4096, "invalid grid");
  INRCT_REQUIRE(theta && image, "theta and image must not be NULL");
  Net n;
  INRCT_TRY(make_net(mlp, grid, &n));
  INRCT_TRY(check_tc(mlp, n));
  INRCT_TRY(eval_dispatch(mlp, n, theta, grid->N, grid_points(grid), image, ws, ws_bytes, stream));
  return grid->fov ? fov_zero(image, grid_points(grid), grid->N, stream) : INRCT_OK;
}

size_t inrct_vjp_ws_bytes(const inrct_mlp* mlp, const inrct_grid* grid, int64_t n_idx) {
  Net n;
  if (!grid || n_idx <= 0 || make_net(mlp, grid, &n) != INRCT_OK) return 0;
  return vjp_ws(mlp, n, n_idx);
}

static int vjp_entry(const inrct_mlp* mlp, const float* theta, const inrct_grid* grid, const int32_t* idx,
                     int64_t n_idx, const float* v, double scale, double* value_out, double* grad_f64,
                     float* grad_f32, void* ws, size_t ws_bytes, cudaStream_t stream) {
  INRCT_REQUIRE(grid && grid->N > 0 && grid->N <= 4096, "invalid grid");
  INRCT_REQUIRE(n_idx > 0, "n_idx must be positive (got %lld)", (long long)n_idx);
  INRCT_REQUIRE(n_idx <= (int64_t)1 << 31, "n_idx too large");
  INRCT_REQUIRE(theta && idx && v && grad_f64, "theta, idx, v and grad_f64 must not be NULL");
  Net n;
  INRCT_TRY(make_net(mlp, grid, &n));
  INRCT_TRY(check_tc(mlp, n));
  return vjp_dispatch(mlp, n, theta, grid->N, idx, n_idx, v, scale, grad_f64, grad_f32, value_out, ws,
                      ws_bytes, stream);
}

int inr_weighted_vjp(const inrct_mlp* mlp, const float* theta, const inrct_grid* grid,
                     const int32_t* idx, int64_t n_idx, const float* v, double scale,
                     double* grad_f64, float* grad_f32, void* ws, size_t ws_bytes,
                     cudaStream_t stream) {
  clear_error();
  return vjp_entry(mlp, theta, grid, idx, n_idx, v, scale, nullptr, grad_f64, grad_f32, ws, ws_bytes, stream);
}

int inr_virtual_loss(const inrct_mlp* mlp, const float* theta, const inrct_grid* grid, const int32_t* idx,
                     int64_t n_idx, const float* v, double scale, double* value_out, double* grad_f64,
                     float* grad_f32, void* ws, size_t ws_bytes, cudaStream_t stream) {
  clear_error();
  INRCT_REQUIRE(value_out, "value_out must not be NULL");
  return vjp_entry(mlp, theta, grid, idx, n_idx, v, scale, value_out, grad_f64, grad_f32, ws, ws_bytes, stream);
}

int inrct_device_status(cudaStream_t stream) {
  clear_error();
  int code = 0;
  INRCT_TRY(tc_device_status(stream, &code));
  if (code == 0) return INRCT_OK;
  const char* role = code < 200 ? "weight-gradient GEMM" : code < 300 ? "weight producer"
                     : code < 400 ? "MMA issuer" : code < 900 ? "epilogue" : "set-up";
  if (code == 901) {
    set_error("a tensor-core kernel found its shared memory misaligned and did nothing (code 901)");
    return INRCT_ERR_CUDA;
  }
  set_error("a bounded wait of a tensor-core kernel gave up (%s, code %d): the outputs of the calls "
            "since the last status check are not valid", role, code);
  return INRCT_ERR_TIMEOUT;
}

int inrct_set_wait_limit(unsigned long long ns) {
  clear_error();
  tc_set_wait_limit(ns);
  return INRCT_OK;
}

int inrct_debug_stall_weight_loads(int on) {
  clear_error();
  tc_set_stall_loads(on);
  return INRCT_OK;
}

// grad_step workspace: x[n], z[m], r[m], v[n], grad[p] (FP64), loss (FP64), then
// one region reused by each stage (the largest stage need).
struct StepWs {
  float *x, *z, *r, *v;
  double *g, *loss;
  void* tables;  // ray tables, built once per step and shared by P and P^T
  size_t tables_bytes;
  void* wprep;   // BF16 weights, converted once per step (tensor-core path)
  size_t wprep_bytes;
  void* stage;
  size_t stage_bytes;
};

static size_t step_layout(const inrct_geom* geom, const inrct_grid* grid, const inrct_mlp* mlp,
                          const Net& n, int64_t n_idx, int loss, void* ws, size_t cap, StepWs* out,
                          bool* ok) {
  Carver c(ws, cap);
  StepWs w;
  const int64_t npix = grid_points(grid), m = num_rays(geom);
  w.x = c.take<float>(npix);
  w.z = c.take<float>(m);
  w.r = c.take<float>(m);
  w.v = c.take<float>(npix);
  w.g = c.take<double>(n.p);
  w.loss = c.take<double>(1);
  w.tables_bytes = tables_bytes(geom);
  w.tables = c.take<char>(w.tables_bytes);
  w.wprep_bytes = use_tc(mlp) ? tc_weights_bytes(n) : 0;
  w.wprep = use_tc(mlp) ? c.take<char>(w.wprep_bytes) : nullptr;
  size_t st = project_ws_bytes(geom, grid, false);
  st = std::max(st, backproject_ws_bytes(geom, grid, false));
  st = std::max(st, eval_ws(mlp, n));
  st = std::max(st, vjp_ws(mlp, n, n_idx));
  if (loss == INRCT_LOSS_FLS) st = std::max(st, ramp_ws_bytes(geom));
  w.stage_bytes = st;
  w.stage = c.take<char>(st);
  if (out) *out = w;
  if (ok) *ok = c.ok;
  return c.off + 256;
}

size_t inrct_step_ws_bytes(const inrct_geom* geom, const inrct_grid* grid, const inrct_mlp* mlp,
                           int64_t n_idx) {
  Net n;
  if (check_geom(geom, grid) != INRCT_OK || make_net(mlp, grid, &n) != INRCT_OK || n_idx <= 0)
    return 0;
  return step_layout(geom, grid, mlp, n, n_idx, INRCT_LOSS_FLS, nullptr, 0, nullptr, nullptr);
}

// One step of Algorithm 1 + Adam.  t_dev != NULL: the Adam step index is read from
// device memory (batched steps recorded in a graph), adam->t is ignored.
static int step_impl(const inrct_geom* geom, const inrct_grid* grid, const inrct_mlp* mlp, int loss,
                     float* theta, const float* y, const int32_t* idx, int64_t n_idx, double scale,
                     const inrct_adam* adam, const long long* t_dev, float* adam_m, float* adam_s,
                     double* loss_out, double* grad_out, void* ws, size_t ws_bytes, cudaStream_t stream) {
  INRCT_TRY(check_geom(geom, grid));
  Net n;
  INRCT_TRY(make_net(mlp, grid, &n));
  INRCT_TRY(check_tc(mlp, n));
  INRCT_REQUIRE(loss == INRCT_LOSS_LS || loss == INRCT_LOSS_FLS, "unknown loss kind %d", loss);
  INRCT_REQUIRE(theta && y && idx, "theta, y and idx must not be NULL");
  INRCT_REQUIRE(n_idx > 0, "n_idx must be positive (got %lld)", (long long)n_idx);
  StepWs w;
  bool ok;
  const size_t need = step_layout(geom, grid, mlp, n, n_idx, loss, ws, ws_bytes, &w, &ok);
  if (!ws || !ok) {
    set_error("grad_step: workspace of %zu bytes too small (need %zu)", ws_bytes, need);
    return INRCT_ERR_WORKSPACE;
  }
  prof_step_begin();
  prof_mark(kMarkStart, stream);
  if (w.wprep) INRCT_TRY(tc_prepare(n, theta, w.wprep, w.wprep_bytes, stream));
  // Algorithm 1: z = P E{f_theta}, computed without gradient tracking; loss epilogue
  INRCT_TRY(eval_dispatch(mlp, n, theta, grid->N, grid_points(grid), w.x, w.stage, w.stage_bytes,
                          stream, w.wprep));
  if (grid->fov) INRCT_TRY(fov_zero(w.x, grid_points(grid), grid->N, stream));  // E{f} inside the FOV
  ProjTables tabs;
  INRCT_TRY(build_tables(geom, grid, w.tables, w.tables_bytes, &tabs, stream));
  double* L = loss_out ? loss_out : w.loss;  // the loss at the incoming theta, written in place
  INRCT_TRY(project_impl(geom, grid, w.x, w.z, y, w.r, L, w.stage, w.stage_bytes, stream, &tabs));
  prof_mark(kMarkProjDone, stream);
  // Algorithm 1: v = P^T dL/dz  (LS: z - y; FLS: F (z - y), Sec. 3)
  if (loss == INRCT_LOSS_FLS) {
    INRCT_TRY(ramp_filter_impl(geom, grid, w.r, w.z, L, w.stage, w.stage_bytes, stream));
    INRCT_TRY(backproject_impl(geom, grid, w.z, w.v, w.stage, w.stage_bytes, stream, &tabs));
  } else {
    INRCT_TRY(backproject_impl(geom, grid, w.r, w.v, w.stage, w.stage_bytes, stream, &tabs));
  }
  prof_mark(kMarkBackDone, stream);
  // steps 3-5: the index set is the caller's; gradient of the virtual loss (Eq. 3)
  double* g = grad_out ? grad_out : w.g;
  INRCT_TRY(vjp_dispatch(mlp, n, theta, grid->N, idx, n_idx, w.v, scale, g, nullptr, nullptr, w.stage,
                         w.stage_bytes, stream, w.wprep));
  prof_mark(kMarkVjpDone, stream);
  if (adam && t_dev) {
    INRCT_TRY(adam_update_devt(theta, g, adam_m, adam_s, n.p, adam, t_dev, stream));
  } else if (adam) {
    INRCT_TRY(adam_update(theta, g, adam_m, adam_s, n.p, adam, stream));
  }
  prof_mark(kMarkEnd, stream);
  return INRCT_OK;
}

int grad_step(const inrct_geom* geom, const inrct_grid* grid, const inrct_mlp* mlp, int loss,
              float* theta, const float* y, const int32_t* idx, int64_t n_idx, double scale,
              const inrct_adam* adam, float* adam_m, float* adam_s, double* loss_out,
              double* grad_out, void* ws, size_t ws_bytes, cudaStream_t stream) {
  clear_error();
  return step_impl(geom, grid, mlp, loss, theta, y, idx, n_idx, scale, adam, nullptr, adam_m, adam_s,
                   loss_out, grad_out, ws, ws_bytes, stream);
}

// ---------------------------------------------------------------------------
// batched independent problems: one CUDA graph, one branch per problem
// ---------------------------------------------------------------------------
struct inrct_batch {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  long long launches = 0;  // kernels per launch of the graph
};

static constexpr int kBatchStreams = 8;

static size_t batch_problem_ws(const inrct_mlp* mlp, const inrct_problem& q) {
  const size_t b = inrct_step_ws_bytes(&q.geom, &q.grid, mlp, q.n_idx);
  return (b + 255) / 256 * 256;
}

static void batch_free(inrct_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->events) cudaEventDestroy(e);
  for (auto s : b->streams) cudaStreamDestroy(s);
  delete b;
}

size_t inrct_batch_ws_bytes(const inrct_mlp* mlp, const inrct_problem* probs, int n_probs) {
  if (!mlp || !probs || n_probs <= 0) return 0;
  size_t total = 0;
  for (int i = 0; i < n_probs; ++i) {
    const size_t b = batch_problem_ws(mlp, probs[i]);
    if (b <= 256) return 0;  // an invalid problem
    total += b;
  }
  return total + 256;
}

int inrct_batch_create(const inrct_mlp* mlp, int loss, const inrct_problem* probs, int n_probs,
                       const inrct_adam* adam, long long* step_counter, void* ws, size_t ws_bytes,
                       inrct_batch** out) {
  clear_error();
  INRCT_REQUIRE(out, "out must not be NULL");
  *out = nullptr;
  INRCT_REQUIRE(mlp && probs && n_probs > 0 && n_probs <= 4096, "invalid problem table (%d problems)",
                n_probs);
  INRCT_REQUIRE(adam && step_counter, "adam parameters and the device step counter are required");
  INRCT_REQUIRE(loss == INRCT_LOSS_LS || loss == INRCT_LOSS_FLS, "unknown loss kind %d", loss);
  // validate every problem up front (the graph must not be half-recorded)
  for (int i = 0; i < n_probs; ++i) {
    const inrct_problem& q = probs[i];
    Net n;
    int rc = check_geom(&q.geom, &q.grid);
    if (rc == INRCT_OK) rc = make_net(mlp, &q.grid, &n);
    if (rc == INRCT_OK) rc = check_tc(mlp, n);
    if (rc != INRCT_OK) {
      char why[400];
      snprintf(why, sizeof(why), "%s", inrct_last_error());
      set_error("problem %d: %s", i, why);
      return rc;
    }
    INRCT_REQUIRE(q.theta && q.y && q.idx && q.adam_m && q.adam_s, "problem %d: NULL buffer", i);
    INRCT_REQUIRE(q.n_idx > 0, "problem %d: n_idx must be positive", i);
  }
  const size_t need = inrct_batch_ws_bytes(mlp, probs, n_probs);
  if (!ws || ws_bytes < need) {
    set_error("grad_step_batched: workspace of %zu bytes too small (need %zu)", ws_bytes, need);
    return INRCT_ERR_WORKSPACE;
  }
  inrct_batch* b = new inrct_batch;
  const int ns = std::min(n_probs, kBatchStreams);
  auto fail = [&](const char* what, cudaError_t e) {
    set_error("grad_step_batched: %s: %s", what, cudaGetErrorString(e));
    batch_free(b);
    return INRCT_ERR_CUDA;
  };
  for (int k = 0; k < ns; ++k) {
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail("stream", e);
    b->streams.push_back(s);
  }
  for (int k = 0; k < ns; ++k) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail("event", e);
    b->events.push_back(ev);
  }
  cudaStream_t s0 = b->streams[0];
  if (use_tc(mlp)) {  // the bounded-wait status word's address, looked up before the capture
    const int rc = tc_status_resolve(s0);
    if (rc != INRCT_OK) {
      batch_free(b);
      return rc;
    }
  }
  // projector launch shapes: tune every geometry without a tuned plan, each in its own
  // problem's part of the workspace (nothing lives there before the first launch)
  {
    char* tp = static_cast<char*>(ws);
    for (int i = 0; i < n_probs; ++i) {
      const inrct_problem& q = probs[i];
      const size_t nb = batch_problem_ws(mlp, q);
      ProjPlan p;
      if (!plan_lookup(&q.geom, &q.grid, &p) && tune_ws_bytes(&q.geom, &q.grid) <= nb) {
        const int rc = tune_impl(&q.geom, &q.grid, tp, nb, s0, nullptr);
        if (rc != INRCT_OK) {
          char why[400];
          snprintf(why, sizeof(why), "%s", inrct_last_error());
          set_error("problem %d: tuning: %s", i, why);
          batch_free(b);
          return rc;
        }
      }
      tp += nb;
    }
  }
  cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail("begin capture", e);
  g_capturing = true;
  const long long l0 = g_launches.load();
  int rc = advance_step_counter(step_counter, s0);
  // fork: every branch stream waits for the counter update
  if (rc == INRCT_OK && cudaEventRecord(b->events[0], s0) != cudaSuccess) rc = INRCT_ERR_CUDA;
  for (int k = 1; k < ns && rc == INRCT_OK; ++k)
    if (cudaStreamWaitEvent(b->streams[k], b->events[0], 0) != cudaSuccess) rc = INRCT_ERR_CUDA;
  char* wp = static_cast<char*>(ws);
  for (int i = 0; i < n_probs && rc == INRCT_OK; ++i) {
    const inrct_problem& q = probs[i];
    const size_t nb = batch_problem_ws(mlp, q);
    rc = step_impl(&q.geom, &q.grid, mlp, loss, q.theta, q.y, q.idx, q.n_idx, q.scale, adam,
                   step_counter, q.adam_m, q.adam_s, q.loss_out, nullptr, wp, nb, b->streams[i % ns]);
    if (rc != INRCT_OK) {
      char why[400];
      snprintf(why, sizeof(why), "%s", inrct_last_error());
      set_error("problem %d: %s", i, why);
    }
    wp += nb;
  }
  // join
  for (int k = 1; k < ns && rc == INRCT_OK; ++k) {
    if (cudaEventRecord(b->events[k], b->streams[k]) != cudaSuccess ||
        cudaStreamWaitEvent(s0, b->events[k], 0) != cudaSuccess)
      rc = INRCT_ERR_CUDA;
  }
  g_capturing = false;
  b->launches = g_launches.load() - l0;
  g_launches.fetch_sub(b->launches);  // recorded, not launched
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(s0, &graph);
  b->graph = graph;
  if (rc != INRCT_OK) {
    if (rc == INRCT_ERR_CUDA && !inrct_last_error()[0]) set_error("grad_step_batched: capture failed");
    batch_free(b);
    return rc;
  }
  if (e != cudaSuccess) return fail("end capture", e);
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return fail("instantiate", e);
  *out = b;
  return INRCT_OK;
}

int grad_step_batched(inrct_batch* b, cudaStream_t stream) {
  clear_error();
  INRCT_REQUIRE(b && b->exec, "invalid batch");
  cudaError_t e = cudaGraphLaunch(b->exec, stream);
  if (e != cudaSuccess) {
    set_error("grad_step_batched: graph launch: %s", cudaGetErrorString(e));
    return INRCT_ERR_CUDA;
  }
  g_launches.fetch_add(b->launches);
  return INRCT_OK;
}

int inrct_batch_destroy(inrct_batch* b) {
  clear_error();
  batch_free(b);
  return INRCT_OK;
}

long long inrct_launch_count(void) { return g_launches.load(); }

int inrct_profile_begin(int max_steps) {
  clear_error();
  INRCT_REQUIRE(max_steps > 0 && max_steps <= 4096, "max_steps=%d out of range", max_steps);
  std::lock_guard<std::mutex> lk(g_prof.mu);
  INRCT_REQUIRE(!g_prof.on, "a profile is already active");
  g_prof.ev.assign((size_t)max_steps * kNumMarks, nullptr);
  g_prof.hit.assign((size_t)max_steps * kNumMarks, 0);
  for (auto& e : g_prof.ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      set_error("cudaEventCreate failed");
      return INRCT_ERR_CUDA;
    }
  }
  g_prof.max_steps = max_steps;
  g_prof.step = -1;
  g_prof.on = true;
  return INRCT_OK;
}

int inrct_profile_end(double* stage_ms, int n_stages, int* steps_out) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_prof.mu);
  INRCT_REQUIRE(g_prof.on, "no active profile");
  g_prof.on = false;
  cudaDeviceSynchronize();
  const int steps = std::min(g_prof.step + 1, g_prof.max_steps);
  for (int k = 0; k < n_stages; ++k) stage_ms[k] = 0.0;
  // stage k = time from the previous recorded mark to mark k+1
  for (int s = 0; s < steps; ++s) {
    int prev = -1;
    for (int m = 0; m < kNumMarks; ++m) {
      const size_t i = (size_t)s * kNumMarks + m;
      if (!g_prof.hit[i]) continue;
      if (prev >= 0 && m - 1 < n_stages) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g_prof.ev[(size_t)s * kNumMarks + prev], g_prof.ev[i]) == cudaSuccess)
          stage_ms[m - 1] += ms;
      }
      prev = m;
    }
  }
  for (auto& e : g_prof.ev) cudaEventDestroy(e);
  g_prof.ev.clear();
  g_prof.hit.clear();
  if (steps_out) *steps_out = steps;
  return INRCT_OK;
}

size_t inrct_gemm_tn_ws_bytes(int64_t K, int M, int N) { return gemm_tn_ws_bytes(K, M, N); }

int inrct_sincospi(const float* x, float* s, float* c, int64_t n, cudaStream_t stream) {
  clear_error();
  return sincospi_diag(x, s, c, n, stream);
}

int inrct_gemm_tn(const void* X, const void* Y, const void* Y16, int64_t K, int M, int N, float* C,
                  void* ws, size_t ws_bytes, cudaStream_t stream) {
  clear_error();
  return gemm_tn(X, Y, Y16, K, M, N, C, ws, ws_bytes, stream);
}

}  // extern "C"

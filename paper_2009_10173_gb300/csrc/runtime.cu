// Runtime around the operators and solvers: the ring-depth autotuner entry
// point, batched reconstructions in one CUDA graph, and a continuous-batching
// request server.  None of this is in the paper, which reconstructs one volume
// at a time; it serves many uneven reconstructions on one GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

using namespace oam;

// ---------------------------------------------------------------- autotune
extern "C" oam_status oam_model_autotune(oam_model *m, int32_t reps, void *stream, int32_t *ring_forward,
                                         int32_t *ring_adjoint) {
  if (!m || reps < 1) return OAM_ERR_INVALID_ARG;
  if (m->precision != OAM_PREC_BF16X3) return OAM_OK;  // nothing to tune on the FP32 path
  int f = 0, a = 0, wf = 0, wa = 0;
  oam_status rc = tc_autotune(m, reps, as_stream(stream), &f, &a, &wf, &wa);
  if (rc) return rc;
  if (ring_forward) *ring_forward = f;
  if (ring_adjoint) *ring_adjoint = a;
  return OAM_OK;
}

extern "C" oam_status oam_model_get_tiles(const oam_model *m, int32_t direction, int32_t *fold_warps,
                                          int32_t *ring) {
  if (!m || (direction != 0 && direction != 1) || !fold_warps || !ring) return OAM_ERR_INVALID_ARG;
  if (m->precision != OAM_PREC_BF16X3) return OAM_ERR_UNSUPPORTED;
  int w = 0, r = 0;
  tc_get_tiles(m, direction, &w, &r);
  *fold_warps = w;
  *ring = r;
  return OAM_OK;
}

extern "C" oam_status oam_model_set_tiles(oam_model *m, int32_t direction, int32_t fold_warps, int32_t ring) {
  if (!m || (direction != 0 && direction != 1)) return OAM_ERR_INVALID_ARG;
  if (m->precision != OAM_PREC_BF16X3) return OAM_ERR_UNSUPPORTED;
  return tc_set_tiles(m, direction, fold_warps, ring);
}

extern "C" oam_status oam_model_get_tiling(const oam_model *m, int32_t direction, int32_t *tiling) {
  if (!m || (direction != 0 && direction != 1) || !tiling) return OAM_ERR_INVALID_ARG;
  if (m->precision != OAM_PREC_BF16X3) return OAM_ERR_UNSUPPORTED;
  *tiling = tc_get_tiling(m, direction);
  return OAM_OK;
}

extern "C" oam_status oam_model_set_tiling(oam_model *m, int32_t direction, int32_t tiling) {
  if (!m || (direction != 0 && direction != 1)) return OAM_ERR_INVALID_ARG;
  if (m->precision != OAM_PREC_BF16X3) return OAM_ERR_UNSUPPORTED;
  return tc_set_tiling(m, direction, tiling);
}

// ---------------------------------------------------------------- batch
struct oam_batch {
  struct Job {
    const oam_model *model = nullptr;
    const float *s = nullptr;
    float *x_l2 = nullptr, *x_l1 = nullptr;
    oam_lsqr_opts lsqr{};
    oam_fista_opts fista{};
    void *work = nullptr;
    size_t work_bytes = 0;
    bool set = false;
    unsigned generation = 0;  // the model's generation when the graph was recorded
  };
  std::vector<Job> jobs;
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
};

namespace {

void batch_release_graph(oam_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void batch_destroy(oam_batch *b) {
  batch_release_graph(b);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

// Do two jobs touch the same model-owned buffers or overlapping workspaces?
// A model's internal staging buffers serve one stream at a time, so such
// jobs must run one after the other.
bool jobs_conflict(const oam_batch::Job &x, const oam_batch::Job &y) {
  if (x.model == y.model) return true;
  const uintptr_t x0 = reinterpret_cast<uintptr_t>(x.work), y0 = reinterpret_cast<uintptr_t>(y.work);
  return x0 < y0 + y.work_bytes && y0 < x0 + x.work_bytes;
}

// Branch of each job: jobs that conflict (directly or through other jobs)
// share the branch of the first of them and run in job order; all others get
// their own branch.
std::vector<int> batch_branches(const oam_batch *b) {
  const int n = (int)b->jobs.size();
  std::vector<int> br(n);
  for (int j = 0; j < n; ++j) br[j] = j;
  for (bool changed = true; changed;) {  // connected components, smallest index as label
    changed = false;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j)
        if (br[j] != br[i] && jobs_conflict(b->jobs[i], b->jobs[j])) {
          const int lo = std::min(br[i], br[j]);
          br[i] = br[j] = lo;
          changed = true;
        }
  }
  return br;
}

// Record every job (LSQR, then FISTA) on its branch of one graph.
oam_status batch_capture(oam_batch *b) {
  batch_release_graph(b);
  const std::vector<int> br = batch_branches(b);
  OAM_CUDA_TRY(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed));
  oam_status rc = OAM_OK;
  if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) rc = OAM_ERR_CUDA;
  for (size_t g = 0; g < b->jobs.size() && !rc; ++g) {
    if (br[g] != (int)g) continue;  // not the first job of a branch
    cudaStream_t st = b->streams[g];
    if (cudaStreamWaitEvent(st, b->fork, 0) != cudaSuccess) {
      rc = OAM_ERR_CUDA;
      break;
    }
    for (size_t j = g; j < b->jobs.size() && !rc; ++j) {
      if (br[j] != (int)g) continue;
      const oam_batch::Job &J = b->jobs[j];
      if (J.lsqr.iters > 0) rc = oam_lsqr(J.model, J.s, J.x_l2, &J.lsqr, nullptr, J.work, J.work_bytes, st);
      if (!rc && J.fista.iters > 0)
        rc = oam_l1_fista(J.model, J.s, J.x_l1, &J.fista, nullptr, J.work, J.work_bytes, st);
    }
    if (!rc && cudaEventRecord(b->joins[g], st) != cudaSuccess) rc = OAM_ERR_CUDA;
    if (!rc && cudaStreamWaitEvent(b->origin, b->joins[g], 0) != cudaSuccess) rc = OAM_ERR_CUDA;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t end = cudaStreamEndCapture(b->origin, &g);
  if (rc || end != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc ? rc : OAM_ERR_CUDA;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    batch_release_graph(b);
    return OAM_ERR_CUDA;
  }
  for (auto &J : b->jobs) J.generation = J.model->generation;
  b->dirty = false;
  return OAM_OK;
}

}  // namespace

extern "C" oam_status oam_batch_create(int32_t n_jobs, oam_batch **out) {
  if (!out || n_jobs < 1 || n_jobs > 4096) return OAM_ERR_INVALID_ARG;
  *out = nullptr;
  oam_batch *b = new (std::nothrow) oam_batch();
  if (!b) return OAM_ERR_OOM;
  b->jobs.resize(n_jobs);
  bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int j = 0; j < n_jobs && ok; ++j) {
    cudaStream_t s;
    cudaEvent_t e;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->streams.push_back(s);
    ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->joins.push_back(e);
  }
  if (!ok) {
    cudaGetLastError();
    batch_destroy(b);
    return OAM_ERR_CUDA;
  }
  *out = b;
  return OAM_OK;
}

extern "C" oam_status oam_batch_set_job(oam_batch *b, int32_t j, const oam_model *model, const float *d_s,
                                        float *d_x_l2, float *d_x_l1, const oam_lsqr_opts *lsqr,
                                        const oam_fista_opts *fista, void *d_work, size_t work_bytes) {
  if (!b || j < 0 || j >= (int)b->jobs.size() || !model || !d_s || !d_work) return OAM_ERR_INVALID_ARG;
  if ((!lsqr || lsqr->iters <= 0) && (!fista || fista->iters <= 0)) return OAM_ERR_INVALID_ARG;
  size_t need = 0, n1 = 0;
  oam_solver_work_bytes(model, 0, &need);
  oam_solver_work_bytes(model, 1, &n1);
  need = std::max(need, n1);
  if (work_bytes < need) return OAM_ERR_INVALID_ARG;
  oam_batch::Job &J = b->jobs[j];
  J.model = model;
  J.s = d_s;
  J.x_l2 = d_x_l2;
  J.x_l1 = d_x_l1;
  J.lsqr = lsqr ? *lsqr : oam_lsqr_opts{};
  J.fista = fista ? *fista : oam_fista_opts{};
  if (J.lsqr.iters > 0 && !d_x_l2) return OAM_ERR_INVALID_ARG;
  if (J.fista.iters > 0 && !d_x_l1) return OAM_ERR_INVALID_ARG;
  J.work = d_work;
  J.work_bytes = work_bytes;
  J.set = true;
  b->dirty = true;
  return OAM_OK;
}

extern "C" oam_status oam_batch_run(oam_batch *b, void *stream) {
  if (!b) return OAM_ERR_INVALID_ARG;
  for (const auto &J : b->jobs) {
    if (!J.set) return OAM_ERR_INVALID_ARG;
    if (J.generation != J.model->generation) b->dirty = true;  // a model's buffers changed: record again
  }
  if (b->dirty) {
    oam_status rc = batch_capture(b);
    if (rc) return rc;
  }
  OAM_CUDA_TRY(cudaGraphLaunch(b->exec, as_stream(stream)));
  count_launch(1);
  return OAM_OK;
}

extern "C" oam_status oam_batch_free(oam_batch *b) {
  if (!b) return OAM_OK;
  cudaDeviceSynchronize();
  batch_destroy(b);
  return OAM_OK;
}

// ---------------------------------------------------------------- server
// Requests carry host signals and host image buffers.  A host thread admits
// queued requests while a slot (stream) is free and the device-memory budget
// holds their footprint, builds each request's model and buffers, and
// enqueues copy-in, LSQR, FISTA and copy-out on the slot's stream; requests on
// different slots overlap on the GPU.  Finished slots free their memory and
// take the next request (continuous batching).  Completion is detected with
// event queries, never with unbounded waits.
struct oam_server {
  struct Req {
    int64_t id = 0;
    oam_sensor sensor{};
    oam_grid grid{};
    oam_eir eir{};
    const float *h_s = nullptr;
    float *h_x2 = nullptr, *h_x1 = nullptr;
    int32_t state = 0;  // 0 queued, 1 running, 2 done, 3 failed
    oam_status error = OAM_OK;
    size_t need = 0;              // reservation planned at submit (model plan + buffers + workspace)
    oam_status plan_rc = OAM_OK;  // the plan's status: a request that cannot be built fails at admission
    size_t reserved = 0;
    std::chrono::steady_clock::time_point t_submit, t_done;
    // device resources while running
    oam_model *model = nullptr;
    float *d_s = nullptr, *d_x2 = nullptr, *d_x1 = nullptr;
    void *d_work = nullptr;
    int slot = -1;
    cudaEvent_t done_ev = nullptr;
  };
  oam_server_opts opts{};
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<bool> slot_busy;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> queue;
  std::map<int64_t, Req> reqs;
  int64_t next_id = 1;
  // Footprint plans by request geometry (the raw bytes of sensor, grid and
  // EIR): repeated geometries skip the host planning at submit.
  std::mutex plan_mu;
  std::map<std::string, std::pair<oam_status, size_t>> plans;
  size_t reserved = 0, peak_reserved = 0;
  int running = 0, peak_running = 0;
  bool stop = false;
  std::thread worker;
};

namespace {

size_t vol_bytes(const oam_grid &g) { return (size_t)g.px * g.py * g.nz * sizeof(float); }
size_t sig_bytes(const oam_grid &g) { return (size_t)g.px * g.py * g.nt * sizeof(float); }

// Device-memory reservation for a request before its model exists: the
// model's planned device bytes (oam_model_bytes, an upper bound of what the
// build allocates), the signals, two images and the solver workspace (the
// larger of LSQR's 2 signal + 3 volume vectors and FISTA's, plus scalars).
oam_status request_footprint(int precision, const oam_sensor *sn, const oam_grid *g, const oam_eir *e,
                             size_t *bytes) {
  size_t model = 0;
  oam_status rc = oam_model_bytes(sn, g, e, (oam_precision)precision, &model);
  if (rc) return rc;
  const size_t work = 256 * 1024 + 2 * sig_bytes(*g) + 3 * vol_bytes(*g);
  *bytes = model + sig_bytes(*g) + 2 * vol_bytes(*g) + work;
  return OAM_OK;
}

void release(oam_server *S, oam_server::Req &r) {
  // the request's stream is idle (its completion event fired): free on it
  cudaStream_t st = r.slot >= 0 ? S->streams[r.slot] : nullptr;
  if (r.model) model_release(r.model, st);
  if (r.d_s) cudaFreeAsync(r.d_s, st);
  if (r.d_x2) cudaFreeAsync(r.d_x2, st);
  if (r.d_x1) cudaFreeAsync(r.d_x1, st);
  if (r.d_work) cudaFreeAsync(r.d_work, st);
  if (r.done_ev) cudaEventDestroy(r.done_ev);
  r.model = nullptr;
  r.d_s = r.d_x2 = r.d_x1 = nullptr;
  r.d_work = nullptr;
  r.done_ev = nullptr;
  if (r.slot >= 0) S->slot_busy[r.slot] = false;
  r.slot = -1;
  S->reserved -= r.reserved;
  r.reserved = 0;
  S->running -= 1;
}

// Build and enqueue one admitted request (server thread, lock not held).
oam_status launch(oam_server *S, oam_server::Req &r, size_t *actual) {
  cudaStream_t st = S->streams[r.slot];
  oam_status rc = oam_build_model(&r.sensor, &r.grid, &r.eir, (oam_precision)S->opts.precision, st, &r.model);
  if (rc) return rc;
  size_t w0 = 0, w1 = 0;
  oam_solver_work_bytes(r.model, 0, &w0);
  oam_solver_work_bytes(r.model, 1, &w1);
  const size_t wb = std::max(w0, w1);
  *actual = r.model->bytes + sig_bytes(r.grid) + 2 * vol_bytes(r.grid) + wb;
  if (cudaMallocAsync((void **)&r.d_s, sig_bytes(r.grid), st) != cudaSuccess ||
      cudaMallocAsync((void **)&r.d_x2, vol_bytes(r.grid), st) != cudaSuccess ||
      cudaMallocAsync((void **)&r.d_x1, vol_bytes(r.grid), st) != cudaSuccess ||
      cudaMallocAsync(&r.d_work, wb, st) != cudaSuccess) {
    cudaGetLastError();
    return OAM_ERR_OOM;
  }
  OAM_CUDA_TRY(cudaEventCreateWithFlags(&r.done_ev, cudaEventDisableTiming));
  OAM_CUDA_TRY(cudaMemcpyAsync(r.d_s, r.h_s, sig_bytes(r.grid), cudaMemcpyHostToDevice, st));
  oam_lsqr_opts lo{S->opts.lsqr_iters, 0.0};
  oam_fista_opts fo{};
  fo.iters = S->opts.fista_iters;
  fo.power_iters = S->opts.power_iters;
  fo.nonneg = 1;
  fo.lambda = -1.0;
  fo.lambda_rel = S->opts.lambda_rel;
  fo.L = 0.0;
  if (lo.iters > 0 && (rc = oam_lsqr(r.model, r.d_s, r.d_x2, &lo, nullptr, r.d_work, wb, st))) return rc;
  if (fo.iters > 0 && (rc = oam_l1_fista(r.model, r.d_s, r.d_x1, &fo, nullptr, r.d_work, wb, st))) return rc;
  if (r.h_x2 && lo.iters > 0)
    OAM_CUDA_TRY(cudaMemcpyAsync(r.h_x2, r.d_x2, vol_bytes(r.grid), cudaMemcpyDeviceToHost, st));
  if (r.h_x1 && fo.iters > 0)
    OAM_CUDA_TRY(cudaMemcpyAsync(r.h_x1, r.d_x1, vol_bytes(r.grid), cudaMemcpyDeviceToHost, st));
  OAM_CUDA_TRY(cudaEventRecord(r.done_ev, st));
  return OAM_OK;
}

void server_loop(oam_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    // 1. retire finished requests
    for (auto &kv : S->reqs) {
      oam_server::Req &r = kv.second;
      if (r.state != 1) continue;
      const cudaError_t q = cudaEventQuery(r.done_ev);
      if (q == cudaErrorNotReady) continue;
      r.state = q == cudaSuccess ? 2 : 3;
      if (q != cudaSuccess) {
        r.error = OAM_ERR_CUDA;
        cudaGetLastError();
      }
      r.t_done = std::chrono::steady_clock::now();
      release(S, r);
      S->cv.notify_all();
    }
    // 2. admit queued requests (first in, first out) while a slot and memory are free
    while (!S->queue.empty()) {
      oam_server::Req &r = S->reqs[S->queue.front()];
      if (r.plan_rc) {  // the model cannot be built (invalid parameters, window, shape)
        S->queue.pop_front();
        r.state = 3;
        r.error = r.plan_rc;
        r.t_done = std::chrono::steady_clock::now();
        S->cv.notify_all();
        continue;
      }
      const size_t need = r.need;
      int slot = -1;
      for (int i = 0; i < (int)S->slot_busy.size(); ++i)
        if (!S->slot_busy[i]) {
          slot = i;
          break;
        }
      if (slot < 0) break;
      if (need > S->opts.hbm_budget_bytes) {  // can never fit
        S->queue.pop_front();
        r.state = 3;
        r.error = OAM_ERR_OOM;
        r.t_done = std::chrono::steady_clock::now();
        S->cv.notify_all();
        continue;
      }
      if (S->reserved + need > S->opts.hbm_budget_bytes) break;
      S->queue.pop_front();
      r.slot = slot;
      S->slot_busy[slot] = true;
      r.reserved = need;
      S->reserved += need;
      S->peak_reserved = std::max(S->peak_reserved, S->reserved);
      S->running += 1;
      S->peak_running = std::max(S->peak_running, S->running);
      r.state = 1;
      lk.unlock();
      size_t actual = 0;
      const oam_status rc = launch(S, r, &actual);
      lk.lock();
      if (!rc && actual > r.reserved) {  // reconcile with what the request really holds
        S->reserved += actual - r.reserved;
        r.reserved = actual;
        S->peak_reserved = std::max(S->peak_reserved, S->reserved);
      }
      if (rc) {
        cudaStreamSynchronize(S->streams[slot]);
        cudaGetLastError();
        r.state = 3;
        r.error = rc;
        r.t_done = std::chrono::steady_clock::now();
        release(S, r);
        S->cv.notify_all();
      }
    }
    if (S->stop && S->queue.empty() && S->running == 0) break;
    S->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

}  // namespace

extern "C" oam_status oam_request_footprint(int32_t precision, const oam_sensor *sensor, const oam_grid *grid,
                                            const oam_eir *eir, size_t *bytes) {
  if (!sensor || !grid || !eir || !bytes) return OAM_ERR_INVALID_ARG;
  if (precision != OAM_PREC_FP32 && precision != OAM_PREC_BF16X3 && precision != OAM_PREC_FFT)
    return OAM_ERR_INVALID_ARG;
  return request_footprint(precision, sensor, grid, eir, bytes);
}

extern "C" oam_status oam_server_create(const oam_server_opts *opts, oam_server **out) {
  if (!opts || !out || opts->max_slots < 1 || opts->max_slots > 256 || opts->hbm_budget_bytes == 0 ||
      opts->lsqr_iters < 0 || opts->fista_iters < 0 || opts->power_iters < 1 ||
      (opts->precision != OAM_PREC_FP32 && opts->precision != OAM_PREC_BF16X3 && opts->precision != OAM_PREC_FFT))
    return OAM_ERR_INVALID_ARG;
  *out = nullptr;
  oam_server *S = new (std::nothrow) oam_server();
  if (!S) return OAM_ERR_OOM;
  S->opts = *opts;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return OAM_ERR_CUDA;
  }
  for (int i = 0; i < opts->max_slots; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t t : S->streams) cudaStreamDestroy(t);
      delete S;
      return OAM_ERR_CUDA;
    }
    S->streams.push_back(s);
  }
  S->slot_busy.assign(opts->max_slots, false);
  S->worker = std::thread(server_loop, S);
  *out = S;
  return OAM_OK;
}

extern "C" oam_status oam_server_submit(oam_server *S, const oam_sensor *sensor, const oam_grid *grid,
                                        const oam_eir *eir, const float *h_s, float *h_x_l2, float *h_x_l1,
                                        int64_t *request_id) {
  if (!S || !sensor || !grid || !eir || !h_s || !request_id) return OAM_ERR_INVALID_ARG;
  oam_server::Req r;
  std::string key(reinterpret_cast<const char *>(sensor), sizeof(oam_sensor));
  key.append(reinterpret_cast<const char *>(grid), sizeof(oam_grid));
  key.append(reinterpret_cast<const char *>(eir), sizeof(oam_eir));
  bool cached = false;
  {
    std::lock_guard<std::mutex> pl(S->plan_mu);
    auto it = S->plans.find(key);
    if (it != S->plans.end()) {
      r.plan_rc = it->second.first;
      r.need = it->second.second;
      cached = true;
    }
  }
  if (!cached) {
    r.plan_rc = request_footprint(S->opts.precision, sensor, grid, eir, &r.need);  // host only, outside the locks
    std::lock_guard<std::mutex> pl(S->plan_mu);
    if (S->plans.size() >= 4096) S->plans.clear();  // bounded
    S->plans[key] = {r.plan_rc, r.need};
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return OAM_ERR_BUSY;
  r.id = S->next_id++;
  r.sensor = *sensor;
  r.grid = *grid;
  r.eir = *eir;
  r.h_s = h_s;
  r.h_x2 = h_x_l2;
  r.h_x1 = h_x_l1;
  r.t_submit = std::chrono::steady_clock::now();
  S->reqs[r.id] = r;
  S->queue.push_back(r.id);
  *request_id = r.id;
  S->cv.notify_all();
  return OAM_OK;
}

extern "C" oam_status oam_server_poll(oam_server *S, int64_t id, oam_request_info *info) {
  if (!S || !info) return OAM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return OAM_ERR_INVALID_ARG;
  const oam_server::Req &r = it->second;
  info->state = r.state;
  info->error = r.error;
  info->latency_s = (r.state >= 2) ? std::chrono::duration<double>(r.t_done - r.t_submit).count() : -1.0;
  return OAM_OK;
}

extern "C" oam_status oam_server_wait(oam_server *S, int64_t id, double timeout_s) {
  if (!S || !(timeout_s >= 0)) return OAM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return OAM_ERR_INVALID_ARG;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (it->second.state < 2) {
    if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state < 2) return OAM_ERR_TIMEOUT;
  }
  return it->second.state == 2 ? OAM_OK : it->second.error;
}

extern "C" oam_status oam_server_stats(oam_server *S, oam_server_stats_t *st) {
  if (!S || !st) return OAM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  st->queued = (int32_t)S->queue.size();
  st->running = S->running;
  st->peak_running = S->peak_running;
  st->reserved_bytes = S->reserved;
  st->peak_reserved_bytes = S->peak_reserved;
  return OAM_OK;
}

extern "C" oam_status oam_server_stop(oam_server *S) {
  if (!S) return OAM_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
  delete S;
  return OAM_OK;
}

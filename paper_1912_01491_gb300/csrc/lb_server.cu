// lb_server.cu -- the serving form: realizations of mixed N arrive as
// requests, are admitted by device memory, assembled (Eqs. (07)-(09)) and
// integrated (RK4) while others are still on the GPU, and report latency.
//
// One scheduler thread per server owns all launches.  Each admitted request
// gets its own non-blocking stream, with a stream priority that favours small
// N, so the block scheduler interleaves a small request's kernels with a
// large one's instead of queueing behind it.  Device memory comes from a
// server-owned stream-ordered pool (cudaFree would synchronize the device
// and stall every running request).  Two engines:
//  * cluster engine (N <= 64, FP32): the requests admitted in one scheduler
//    pass are assembled on one stream and integrated by one launch of the
//    cluster-persistent batched RK4 kernel, which occupies only C SMs per
//    realization;
//  * stream engine (any N, any precision): the RK4 step loop is captured
//    once per request as a CUDA graph of `chunk` steps (fused stage kernels
//    plus the FP64 correction), and the graph is replayed nsteps/chunk times.
// Completion is signalled by a host function enqueued after the result copy,
// which stamps the completion time and wakes the scheduler.  A request's
// result does not depend on what else is running: the kernels, launch shapes
// and cluster size it gets are functions of its own (N, precision) alone.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lb_internal.h"
#include "lb_sched.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

inline int64_t r256(int64_t x) { return (x + 255) & ~int64_t(255); }

int engine_of(int N, int precision) {
  return (N <= lbi::kBatchMaxN && precision == LB_FP32) ? LB_ENGINE_CLUSTER : LB_ENGINE_STREAM;
}

int64_t footprint(int N, int precision, bool with_h) {
  const int64_t M = (int64_t)N * N - 1;
  int64_t b = r256(8 * M * M) + 2 * r256(8 * M);  // A64, K, v
  if (precision == LB_FP32) b += r256(4 * M * M);
  if (precision == LB_BF16) b += r256(2 * M * M) + r256(4 * M);
  if (with_h) b += r256(8 * M) + r256(16 * M);  // h and the complex expansion
  if (engine_of(N, precision) == LB_ENGINE_STREAM) b += r256((int64_t)lbi::rk4_workspace_bytes(M));
  return b;
}

// steps per captured graph: a multiple of the correction period, about 50
int64_t chunk_steps(int precision, int correct_every) {
  const int64_t base = (precision != LB_FP64 && correct_every > 0) ? correct_every : 1;
  return base * std::max<int64_t>(1, 50 / base);
}

struct Req {
  uint64_t id = 0;
  lb_request q{};
  int64_t M = 0, bytes = 0;
  int engine = LB_ENGINE_STREAM, cluster = 0;
  std::atomic<int> state{LB_REQ_QUEUED};
  int status = LB_OK;
  std::string err;
  Clock::time_point t_submit, t_admit, t_done;
  const lb_basis_t* basis = nullptr;
  // device memory from the server pool
  double *A64 = nullptr, *K = nullptr, *v = nullptr, *h = nullptr;
  double2* coef = nullptr;
  void* Alp = nullptr;
  float* scale = nullptr;
  void* work = nullptr;
  cudaStream_t st = nullptr;  // own stream (stream engine) or the group's
  bool owns_stream = false;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ready = nullptr;  // recorded on the caller's stream at submission
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float gpu_ms = 0.f;
};

}  // namespace

struct lb_server {
  int dev = 0;
  lbs::Policy pol;
  cudaMemPool_t pool = nullptr;
  int prio_least = 0, prio_greatest = 0;
  cudaStream_t cap = nullptr;  // capture-only stream of the scheduler thread
  std::mutex mu;
  std::condition_variable cv;
  std::deque<lbs::Pending> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  std::vector<Req*> done;  // completed on the GPU, not yet retired
  std::map<int, lb_basis_t*> bases;
  std::map<int, int> cluster_of_N;
  uint64_t next_id = 1;
  bool stop = false, kick = false;
  std::thread th;
  Clock::time_point t0;
  // statistics since creation or the last reset
  std::vector<double> lat;
  bool have_first = false;
  Clock::time_point t_first, t_last;
};

namespace {

struct DoneCtx {
  lb_server* s;
  std::vector<Req*> rs;
};

void CUDART_CB on_assembled(void* p) {
  auto* c = static_cast<DoneCtx*>(p);
  for (Req* r : c->rs) r->state.store(LB_REQ_ASSEMBLED);
  delete c;
}

void CUDART_CB on_done(void* p) {
  auto* c = static_cast<DoneCtx*>(p);
  const auto now = Clock::now();
  {
    // notify under the lock: once it is released the server may be destroyed
    std::lock_guard<std::mutex> lk(c->s->mu);
    for (Req* r : c->rs) {
      r->t_done = now;
      c->s->done.push_back(r);
    }
    c->s->cv.notify_all();
  }
  delete c;
}

template <class T>
cudaError_t palloc(lb_server* s, T** p, int64_t bytes, cudaStream_t st) {
  void* q = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&q, (size_t)bytes, s->pool, st);
  *p = static_cast<T*>(q);
  return e;
}

void pfree(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

void free_request_memory(Req* r) {
  pfree(r->A64, r->st);
  pfree(r->K, r->st);
  pfree(r->v, r->st);
  pfree(r->h, r->st);
  pfree(r->coef, r->st);
  pfree(r->Alp, r->st);
  pfree(r->scale, r->st);
  pfree(r->work, r->st);
  r->A64 = r->K = r->v = r->h = nullptr;
  r->coef = nullptr;
  r->Alp = r->work = nullptr;
  r->scale = nullptr;
}

// Allocation, expansion of H, assembly (closed-form kernels) and the
// low-precision pack of one request on r->st.
cudaError_t enqueue_assembly(lb_server* s, Req* r) {
  const int64_t M = r->M;
  cudaStream_t st = r->st;
  cudaError_t e;
  if ((e = palloc(s, &r->A64, 8 * M * M, st)) != cudaSuccess) return e;
  if ((e = palloc(s, &r->K, 8 * M, st)) != cudaSuccess) return e;
  if ((e = palloc(s, &r->v, 8 * M, st)) != cudaSuccess) return e;
  if (r->q.precision == LB_FP32 && (e = palloc(s, &r->Alp, 4 * M * M, st)) != cudaSuccess) return e;
  if (r->q.precision == LB_BF16) {
    if ((e = palloc(s, &r->Alp, 2 * M * M, st)) != cudaSuccess) return e;
    if ((e = palloc(s, &r->scale, 4 * M, st)) != cudaSuccess) return e;
  }
  if (r->engine == LB_ENGINE_STREAM &&
      (e = palloc(s, &r->work, (int64_t)lbi::rk4_workspace_bytes(M), st)) != cudaSuccess)
    return e;
  const lb::BasisView B = r->basis->view();
  if (r->q.H) {
    if ((e = palloc(s, &r->h, 8 * M, st)) != cudaSuccess) return e;
    if ((e = palloc(s, &r->coef, 16 * M, st)) != cudaSuccess) return e;
    if ((e = lbi::expand(B, reinterpret_cast<const double2*>(r->q.H), r->coef, st)) != cudaSuccess) return e;
    // h_m = Re coef_m (Eq. (02) on a Hermitian H is real)
    if ((e = cudaMemcpy2DAsync(r->h, sizeof(double), r->coef, sizeof(double2), sizeof(double), (size_t)M,
                               cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return e;
  }
  if ((e = lbi::assemble_dense(B, r->h, reinterpret_cast<const double2*>(r->q.a), r->A64, nullptr, nullptr, r->K,
                               LB_ALG_CLOSED, st)) != cudaSuccess)
    return e;
  if (r->q.precision == LB_FP32 && (e = lbi::pack_fp32(M, r->A64, static_cast<float*>(r->Alp), st)) != cudaSuccess)
    return e;
  if (r->q.precision == LB_BF16 &&
      (e = lbi::pack_bf16(M, r->A64, static_cast<uint16_t*>(r->Alp), r->scale, st)) != cudaSuccess)
    return e;
  return cudaMemcpyAsync(r->v, r->q.v0, 8 * M, cudaMemcpyDeviceToDevice, st);
}

int kernels_per_chunk(int precision, int correct_every, int64_t chunk) {
  int64_t k = 4 * chunk;
  if (precision != LB_FP64) k += 1;
  if (precision != LB_FP64 && correct_every > 0) k += (chunk + correct_every - 1) / correct_every;
  return (int)k;
}

// Stream engine: graph of chunk steps captured on the scheduler's capture
// stream, replayed on the request's stream.
cudaError_t enqueue_stream_rk4(lb_server* s, Req* r) {
  const int64_t M = r->M, n = r->q.nsteps;
  const int prec = r->q.precision, corr = r->q.correct_every;
  const int64_t chunk = chunk_steps(prec, corr);
  const int64_t full = n / chunk, tail = n % chunk;
  const double* A64 = prec == LB_FP64 ? nullptr : r->A64;
  const void* Ap = prec == LB_FP64 ? static_cast<const void*>(r->A64) : r->Alp;
  cudaError_t e;
  if (full > 0) {
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    const cudaError_t ec = lbi::rk4_dense(M, prec, Ap, r->scale, A64, corr, r->K, r->v, r->q.dt, chunk, nullptr, 0,
                                          r->work, s->cap);
    e = cudaStreamEndCapture(s->cap, &g);
    if (ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return ec;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&r->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    for (int64_t i = 0; i < full; ++i)
      if ((e = cudaGraphLaunch(r->exec, r->st)) != cudaSuccess) return e;
    // the capture counted one chunk's kernels; count the other replays
    lbi::note_launch((int)((full - 1) * kernels_per_chunk(prec, corr, chunk)));
  }
  if (tail > 0)
    if ((e = lbi::rk4_dense(M, prec, Ap, r->scale, A64, corr, r->K, r->v, r->q.dt, tail, nullptr, 0, r->work,
                            r->st)) != cudaSuccess)
      return e;
  return cudaSuccess;
}

void fail(Req* r, cudaError_t e, const char* what) {
  r->status = e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA;
  r->err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
}

// Stream priority by size: the cluster engine's groups first, then N <= 100,
// N <= 150, and the largest requests last.
int prio_for(const lb_server* s, int N, int engine) {
  const int hi = s->prio_greatest, lo = s->prio_least;  // hi <= lo numerically
  int p;
  if (engine == LB_ENGINE_CLUSTER) p = hi;
  else if (N <= 100) p = hi + 1;
  else if (N <= 150) p = (hi + lo) / 2 + 1;
  else p = lo;
  return std::max(hi, std::min(lo, p));
}

// Enqueue the admitted requests (called without the server lock).  Requests
// that fail to enqueue are completed with an error through the same path.
void launch(lb_server* s, const std::vector<Req*>& adm) {
  std::vector<Req*> small, big;
  for (Req* r : adm) (r->engine == LB_ENGINE_CLUSTER ? small : big).push_back(r);
  for (Req* r : big) {
    cudaError_t e = cudaStreamCreateWithPriority(&r->st, cudaStreamNonBlocking, prio_for(s, r->q.N, r->engine));
    if (e != cudaSuccess) {
      fail(r, e, "stream");
      std::lock_guard<std::mutex> lk(s->mu);
      r->t_done = Clock::now();
      s->done.push_back(r);
      continue;
    }
    r->owns_stream = true;
    cudaStreamWaitEvent(r->st, r->ready, 0);
    cudaEventCreate(&r->e0);
    cudaEventCreate(&r->e1);
    cudaEventRecord(r->e0, r->st);
    if ((e = enqueue_assembly(s, r)) != cudaSuccess) {
      fail(r, e, "assembly");
    } else {
      cudaLaunchHostFunc(r->st, on_assembled, new DoneCtx{s, {r}});
      if ((e = enqueue_stream_rk4(s, r)) != cudaSuccess) fail(r, e, "integration");
    }
    if (r->status == LB_OK)
      if ((e = cudaMemcpyAsync(r->q.v_out, r->v, 8 * r->M, cudaMemcpyDeviceToDevice, r->st)) != cudaSuccess)
        fail(r, e, "result copy");
    cudaEventRecord(r->e1, r->st);
    free_request_memory(r);
    cudaLaunchHostFunc(r->st, on_done, new DoneCtx{s, {r}});
  }
  if (small.empty()) return;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_for(s, 0, LB_ENGINE_CLUSTER));
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Req* r : small) {
      fail(r, e, "stream");
      r->t_done = Clock::now();
      s->done.push_back(r);
    }
    return;
  }
  small.front()->owns_stream = true;  // the first request of the group destroys it
  std::vector<Req*> ok;
  for (Req* r : small) {
    r->st = st;
    cudaStreamWaitEvent(st, r->ready, 0);
    cudaEventCreate(&r->e0);
    cudaEventCreate(&r->e1);
    cudaEventRecord(r->e0, st);
    if ((e = enqueue_assembly(s, r)) != cudaSuccess)
      fail(r, e, "assembly");
    else
      ok.push_back(r);
  }
  if (!ok.empty()) cudaLaunchHostFunc(st, on_assembled, new DoneCtx{s, ok});
  // one launch per (cluster size, step parameters)
  std::vector<bool> used(ok.size(), false);
  for (size_t i = 0; i < ok.size(); ++i) {
    if (used[i]) continue;
    std::vector<lbi::BatchItem> items;
    std::vector<Req*> grp;
    for (size_t j = i; j < ok.size(); ++j) {
      Req* a = ok[i];
      Req* b = ok[j];
      if (used[j] || a->cluster != b->cluster || a->q.nsteps != b->q.nsteps || a->q.dt != b->q.dt ||
          a->q.correct_every != b->q.correct_every)
        continue;
      used[j] = true;
      grp.push_back(b);
      items.push_back(lbi::BatchItem{b->M, static_cast<const float*>(b->Alp),
                                     b->q.correct_every > 0 ? b->A64 : nullptr, b->K, b->v});
    }
    e = lbi::batch_launch_async(items.data(), (int)items.size(), ok[i]->cluster, ok[i]->q.nsteps, ok[i]->q.dt,
                                ok[i]->q.correct_every, s->pool, st);
    if (e != cudaSuccess)
      for (Req* r : grp) fail(r, e, "batched integration");
  }
  for (Req* r : small) {
    if (r->status == LB_OK)
      if ((e = cudaMemcpyAsync(r->q.v_out, r->v, 8 * r->M, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        fail(r, e, "result copy");
    cudaEventRecord(r->e1, st);
    free_request_memory(r);
  }
  cudaLaunchHostFunc(st, on_done, new DoneCtx{s, small});
}

// Release what a finished request holds (called without the server lock).
void retire(Req* r) {
  if (r->e0 && r->e1 && r->status == LB_OK) cudaEventElapsedTime(&r->gpu_ms, r->e0, r->e1);
  if (r->e0) cudaEventDestroy(r->e0);
  if (r->e1) cudaEventDestroy(r->e1);
  if (r->ready) cudaEventDestroy(r->ready);
  r->e0 = r->e1 = r->ready = nullptr;
  if (r->exec) cudaGraphExecDestroy(r->exec);
  r->exec = nullptr;
  if (r->owns_stream && r->st) cudaStreamDestroy(r->st);
  r->st = nullptr;
}

void scheduler(lb_server* s) {
  cudaSetDevice(s->dev);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    if (!s->done.empty()) {
      std::vector<Req*> fin;
      fin.swap(s->done);
      lk.unlock();
      for (Req* r : fin) retire(r);
      lk.lock();
      for (Req* r : fin) {
        s->pol.release(r->bytes);
        r->state.store(r->status == LB_OK ? LB_REQ_DONE : LB_REQ_FAILED);
        if (r->status == LB_OK) {
          s->lat.push_back(ms_between(r->t_submit, r->t_done));
          s->t_last = r->t_done;
        }
      }
      s->cv.notify_all();
    }
    if (s->stop && s->queue.empty() && s->pol.inflight == 0) break;
    const double now = ms_between(s->t0, Clock::now());
    std::vector<uint64_t> ids = s->pol.admit(s->queue, now);
    if (!ids.empty()) {
      std::vector<Req*> adm;
      const auto t = Clock::now();
      for (uint64_t id : ids) {
        Req* r = s->reqs[id].get();
        r->t_admit = t;
        if (r->engine == LB_ENGINE_CLUSTER) {
          auto it = s->cluster_of_N.find(r->q.N);
          r->cluster = it != s->cluster_of_N.end() ? it->second : lbi::batch_default_cluster(r->M);
        }
        r->state.store(LB_REQ_RUNNING);
        adm.push_back(r);
      }
      lk.unlock();
      launch(s, adm);
      lk.lock();
      continue;
    }
    s->kick = false;
    s->cv.wait_for(lk, std::chrono::milliseconds(1), [&] { return !s->done.empty() || s->stop || s->kick; });
  }
}

}  // namespace

extern "C" {

int64_t lb_request_bytes(int N, int precision, int with_H) {
  if (N < 2 || N > lbi::kMaxDenseN || precision < LB_FP64 || precision > LB_BF16) return -1;
  return footprint(N, precision, with_H != 0);
}

int lb_server_create(int64_t budget_bytes, int slots, double bypass_ms, lb_server_t** out) {
  if (!out || budget_bytes <= 0 || slots < 1 || !(bypass_ms >= 0.0)) {
    lbi::set_error("lb_server_create: bad arguments");
    return LB_EINVAL;
  }
  *out = nullptr;
  auto s = std::make_unique<lb_server>();
  cudaError_t e = cudaGetDevice(&s->dev);
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&s->prio_least, &s->prio_greatest);
  if (e == cudaSuccess) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->dev;
    e = cudaMemPoolCreate(&s->pool, &props);
  }
  if (e == cudaSuccess) {
    uint64_t keep = (uint64_t)budget_bytes;  // keep up to the budget mapped between requests
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e == cudaSuccess) {
    int on = 1;
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowOpportunistic, &on);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (s->pool) cudaMemPoolDestroy(s->pool);
    return lbi::cuda_fail(e, "lb_server_create");
  }
  s->pol.budget = budget_bytes;
  s->pol.slots = slots;
  s->pol.bypass_ms = bypass_ms;
  s->t0 = Clock::now();
  lb_server* raw = s.release();
  raw->th = std::thread(scheduler, raw);
  *out = raw;
  return LB_OK;
}

int lb_server_set_cluster(lb_server_t* s, int N, int C) {
  if (!s || N < 2 || N > lbi::kBatchMaxN || !(C == 1 || C == 2 || C == 4 || C == 8 || C == 16)) {
    lbi::set_error("lb_server_set_cluster: bad arguments");
    return LB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->cluster_of_N[N] = C;
  return LB_OK;
}

int lb_submit(lb_server_t* s, const lb_request* q, uint64_t* id) {
  if (!s || !q || !id || q->N < 2 || q->N > lbi::kMaxDenseN || !q->a || !q->v0 || !q->v_out || q->nsteps < 0 ||
      !(q->dt == q->dt) || q->precision < LB_FP64 || q->precision > LB_BF16 || q->correct_every < 0) {
    lbi::set_error("lb_submit: bad request");
    return LB_EINVAL;
  }
  const int64_t bytes = footprint(q->N, q->precision, q->H != nullptr);
  if (bytes > s->pol.budget) {
    lbi::set_error("lb_submit: request needs %lld bytes, above the server budget %lld", (long long)bytes,
                   (long long)s->pol.budget);
    return LB_ENOMEM;
  }
  lb_basis_t* basis = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      lbi::set_error("lb_submit: server is shutting down");
      return LB_EINVAL;
    }
    auto it = s->bases.find(q->N);
    if (it != s->bases.end()) basis = it->second;
  }
  if (!basis) {
    int rc = lb_basis_create(q->N, nullptr, &basis);
    if (rc != LB_OK) return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->bases.find(q->N);
    if (it != s->bases.end()) {
      lb_basis_destroy(basis);
      basis = it->second;
    } else {
      s->bases[q->N] = basis;
    }
  }
  auto r = std::make_unique<Req>();
  cudaError_t e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r->ready, static_cast<cudaStream_t>(q->stream));
  if (e != cudaSuccess) {
    if (r->ready) cudaEventDestroy(r->ready);
    return lbi::cuda_fail(e, "lb_submit: input-ready event");
  }
  r->q = *q;
  r->M = (int64_t)q->N * q->N - 1;
  r->bytes = bytes;
  r->engine = engine_of(q->N, q->precision);
  r->basis = basis;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    *id = r->id;
    if (!s->have_first) {
      s->have_first = true;
      s->t_first = r->t_submit;
    }
    s->queue.push_back(lbs::Pending{r->id, bytes, ms_between(s->t0, r->t_submit)});
    s->reqs[r->id] = std::move(r);
    s->kick = true;
  }
  s->cv.notify_all();
  return LB_OK;
}

static void fill_result(const Req* r, lb_result* out) {
  out->state = r->state.load();
  out->status = r->status;
  out->engine = r->engine;
  out->cluster = r->cluster;
  const bool admitted = out->state != LB_REQ_QUEUED && out->state != LB_REQ_CANCELLED;
  const bool fin = out->state == LB_REQ_DONE || out->state == LB_REQ_FAILED;
  out->queue_ms = admitted ? ms_between(r->t_submit, r->t_admit) : 0.0;
  out->latency_ms = fin ? ms_between(r->t_submit, r->t_done) : 0.0;
  out->gpu_ms = fin ? r->gpu_ms : 0.0;
}

int lb_poll(lb_server_t* s, uint64_t id, lb_result* out) {
  if (!s || !out) {
    lbi::set_error("lb_poll: NULL argument");
    return LB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    lbi::set_error("lb_poll: unknown request %llu", (unsigned long long)id);
    return LB_EINVAL;
  }
  fill_result(it->second.get(), out);
  if (out->state == LB_REQ_FAILED) {
    lbi::set_error("request %llu failed: %s", (unsigned long long)id, it->second->err.c_str());
    return it->second->status;
  }
  return out->state == LB_REQ_DONE ? LB_OK : LB_EAGAIN;
}

int lb_wait(lb_server_t* s, uint64_t id, double timeout_ms, lb_result* out) {
  if (!s || !out || !(timeout_ms >= 0.0)) {
    lbi::set_error("lb_wait: bad arguments");
    return LB_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    lbi::set_error("lb_wait: unknown request %llu", (unsigned long long)id);
    return LB_EINVAL;
  }
  Req* r = it->second.get();
  auto finished = [&] {
    const int st = r->state.load();
    return st == LB_REQ_DONE || st == LB_REQ_FAILED || st == LB_REQ_CANCELLED;
  };
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), finished);
  fill_result(r, out);
  if (!ok) {
    lbi::set_error("lb_wait: request %llu not finished after %.1f ms", (unsigned long long)id, timeout_ms);
    return LB_ETIMEOUT;
  }
  if (out->state == LB_REQ_FAILED) {
    lbi::set_error("request %llu failed: %s", (unsigned long long)id, r->err.c_str());
    return r->status;
  }
  if (out->state == LB_REQ_CANCELLED) {
    lbi::set_error("request %llu was cancelled", (unsigned long long)id);
    return LB_EINVAL;
  }
  return LB_OK;
}

int lb_server_stats(lb_server_t* s, double* p50_ms, double* p99_ms, double* throughput, int64_t* completed) {
  if (!s) {
    lbi::set_error("lb_server_stats: NULL server");
    return LB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (p50_ms) *p50_ms = lbs::percentile(s->lat, 50.0);
  if (p99_ms) *p99_ms = lbs::percentile(s->lat, 99.0);
  if (completed) *completed = (int64_t)s->lat.size();
  if (throughput) {
    const double span = s->lat.empty() ? 0.0 : ms_between(s->t_first, s->t_last);
    *throughput = span > 0.0 ? 1000.0 * (double)s->lat.size() / span : 0.0;
  }
  return LB_OK;
}

int lb_server_reset_stats(lb_server_t* s) {
  if (!s) {
    lbi::set_error("lb_server_reset_stats: NULL server");
    return LB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat.clear();
  s->have_first = false;
  return LB_OK;
}

int lb_server_destroy(lb_server_t* s) {
  if (!s) return LB_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (const lbs::Pending& p : s->queue) {
      Req* r = s->reqs[p.id].get();
      r->state.store(LB_REQ_CANCELLED);
      if (r->ready) cudaEventDestroy(r->ready);
      r->ready = nullptr;
    }
    s->queue.clear();
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();  // admitted work is finite: the loop ends when it has drained
  for (auto& kv : s->bases) lb_basis_destroy(kv.second);
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
  return LB_OK;
}

int lb_sched_simulate(int n, const double* arrival_ms, const int64_t* bytes, const double* service_ms,
                      int64_t budget, int slots, double bypass_ms, double* start_ms, double* finish_ms) {
  if (n < 0 || (n > 0 && (!arrival_ms || !bytes || !service_ms || !start_ms || !finish_ms)) || budget <= 0 ||
      slots < 1 || !(bypass_ms >= 0.0)) {
    lbi::set_error("lb_sched_simulate: bad arguments");
    return LB_EINVAL;
  }
  for (int i = 1; i < n; ++i)
    if (arrival_ms[i] < arrival_ms[i - 1]) {
      lbi::set_error("lb_sched_simulate: arrivals must be non-decreasing");
      return LB_EINVAL;
    }
  lbs::simulate(n, arrival_ms, bytes, service_ms, budget, slots, bypass_ms, start_ms, finish_ms);
  return LB_OK;
}

}  // extern "C"

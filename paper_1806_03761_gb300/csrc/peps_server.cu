// peps_server.cu -- the serving loop (include/peps.h, "Serving"): a worker
// thread that admits evaluation jobs of any shape under an HBM budget, keeps
// their tensors and environments resident, and interleaves their waves on
// the device (continuous batching).  Host code only: the device work is the
// library's own peps_local_energy launches, one stream per admitted job.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/peps.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Contexts are pooled by shape and wave size: a finished job's context (its
// converted tensors and environment workspace) stays allocated for the next
// job of the same shape, so that admission does not free device memory
// (cudaFree waits for the whole device) unless the budget requires it.
typedef std::tuple<int, int, int, double, double, int, int> CtxKey;

CtxKey key_of(const peps_shape& s, int slots) {
  return CtxKey(s.L, s.D, s.Dc, s.J1, s.J2, s.precision, slots);
}

struct Job {
  int64_t id = 0;
  peps_job spec;
  int slots = 0;
  size_t ctx_bytes = 0, buf_bytes = 0;
  // device state while admitted
  peps_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool inflight = false;
  int64_t next = 0;
  double* dA = nullptr;
  uint8_t* dspins = nullptr;
  double* de = nullptr;
  double* dla = nullptr;
  int8_t* dsg = nullptr;
  bool done = false;
  peps_job_stats st;
};

struct IdleCtx {
  CtxKey key;
  peps_ctx* ctx;
  size_t bytes;
};

}  // namespace

struct peps_server {
  int device = 0;
  int default_slots = 0;
  size_t budget = 0;
  size_t active_bytes = 0, idle_bytes = 0;
  int64_t next_id = 1;
  bool stop = false, reap_stop = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> pending;
  std::vector<Job*> active;
  std::map<int64_t, Job*> jobs;
  std::vector<IdleCtx> idle;  // least recently used first
  // evicted contexts on their way out: freed by the reaper thread, so that
  // cudaFree (which waits for the whole device) never stalls the worker;
  // their bytes stay reserved until the memory is back
  std::deque<IdleCtx> reap;
  size_t reaping_bytes = 0;
  std::condition_variable cv_reap;
  std::thread worker, reaper;

  void run();
  void reap_loop();
  bool admit(Job* j);
  void finish(Job* j, int status);
  void release(Job* j);
};

namespace {

size_t tensor_bytes(const peps_shape& s) {
  const size_t D4 = (size_t)s.D * s.D * s.D * s.D;
  return (size_t)s.L * s.L * 2 * D4 * 8;
}

}  // namespace

// Device resources of an admitted job: a pooled or new context, a stream,
// the staged inputs and the outputs.  Called by the worker with the lock
// released; the budget was reserved by the caller.
bool peps_server::admit(Job* j) {
  const peps_shape& s = j->spec.shape;
  const int64_t N = (int64_t)s.L * s.L, B = j->spec.B;
  j->st.admit_s = now_s();
  if (!j->ctx) {
    int rc = peps_create(&s, j->slots, &j->ctx);
    if (rc != PEPS_OK) {
      j->ctx = nullptr;
      finish(j, rc);
      return false;
    }
  }
  if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
    finish(j, PEPS_ECUDA);
    return false;
  }
  bool ok = cudaMallocAsync((void**)&j->dA, tensor_bytes(s), j->stream) == cudaSuccess &&
            cudaMallocAsync((void**)&j->dspins, (size_t)(B * N), j->stream) == cudaSuccess &&
            cudaMallocAsync((void**)&j->de, (size_t)B * 8, j->stream) == cudaSuccess &&
            cudaMallocAsync((void**)&j->dla, (size_t)B * 8, j->stream) == cudaSuccess &&
            cudaMallocAsync((void**)&j->dsg, (size_t)B, j->stream) == cudaSuccess;
  if (!ok) {
    finish(j, PEPS_ENOMEM);
    return false;
  }
  ok = cudaMemcpyAsync(j->dA, j->spec.A, tensor_bytes(s), cudaMemcpyHostToDevice, j->stream) == cudaSuccess &&
       cudaMemcpyAsync(j->dspins, j->spec.spins, (size_t)(B * N), cudaMemcpyHostToDevice, j->stream) == cudaSuccess;
  if (!ok) {
    finish(j, PEPS_ECUDA);
    return false;
  }
  int rc = peps_set_tensors(j->ctx, j->dA, j->stream);
  if (rc != PEPS_OK) {
    finish(j, rc);
    return false;
  }
  return true;
}

// Free a job's per-job device state and return its context to the pool.
// Nothing here waits: the frees are stream-ordered (they take effect when the
// job's stream reaches them) and cudaStreamDestroy returns at once, the
// stream's resources being released when its work is done.
void peps_server::release(Job* j) {
  if (j->stream) {
    if (j->dA) cudaFreeAsync(j->dA, j->stream);
    if (j->dspins) cudaFreeAsync(j->dspins, j->stream);
    if (j->de) cudaFreeAsync(j->de, j->stream);
    if (j->dla) cudaFreeAsync(j->dla, j->stream);
    if (j->dsg) cudaFreeAsync(j->dsg, j->stream);
    cudaStreamDestroy(j->stream);
  }
  if (j->ev) cudaEventDestroy(j->ev);
  j->dA = nullptr; j->dspins = nullptr; j->de = nullptr; j->dla = nullptr; j->dsg = nullptr;
  j->stream = nullptr;
  j->ev = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  active_bytes -= j->ctx_bytes + j->buf_bytes;
  if (j->ctx) {
    idle.push_back(IdleCtx{key_of(j->spec.shape, j->slots), j->ctx, j->ctx_bytes});
    idle_bytes += j->ctx_bytes;
    j->ctx = nullptr;
  }
}

void peps_server::finish(Job* j, int status) {
  j->st.status = status;
  j->st.done_s = now_s();
  release(j);
  std::lock_guard<std::mutex> lock(mu);
  j->done = true;
  cv_done.notify_all();
}

void peps_server::run() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<Job*> admitted;
    int evicted = 0;
    {
      std::unique_lock<std::mutex> lock(mu);
      // admission in arrival order while the budget allows
      while (!pending.empty()) {
        Job* j = pending.front();
        const CtxKey k = key_of(j->spec.shape, j->slots);
        int reuse = -1;
        for (int q = (int)idle.size() - 1; q >= 0; --q)
          if (idle[q].key == k) { reuse = q; break; }
        const size_t need = j->buf_bytes + (reuse >= 0 ? 0 : j->ctx_bytes);
        // evict idle contexts (least recently used first) while they stand
        // between this job and the budget
        size_t freeable = idle_bytes - (reuse >= 0 ? idle[reuse].bytes : 0);
        if (active_bytes + idle_bytes + reaping_bytes + need > budget + freeable) break;
        for (int q = 0; active_bytes + idle_bytes + reaping_bytes + need > budget && q < (int)idle.size();) {
          if (q == reuse) { ++q; continue; }
          reap.push_back(idle[q]);
          reaping_bytes += idle[q].bytes;
          idle_bytes -= idle[q].bytes;
          idle.erase(idle.begin() + q);
          if (reuse > q) --reuse;
          ++evicted;
        }
        // the evicted memory is not back yet: admit once the reaper has
        // freed enough of it (the other jobs keep running meanwhile)
        if (active_bytes + idle_bytes + reaping_bytes + need > budget) break;
        if (reuse >= 0) {
          j->ctx = idle[reuse].ctx;
          idle_bytes -= idle[reuse].bytes;
          idle.erase(idle.begin() + reuse);
        }
        active_bytes += j->ctx_bytes + j->buf_bytes;
        pending.pop_front();
        admitted.push_back(j);
      }
      if (stop && pending.empty() && active.empty() && admitted.empty()) break;
    }
    if (evicted) cv_reap.notify_one();
    for (Job* j : admitted)
      if (admit(j)) active.push_back(j);
    // progress: one wave in flight per job
    bool progressed = !admitted.empty();
    for (size_t q = 0; q < active.size();) {
      Job* j = active[q];
      if (j->inflight) {
        if (cudaEventQuery(j->ev) == cudaErrorNotReady) { ++q; continue; }
        j->inflight = false;
      }
      progressed = true;
      const int64_t N = (int64_t)j->spec.shape.L * j->spec.shape.L, B = j->spec.B;
      if (j->next < B) {
        const int64_t nb = std::min<int64_t>(j->slots, B - j->next);
        int rc = peps_local_energy(j->ctx, j->dspins + j->next * N, nb, j->de + j->next,
                                   j->dla + j->next, j->dsg + j->next, nullptr, nullptr, j->stream);
        if (rc == PEPS_OK && cudaEventRecord(j->ev, j->stream) != cudaSuccess) rc = PEPS_ECUDA;
        if (rc != PEPS_OK) {
          active.erase(active.begin() + q);
          finish(j, rc);
          continue;
        }
        j->inflight = true;
        j->next += nb;
        ++q;
        continue;
      }
      // every wave done: status, results to the host, resources back
      int32_t flags = 0;
      int rc = peps_sync_status(j->ctx, j->stream, &flags);
      j->st.flags = flags;
      if (rc == PEPS_OK || rc == PEPS_ENUMERIC) {
        bool ok = cudaMemcpy(j->spec.e_loc, j->de, (size_t)B * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
        if (ok && j->spec.log_abs)
          ok = cudaMemcpy(j->spec.log_abs, j->dla, (size_t)B * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
        if (ok && j->spec.sign)
          ok = cudaMemcpy(j->spec.sign, j->dsg, (size_t)B, cudaMemcpyDeviceToHost) == cudaSuccess;
        if (!ok) rc = PEPS_ECUDA;
      }
      active.erase(active.begin() + q);
      finish(j, rc);
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lock(mu);
      if (pending.empty() || !active.empty() || reaping_bytes > 0)
        cv_work.wait_for(lock, std::chrono::microseconds(200));
    }
  }
  {
    std::lock_guard<std::mutex> lock(mu);
    reap_stop = true;
  }
  cv_reap.notify_one();
}

// The reaper: destroys evicted contexts (peps_destroy -> cudaFree) off the
// worker thread and hands their bytes back to the budget.
void peps_server::reap_loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lock(mu);
  for (;;) {
    cv_reap.wait(lock, [this] { return !reap.empty() || reap_stop; });
    if (reap.empty()) break;
    IdleCtx c = reap.front();
    reap.pop_front();
    lock.unlock();
    peps_destroy(c.ctx);
    lock.lock();
    reaping_bytes -= c.bytes;
    cv_work.notify_one();
  }
}

extern "C" {

int peps_server_create(size_t hbm_budget_bytes, int32_t slots_per_job, peps_server** out) {
  if (!out || slots_per_job < 0) return PEPS_EINVAL;
  *out = nullptr;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PEPS_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PEPS_ECUDA;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return PEPS_ECUDA;
  peps_server* s = new (std::nothrow) peps_server();
  if (!s) return PEPS_ENOMEM;
  s->device = dev;
  s->default_slots = slots_per_job > 0 ? slots_per_job : 2 * sms;
  s->budget = hbm_budget_bytes > 0 ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
  s->reaper = std::thread([s] { s->reap_loop(); });
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return PEPS_OK;
}

int peps_server_submit(peps_server* s, const peps_job* job, int64_t* job_id) {
  if (!s || !job || !job_id) return PEPS_EINVAL;
  const peps_shape& sh = job->shape;
  if (job->B < 1 || !job->A || !job->spins || !job->e_loc) return PEPS_EINVAL;
  const int slots = (int)std::min<int64_t>(job->B, s->default_slots);
  const size_t ws = peps_workspace_bytes(&sh, slots);
  if (ws == 0) return PEPS_EINVAL;  // invalid shape
  Job* j = new (std::nothrow) Job();
  if (!j) return PEPS_ENOMEM;
  const int64_t N = (int64_t)sh.L * sh.L;
  j->spec = *job;
  j->slots = slots;
  j->ctx_bytes = ws + tensor_bytes(sh);
  j->buf_bytes = tensor_bytes(sh) + (size_t)(job->B * N) + (size_t)job->B * 17;
  std::memset(&j->st, 0, sizeof(j->st));
  j->st.footprint_bytes = (int64_t)(j->ctx_bytes + j->buf_bytes);
  if (j->ctx_bytes + j->buf_bytes > s->budget) {
    delete j;
    return PEPS_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    j->id = s->next_id++;
    j->st.submit_s = now_s();
    s->jobs[j->id] = j;
    s->pending.push_back(j);
  }
  s->cv_work.notify_one();
  *job_id = j->id;
  return PEPS_OK;
}

int peps_server_wait(peps_server* s, int64_t job_id, double timeout_s, peps_job_stats* stats) {
  if (!s) return PEPS_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return PEPS_EINVAL;
  Job* j = it->second;
  if (timeout_s > 0) {
    if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [j] { return j->done; }))
      return PEPS_ETIMEOUT;
  } else {
    s->cv_done.wait(lock, [j] { return j->done; });
  }
  if (stats) *stats = j->st;
  const int rc = j->st.status;
  s->jobs.erase(it);
  delete j;
  return rc;
}

int peps_server_destroy(peps_server* s) {
  if (!s) return PEPS_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->reaper.joinable()) s->reaper.join();
  cudaSetDevice(s->device);
  for (IdleCtx& c : s->idle) peps_destroy(c.ctx);
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
  return PEPS_OK;
}

}  // extern "C"

// Simulation server with continuous batching (C ABI lbm_server_*, declared
// in include/d2q37.h).
//
// Jobs (lattice size, step count, parameters, precision, seed) are queued on
// submission and admitted in arrival order, skipping ahead to any later job
// that fits, whenever their device memory fits in the free part of one
// pre-allocated pool (the HBM budget; first-fit with coalescing).  Admitted
// jobs keep their state on the device.  Each tick advances every active job
// by min(steps per tick, its steps left) steps through its own handle's step
// (replays of captured 16- and 2-step graphs of the fused step) on the job's
// stream: one of kStreams streams, assigned at admission to the one with the
// fewest active sites, so that the jobs run side by side (on GB300 per-job
// launches beat one batched launch per step over all jobs by 14-30 %).  A job
// that reaches its step count has its fields computed into its scratch and
// an event recorded behind them; a later tick, once the event has passed,
// copies them to host memory and returns the job's device memory to the pool,
// so that queued jobs can be admitted into it.  Ticks do not wait for the GPU
// except to stay at most two ticks ahead of it.
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "d2q37_handle.h"

namespace {

constexpr int kStreams = 8;
constexpr int kTicksAhead = 2;  // ticks the host may enqueue ahead of the GPU

struct Job {
  int64_t id;
  int Lx, Ly, steps_total, steps_left;
  lbm_params prm;
  uint64_t seed;
  int state;  // LBM_JOB_*
  size_t bytes, offset;
  lbm_t* h;
  int stream;  // index into lbm_server_t::stream
  bool draining;        // fields enqueued into the scratch, waiting for done_ev
  cudaEvent_t done_ev;  // recorded behind the fields kernel
  std::vector<double> rho, u, T;  // results once done
};

// First-fit allocator over [0, size) with coalescing of freed ranges.
class Pool {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t start = it->first + bytes;
      free_.erase(it);
      if (rest) free_[start] = rest;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (const auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  std::map<size_t, size_t> free_;
};

size_t round256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

struct lbm_server_t {
  size_t budget, in_use;
  char* pool_mem;
  Pool pool;
  int max_steps_per_tick;
  int64_t next_id;
  std::deque<Job*> queue;
  std::vector<Job*> active;
  std::unordered_map<int64_t, Job*> jobs;
  std::vector<int64_t> finished;  // not yet reported by lbm_server_poll
  cudaStream_t stream[kStreams];
  long long stream_sites[kStreams];  // sites of the active jobs on each stream
  cudaEvent_t tick_ev[kTicksAhead][kStreams];  // the end of each stream's work of recent ticks
  bool tick_ev_used[kTicksAhead];
  lbm_server_stats stats;
};

namespace {

void release_job_memory(lbm_server_t* s, Job* j) {
  if (j->done_ev) {
    cudaEventDestroy(j->done_ev);
    j->done_ev = nullptr;
  }
  if (j->h) {
    lbm_destroy(j->h);
    j->h = nullptr;
  }
  if (j->bytes) {
    s->pool.release(j->offset, j->bytes);
    s->in_use -= j->bytes;
    j->bytes = 0;
  }
}

// Admit queued jobs in arrival order while memory allows (skipping jobs that
// do not fit yet).
int admit(lbm_server_t* s) {
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    Job* j = *it;
    const size_t need = round256(lbm_required_bytes(j->Lx, j->Ly, &j->prm));
    size_t off = 0;
    if (!s->pool.alloc(need, &off)) {
      ++it;
      continue;
    }
    j->offset = off;
    j->bytes = need;
    s->in_use += need;
    j->stream = (int)(std::min_element(s->stream_sites, s->stream_sites + kStreams) - s->stream_sites);
    cudaStream_t st = s->stream[j->stream];
    int rc = lbm_create_ext(j->Lx, j->Ly, &j->prm, s->pool_mem + off, need, st, &j->h);
    if (!rc) rc = lbm_init_rayleigh_taylor(j->h, j->seed);
    if (!rc) rc = handle_prepare_halos(j->h, st);
    if (rc) {
      release_job_memory(s, j);
      return rc;
    }
    s->stream_sites[j->stream] += (long long)j->Lx * j->Ly;
    j->state = LBM_JOB_ACTIVE;
    s->active.push_back(j);
    it = s->queue.erase(it);
  }
  return LBM_OK;
}

// Jobs whose fields are ready: copy them to host memory, return the device
// memory.  block: wait for the first draining job if none is ready.
int finalize(lbm_server_t* s, bool block) {
  bool any = false;
  for (int pass = 0; pass < 2 && !any; ++pass) {
    for (Job* j : s->active) {
      if (!j->draining) continue;
      cudaError_t e = cudaEventQuery(j->done_ev);
      if (e == cudaErrorNotReady && pass == 1 && block) e = cudaEventSynchronize(j->done_ev);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) return LBM_ECUDA;
      const size_t n = (size_t)j->Lx * j->Ly;
      j->rho.resize(n);
      j->u.resize(2 * n);
      j->T.resize(n);
      const double* sc = j->h->scratch;  // rho, ux, uy, T planes
      if (cudaMemcpy(j->rho.data(), sc, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(j->u.data(), sc + n, 2 * n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(j->T.data(), sc + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return LBM_ECUDA;
      s->stream_sites[j->stream] -= (long long)j->Lx * j->Ly;
      release_job_memory(s, j);
      j->state = LBM_JOB_DONE;
      j->draining = false;
      s->finished.push_back(j->id);
      s->stats.completed++;
      any = true;
      if (pass == 1) break;  // one blocking wait per call
    }
    if (!block) break;
  }
  if (any)
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(),
                                   [](Job* j) { return j->state == LBM_JOB_DONE; }),
                    s->active.end());
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_server_create(size_t hbm_budget_bytes, int max_steps_per_tick, lbm_server_t** out) {
  if (!out || hbm_budget_bytes < 4096 || max_steps_per_tick <= 0) return LBM_EINVAL;
  int rc = handle_device_consts();
  if (rc) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
  lbm_server_t* s = new lbm_server_t();
  s->budget = hbm_budget_bytes & ~size_t(255);
  s->max_steps_per_tick = max_steps_per_tick;
  s->next_id = 1;
  if (cudaMalloc(&s->pool_mem, s->budget) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return LBM_ENOMEM;
  }
  s->pool.reset(s->budget);
  for (int g = 0; g < kStreams && !rc; ++g) {
    if (cudaStreamCreateWithFlags(&s->stream[g], cudaStreamNonBlocking) != cudaSuccess) rc = LBM_ECUDA;
    for (int a = 0; a < kTicksAhead && !rc; ++a)
      if (cudaEventCreateWithFlags(&s->tick_ev[a][g], cudaEventDisableTiming) != cudaSuccess) rc = LBM_ECUDA;
  }
  if (rc) {
    lbm_server_destroy(s);
    return rc;
  }
  s->stats.budget_bytes = s->budget;
  *out = s;
  return LBM_OK;
}

int lbm_server_submit(lbm_server_t* s, int Lx, int Ly, int steps, const lbm_params* p, uint64_t seed,
                      int64_t* job_id) {
  if (!s || !p || steps < 0 || !job_id) return LBM_EINVAL;
  const size_t need = lbm_required_bytes(Lx, Ly, p);
  if (!need) return LBM_EINVAL;
  if (round256(need) > s->budget) return LBM_ENOMEM;  // could never be admitted
  Job* j = new Job();
  j->id = s->next_id++;
  j->Lx = Lx;
  j->Ly = Ly;
  j->steps_total = j->steps_left = steps;
  j->prm = *p;
  j->prm.kernel = LBM_KERNEL_FUSED;
  j->seed = seed;
  j->state = LBM_JOB_QUEUED;
  s->jobs[j->id] = j;
  s->queue.push_back(j);
  s->stats.submitted++;
  *job_id = j->id;
  return LBM_OK;
}

int lbm_server_tick(lbm_server_t* s, int* steps_done) {
  const TraceRange trace("lbm_server_tick");
  if (!s) return LBM_EINVAL;
  if (steps_done) *steps_done = 0;
  int rc = finalize(s, false);
  if (!rc) rc = admit(s);
  if (rc) return rc;
  if (s->active.empty()) return LBM_OK;
  // stay at most kTicksAhead ticks ahead of the GPU
  const int slot = (int)(s->stats.ticks % kTicksAhead);
  if (s->tick_ev_used[slot])
    for (int g = 0; g < kStreams; ++g)
      if (cudaEventSynchronize(s->tick_ev[slot][g]) != cudaSuccess) return LBM_ECUDA;
  // each job's steps in order on its stream (lbm_step: replays of its captured
  // graphs); the streams run side by side.  A job that reaches its step count
  // gets its fields computed into its scratch, and an event behind them.
  int kmax = 0;
  for (Job* j : s->active) {
    if (j->draining) continue;
    const int k = std::min(s->max_steps_per_tick, j->steps_left);
    if (k > 0) {
      const int64_t before = j->h->launches;
      rc = lbm_step(j->h, k);
      if (rc) return rc;
      s->stats.launches += j->h->launches - before;
      j->steps_left -= k;
      s->stats.steps += k;
      kmax = std::max(kmax, k);
    }
    if (j->steps_left == 0) {
      const size_t n = (size_t)j->Lx * j->Ly;
      double* sc = j->h->scratch;
      rc = lbm_fields_device(j->h, sc, sc + n, sc + 3 * n);
      if (!rc && cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming) != cudaSuccess) rc = LBM_ECUDA;
      if (!rc && cudaEventRecord(j->done_ev, s->stream[j->stream]) != cudaSuccess) rc = LBM_ECUDA;
      if (rc) return rc;
      j->draining = true;
    }
  }
  for (int g = 0; g < kStreams; ++g)
    if (cudaEventRecord(s->tick_ev[slot][g], s->stream[g]) != cudaSuccess) return LBM_ECUDA;
  s->tick_ev_used[slot] = true;
  s->stats.ticks++;
  if (kmax == 0) {
    // only jobs whose fields are on their way: wait for the first of them
    rc = finalize(s, true);
    if (rc) return rc;
  }
  if (steps_done) *steps_done = kmax;
  return LBM_OK;
}

int lbm_server_poll(lbm_server_t* s, int64_t* ids, int max_ids, int* n) {
  if (!s || !n || (max_ids > 0 && !ids)) return LBM_EINVAL;
  const int m = std::min<int>(max_ids, (int)s->finished.size());
  for (int i = 0; i < m; ++i) ids[i] = s->finished[i];
  s->finished.erase(s->finished.begin(), s->finished.begin() + m);
  *n = m;
  return LBM_OK;
}

int lbm_server_job_state(const lbm_server_t* s, int64_t id, int* state, int* steps_left) {
  if (!s || !state) return LBM_EINVAL;
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return LBM_EINVAL;
  *state = it->second->state;
  if (steps_left) *steps_left = it->second->steps_left;
  return LBM_OK;
}

int lbm_server_fetch(lbm_server_t* s, int64_t id, double* rho, double* u, double* T) {
  if (!s || !rho || !u || !T) return LBM_EINVAL;
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return LBM_EINVAL;
  Job* j = it->second;
  if (j->state != LBM_JOB_DONE) return LBM_ESTATE;
  std::memcpy(rho, j->rho.data(), j->rho.size() * sizeof(double));
  std::memcpy(u, j->u.data(), j->u.size() * sizeof(double));
  std::memcpy(T, j->T.data(), j->T.size() * sizeof(double));
  s->jobs.erase(it);
  delete j;
  return LBM_OK;
}

int lbm_server_stats_get(const lbm_server_t* s, lbm_server_stats* out) {
  if (!s || !out) return LBM_EINVAL;
  *out = s->stats;
  out->queued = (int64_t)s->queue.size();
  out->active = (int64_t)s->active.size();
  out->bytes_in_use = s->in_use;
  out->largest_free_bytes = s->pool.largest();
  return LBM_OK;
}

void lbm_server_destroy(lbm_server_t* s) {
  if (!s) return;
  for (int g = 0; g < kStreams; ++g)
    if (s->stream[g]) cudaStreamSynchronize(s->stream[g]);
  for (auto& kv : s->jobs) {
    if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
    if (kv.second->h) lbm_destroy(kv.second->h);
    delete kv.second;
  }
  for (int g = 0; g < kStreams; ++g) {
    if (s->stream[g]) cudaStreamDestroy(s->stream[g]);
    for (int a = 0; a < kTicksAhead; ++a)
      if (s->tick_ev[a][g]) cudaEventDestroy(s->tick_ev[a][g]);
  }
  if (s->pool_mem) cudaFree(s->pool_mem);
  delete s;
}

}  // extern "C"

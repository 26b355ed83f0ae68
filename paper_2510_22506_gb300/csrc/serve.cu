// Serving loop: continuous batching of completion jobs on one GPU.
//
// Jobs of any order, size, rank and sampling rate are submitted at any time.
// A job is admitted when a slot is free and its device footprint
// (fctn_footprint_bytes) fits the memory budget; it then owns a handle whose
// factors, X and mask stay resident on the device until its result is taken.
// Every admitted job runs on its own stream and each of its sweeps is one
// CUDA-graph launch, so the sweeps of different jobs overlap on the device;
// finished jobs leave and waiting jobs take their slot and memory without
// waiting for the rest.  The stop test (rel_change <= tol, or the sweep cap)
// is read from a pinned copy of each job's last-sweep values.
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fctn_internal.cuh"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
  uint64_t id = 0;
  fctn_params p{};
  double tol = 0.0;
  int max_sweeps = 0;
  int state = FCTN_JOB_QUEUED;
  int status = FCTN_OK;
  std::vector<unsigned char> Y, mask;
  std::vector<std::vector<unsigned char>> factors;
  size_t footprint = 0;
  fctn_handle* h = nullptr;
  double* pinned = nullptr;  // {rel, objective, data, nonfinite, status bits, t}
  cudaEvent_t ev = nullptr;
  bool inflight = false;
  int64_t t = 0;
  double rel = 0.0, objective = 0.0, data = 0.0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  std::string err;
};

}  // namespace

struct fctn_server {
  fctn_server_config cfg{};
  std::mutex mu;
  uint64_t next_id = 1;
  std::deque<uint64_t> queue;
  std::map<uint64_t, Job> jobs;
  size_t used = 0;
  int active = 0;
  int64_t sweeps_launched = 0;
  std::vector<uint64_t> finished;  // jobs that reached DONE / FAILED, not yet reported
};

namespace {

int svr_fail(int code, const std::string& m) { return fctn_internal_fail(code, m.c_str()); }

void release(fctn_server* S, Job& j) {
  if (j.h) {
    fctn_destroy(j.h);
    j.h = nullptr;
    S->used -= j.footprint;
    S->active--;
  }
  if (j.ev) {
    cudaEventDestroy(j.ev);
    j.ev = nullptr;
  }
  if (j.pinned) {
    cudaFreeHost(j.pinned);
    j.pinned = nullptr;
  }
}

void finish(fctn_server* S, Job& j, int state, int status, const char* msg) {
  S->finished.push_back(j.id);
  j.state = state;
  j.status = status;
  j.t_done = now_s();
  if (msg) j.err = msg;
  // keep the handle (X stays resident) until fctn_server_result; drop staging
  std::vector<unsigned char>().swap(j.Y);
  std::vector<unsigned char>().swap(j.mask);
  j.factors.clear();
  if (state == FCTN_JOB_FAILED) release(S, j);
}

int admit(fctn_server* S, Job& j) {
  fctn_handle* h = nullptr;
  int rc = fctn_create(&j.p, nullptr, &h);
  if (rc) return rc;
  j.h = h;
  S->used += j.footprint;
  S->active++;
  if (cudaHostAlloc((void**)&j.pinned, 8 * sizeof(double), cudaHostAllocDefault) != cudaSuccess)
    return svr_fail(FCTN_E_OOM, "pinned stats buffer");
  memset(j.pinned, 0, 8 * sizeof(double));
  if (cudaEventCreateWithFlags(&j.ev, cudaEventDisableTiming) != cudaSuccess)
    return svr_fail(FCTN_E_CUDA, "cudaEventCreate");
  rc = fctn_set_data(h, j.Y.data(), j.mask.data(), FCTN_HOST);
  if (rc) return rc;
  std::vector<const void*> fp;
  for (auto& f : j.factors) fp.push_back(f.data());
  rc = fctn_set_factors(h, fp.data(), FCTN_HOST);
  if (rc) return rc;
  j.state = FCTN_JOB_RUNNING;
  j.t_admit = now_s();
  return FCTN_OK;
}

int launch_sweep(fctn_server* S, Job& j) {
  int rc = fctn_internal_sweep_async(j.h, j.pinned);
  if (rc) return rc;
  if (cudaEventRecord(j.ev, fctn_internal_stream(j.h)) != cudaSuccess) return svr_fail(FCTN_E_CUDA, "event record");
  j.inflight = true;
  S->sweeps_launched++;
  return FCTN_OK;
}

}  // namespace

extern "C" {

int fctn_server_create(const fctn_server_config* cfg, fctn_server** out) {
  if (!cfg || !out) return svr_fail(FCTN_E_ARG, "NULL argument");
  if (cfg->max_jobs < 1 || cfg->max_jobs > 1024) return svr_fail(FCTN_E_ARG, "max_jobs outside [1, 1024]");
  fctn_server* S = new fctn_server();
  S->cfg = *cfg;
  if (S->cfg.mem_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete S;
      return svr_fail(FCTN_E_CUDA, "cudaMemGetInfo");
    }
    S->cfg.mem_budget_bytes = fr / 10 * 8;  // 80 % of what is free now
  }
  *out = S;
  return FCTN_OK;
}

int fctn_server_submit(fctn_server* S, const fctn_params* p, const void* Y, const uint8_t* mask,
                       const void* const* factors, double tol, int max_sweeps, uint64_t* job_id) {
  if (!S || !p || !Y || !mask || !factors || !job_id) return svr_fail(FCTN_E_ARG, "NULL argument");
  if (max_sweeps < 1) return svr_fail(FCTN_E_ARG, "max_sweeps < 1");
  size_t fp = 0;
  int rc = fctn_footprint_bytes(p, &fp);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(S->mu);
  if (fp > S->cfg.mem_budget_bytes) return svr_fail(FCTN_E_OOM, "job footprint exceeds the server's memory budget");
  Job j;
  j.id = S->next_id++;
  j.p = *p;
  j.tol = tol;
  j.max_sweeps = max_sweeps;
  j.footprint = fp;
  int64_t P = 1;
  for (int k = 0; k < p->order; ++k) P *= p->dims[k];
  const size_t e = p->precision == FCTN_FP64 ? 8 : 4;
  j.Y.assign((const unsigned char*)Y, (const unsigned char*)Y + P * e);
  j.mask.assign(mask, mask + P);
  for (int k = 0; k < p->order; ++k) {
    int64_t n = p->dims[k];
    for (int t = 0; t < p->order; ++t)
      if (t != k) n *= p->ranks[k < t ? k : t][k < t ? t : k];
    j.factors.emplace_back((const unsigned char*)factors[k], (const unsigned char*)factors[k] + n * e);
  }
  j.t_submit = now_s();
  *job_id = j.id;
  S->queue.push_back(j.id);
  S->jobs.emplace(j.id, std::move(j));
  return FCTN_OK;
}

// One scheduling pass: retire finished sweeps, launch the next sweep of every
// running job whose previous sweep completed, admit waiting jobs.
int fctn_server_step(fctn_server* S, int* running, int* queued) {
  if (!S) return svr_fail(FCTN_E_ARG, "NULL server");
  std::lock_guard<std::mutex> lock(S->mu);
  for (auto& kv : S->jobs) {
    Job& j = kv.second;
    if (j.state != FCTN_JOB_RUNNING) continue;
    if (j.inflight) {
      cudaError_t q = cudaEventQuery(j.ev);
      if (q == cudaErrorNotReady) continue;
      j.inflight = false;
      if (q != cudaSuccess) {
        finish(S, j, FCTN_JOB_FAILED, FCTN_E_CUDA, cudaGetErrorString(q));
        continue;
      }
      int st = 0;
      memcpy(&st, j.pinned + 4, sizeof st);
      j.rel = j.pinned[0];
      j.objective = j.pinned[1];
      j.data = j.pinned[2];
      j.t = (int64_t)j.pinned[5];
      if (st != FCTN_OK) {
        finish(S, j, FCTN_JOB_FAILED, st, "device status");
        continue;
      }
      if (j.pinned[3] != 0.0) {
        finish(S, j, FCTN_JOB_FAILED, FCTN_E_NONFINITE, "non-finite stop-test value");
        continue;
      }
      if ((j.tol > 0 && j.rel <= j.tol) || j.t >= j.max_sweeps) {
        finish(S, j, FCTN_JOB_DONE, FCTN_OK, nullptr);
        continue;
      }
    }
    int rc = launch_sweep(S, j);
    if (rc) finish(S, j, FCTN_JOB_FAILED, rc, "launch");
  }
  // admission: free slot and memory
  while (!S->queue.empty() && S->active < S->cfg.max_jobs) {
    Job& j = S->jobs[S->queue.front()];
    if (S->used + j.footprint > S->cfg.mem_budget_bytes) break;
    S->queue.pop_front();
    int rc = admit(S, j);
    if (rc) {
      char buf[256];
      fctn_last_error(buf, sizeof buf);
      finish(S, j, FCTN_JOB_FAILED, rc, buf);
      continue;
    }
    rc = launch_sweep(S, j);
    if (rc) finish(S, j, FCTN_JOB_FAILED, rc, "launch");
  }
  if (running) *running = S->active;
  if (queued) *queued = (int)S->queue.size();
  return FCTN_OK;
}

int fctn_server_poll(fctn_server* S, uint64_t job_id, fctn_job_info* info) {
  if (!S || !info) return svr_fail(FCTN_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return svr_fail(FCTN_E_ARG, "unknown job id");
  const Job& j = it->second;
  info->state = j.state;
  info->status = j.status;
  info->sweeps = j.t;
  info->rel_change = j.rel;
  info->objective = j.objective;
  info->t_submit = j.t_submit;
  info->t_admit = j.t_admit;
  info->t_done = j.t_done;
  return FCTN_OK;
}

int fctn_server_result(fctn_server* S, uint64_t job_id, void* out_X, int where) {
  if (!S) return svr_fail(FCTN_E_ARG, "NULL server");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return svr_fail(FCTN_E_ARG, "unknown job id");
  Job& j = it->second;
  if (j.state != FCTN_JOB_DONE) return svr_fail(FCTN_E_STATE, "job has not finished");
  int rc = FCTN_OK;
  if (out_X) rc = fctn_get_X(j.h, out_X, where);
  release(S, j);
  S->jobs.erase(it);
  return rc;
}

int fctn_server_finished(fctn_server* S, uint64_t* ids, int cap, int* n) {
  if (!S || !n || (cap > 0 && !ids)) return svr_fail(FCTN_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lock(S->mu);
  int c = (int)S->finished.size() < cap ? (int)S->finished.size() : cap;
  for (int i = 0; i < c; ++i) ids[i] = S->finished[i];
  S->finished.erase(S->finished.begin(), S->finished.begin() + c);
  *n = c;
  return FCTN_OK;
}

int fctn_server_stats(fctn_server* S, int64_t* sweeps_launched, size_t* bytes_in_use) {
  if (!S) return svr_fail(FCTN_E_ARG, "NULL server");
  std::lock_guard<std::mutex> lock(S->mu);
  if (sweeps_launched) *sweeps_launched = S->sweeps_launched;
  if (bytes_in_use) *bytes_in_use = S->used;
  return FCTN_OK;
}

int fctn_server_destroy(fctn_server* S) {
  if (!S) return FCTN_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    for (auto& kv : S->jobs) release(S, kv.second);
    S->jobs.clear();
  }
  delete S;
  return FCTN_OK;
}

}  // extern "C"

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
//
// Grouped sweeps (FCTN_SERVER_GROUP): the ready jobs of one shape class
// (identical fctn_params), at most kGroupMax at a time, sweep as one CUDA
// graph.  The graph is captured on the group's stream: a fork event joins
// every member's stream to the capture, each member's sweep kernels and
// stop-test copy are issued on its own stream (so the members' kernels stay
// independent branches of the graph and overlap), and a join event per
// member brings the branch back.  While the members and their sweep
// signatures (which kernels a sweep launches, with which arguments) are
// unchanged the same executable graph is launched again after each member's
// host bookkeeping; a change of membership or signature captures anew.
#include <algorithm>
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
  bool in_group = false;  // the sweep in flight belongs to a group graph
  uint64_t cls = 0;       // shape class: hash of the job's fctn_params
  int64_t t = 0;
  double rel = 0.0, objective = 0.0, data = 0.0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  std::string err;
};

constexpr int kGroupMax = 16;  // members of one group graph at most

struct Group {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr, fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> sig;      // member ids and sweep keys of the captured graph
  std::vector<uint64_t> members;  // of the launch in flight
  bool inflight = false;
};

uint64_t params_hash(const fctn_params& p) {
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the parameter bytes
  const unsigned char* b = (const unsigned char*)&p;
  for (size_t i = 0; i < sizeof p; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

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
  std::map<uint64_t, Group> groups;
  int64_t group_launches = 0, group_captures = 0;
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
  j.in_group = false;
  S->sweeps_launched++;
  return FCTN_OK;
}

// The sweep of job j completed (q: its event's status): read the stop-test
// values and retire the job, or leave it ready for its next sweep.
void retire_sweep(fctn_server* S, Job& j, cudaError_t q) {
  j.inflight = false;
  j.in_group = false;
  if (q != cudaSuccess) {
    finish(S, j, FCTN_JOB_FAILED, FCTN_E_CUDA, cudaGetErrorString(q));
    return;
  }
  int st = 0;
  memcpy(&st, j.pinned + 4, sizeof st);
  j.rel = j.pinned[0];
  j.objective = j.pinned[1];
  j.data = j.pinned[2];
  j.t = (int64_t)j.pinned[5];
  if (st != FCTN_OK) {
    finish(S, j, FCTN_JOB_FAILED, st, "device status");
    return;
  }
  if (j.pinned[3] != 0.0) {
    finish(S, j, FCTN_JOB_FAILED, FCTN_E_NONFINITE, "non-finite stop-test value");
    return;
  }
  if ((j.tol > 0 && j.rel <= j.tol) || j.t >= j.max_sweeps) {
    finish(S, j, FCTN_JOB_DONE, FCTN_OK, nullptr);
    return;
  }
  fctn_internal_after_sweep(j.h, j.rel);  // mixed precision: FP32 products for the last sweeps
}

// One sweep of every member as one graph launch on the group's stream.
int group_launch(fctn_server* S, uint64_t gkey, const std::vector<Job*>& mem) {
  Group& g = S->groups[gkey];
  if (!g.st) {
    if (cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming) != cudaSuccess)
      return svr_fail(FCTN_E_CUDA, "group stream / events");
  }
  while (g.joins.size() < mem.size()) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return svr_fail(FCTN_E_CUDA, "event");
    g.joins.push_back(e);
  }
  std::vector<uint64_t> sig;
  for (Job* j : mem) {
    sig.push_back(j->id);
    sig.push_back(fctn_internal_sweep_key(j->h));
  }
  int rc = FCTN_OK;
  if (g.exec && g.sig == sig) {
    for (Job* j : mem)
      if ((rc = fctn_internal_sweep_dry(j->h, j->pinned))) return rc;
  } else {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    g.sig.clear();
    if (cudaStreamBeginCapture(g.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return svr_fail(FCTN_E_CUDA, "group capture");
    cudaError_t ce = cudaEventRecord(g.fork, g.st);
    for (size_t i = 0; i < mem.size() && ce == cudaSuccess && rc == FCTN_OK; ++i) {
      cudaStream_t js = fctn_internal_stream(mem[i]->h);
      ce = cudaStreamWaitEvent(js, g.fork, 0);
      if (ce == cudaSuccess) rc = fctn_internal_sweep_eager(mem[i]->h, mem[i]->pinned);
      if (ce == cudaSuccess && rc == FCTN_OK) ce = cudaEventRecord(g.joins[i], js);
      if (ce == cudaSuccess && rc == FCTN_OK) ce = cudaStreamWaitEvent(g.st, g.joins[i], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(g.st, &graph);
    if (rc || ce != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc ? rc : svr_fail(FCTN_E_CUDA, "group capture failed");
    }
    ce = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      g.exec = nullptr;
      return svr_fail(FCTN_E_CUDA, "group graph instantiate");
    }
    g.sig = sig;
    S->group_captures++;
  }
  if (cudaGraphLaunch(g.exec, g.st) != cudaSuccess || cudaEventRecord(g.ev, g.st) != cudaSuccess)
    return svr_fail(FCTN_E_CUDA, "group launch");
  g.members.clear();
  for (Job* j : mem) {
    g.members.push_back(j->id);
    j->inflight = true;
    j->in_group = true;
    S->sweeps_launched++;
  }
  g.inflight = true;
  S->group_launches++;
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
  j.cls = params_hash(*p);
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
  // retire completed group launches and single sweeps
  for (auto& gk : S->groups) {
    Group& g = gk.second;
    if (!g.inflight) continue;
    cudaError_t q = cudaEventQuery(g.ev);
    if (q == cudaErrorNotReady) continue;
    g.inflight = false;
    for (uint64_t id : g.members) {
      auto it = S->jobs.find(id);
      if (it != S->jobs.end() && it->second.state == FCTN_JOB_RUNNING) retire_sweep(S, it->second, q);
    }
  }
  for (auto& kv : S->jobs) {
    Job& j = kv.second;
    if (j.state != FCTN_JOB_RUNNING || !j.inflight || j.in_group) continue;
    cudaError_t q = cudaEventQuery(j.ev);
    if (q == cudaErrorNotReady) continue;
    retire_sweep(S, j, q);
  }
  // next sweeps: ready jobs of one shape class together, the rest alone
  std::map<uint64_t, std::vector<Job*>> ready;
  for (auto& kv : S->jobs) {
    Job& j = kv.second;
    if (j.state == FCTN_JOB_RUNNING && !j.inflight) ready[(S->cfg.flags & FCTN_SERVER_GROUP) ? j.cls : j.id].push_back(&j);
  }
  for (auto& rk : ready) {
    std::vector<Job*>& v = rk.second;
    size_t b = 0;
    if (S->cfg.flags & FCTN_SERVER_GROUP) {
      for (int chunk = 0; v.size() - b >= 2; ++chunk) {
        const size_t n = std::min(v.size() - b, (size_t)kGroupMax);
        std::vector<Job*> mem(v.begin() + b, v.begin() + b + n);
        b += n;
        int rc = group_launch(S, rk.first * 131 + (uint64_t)chunk, mem);
        if (rc)
          for (Job* j : mem)
            if (!j->inflight) finish(S, *j, FCTN_JOB_FAILED, rc, "group launch");
      }
    }
    for (; b < v.size(); ++b) {
      int rc = launch_sweep(S, *v[b]);
      if (rc) finish(S, *v[b], FCTN_JOB_FAILED, rc, "launch");
    }
  }
  // admission: free slot and memory (the first sweep runs alone; the job joins
  // its class's group from the next pass)
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

int fctn_server_group_stats(fctn_server* S, int64_t* group_launches, int64_t* group_captures) {
  if (!S) return svr_fail(FCTN_E_ARG, "NULL server");
  std::lock_guard<std::mutex> lock(S->mu);
  if (group_launches) *group_launches = S->group_launches;
  if (group_captures) *group_captures = S->group_captures;
  return FCTN_OK;
}

int fctn_server_destroy(fctn_server* S) {
  if (!S) return FCTN_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    for (auto& gk : S->groups) {
      Group& g = gk.second;
      if (g.st) cudaStreamSynchronize(g.st);
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (cudaEvent_t e : g.joins) cudaEventDestroy(e);
      if (g.ev) cudaEventDestroy(g.ev);
      if (g.fork) cudaEventDestroy(g.fork);
      if (g.st) cudaStreamDestroy(g.st);
    }
    S->groups.clear();
    for (auto& kv : S->jobs) release(S, kv.second);
    S->jobs.clear();
  }
  delete S;
  return FCTN_OK;
}

}  // extern "C"

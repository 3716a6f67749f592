// Request server with continuous batching (declared in include/seg.h).
//
// Requests wait in a FIFO queue.  A tick
//   1. admits queued requests in order while their device footprint fits the
//      memory budget (and the resident count limit),
//   2. rebuilds the batch of every class whose membership changed (states of
//      one class -- precision, lanes per row, row width, device -- share
//      batched launches; each class has its own stream so classes overlap),
//   3. advances every batch by steps_per_tick steps (all batches enqueued
//      before any is waited for),
//   4. retires the requests that met their stop rule or step limit: the
//      result is copied to host memory and the state's device memory freed.
// Each state keeps its own launch geometry and control block, so a request's
// result does not depend on what else is resident.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "seg_internal.h"

namespace {

struct Request {
  int64_t id = 0;
  const seg_problem* p = nullptr;
  int32_t m = 0;
  double eps = 0;
  seg_init init = SEG_INIT_UNIFORM;
  uint64_t seed = 0;
  seg_params prm{};
  uint64_t bytes = 0;
  int64_t n_vert = 0;
  seg_request_info info{};
  seg_state* st = nullptr;
  long long key = 0;
  std::vector<double> result;
};

struct Group {
  cudaStream_t stream = nullptr;
  std::vector<int64_t> members;    // request ids
  std::vector<seg_batch*> batches;  // up to 32 members each
  bool dirty = false;
};

seg_status fail(seg_status code, const std::string& msg) {
  segimpl::set_last_error(msg.c_str());
  return code;
}

}  // namespace

struct seg_server {
  seg_server_params prm{};
  std::chrono::steady_clock::time_point t0;
  std::vector<std::unique_ptr<Request>> reqs;  // index = id
  std::deque<int64_t> queue;
  uint64_t used = 0;
  int resident = 0;
  std::map<long long, Group> groups;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

void release_batches(Group& g) {
  for (seg_batch* b : g.batches) seg_batch_destroy(b);
  g.batches.clear();
}

// Copy the result of a finished request, free its state.
void retire(seg_server* srv, Request& r, Group& g, int phase, seg_status status) {
  r.result.assign((size_t)r.n_vert * r.m, 0.0);
  seg_status st = seg_get_u(r.st, r.result.data(), 0);
  seg_stats stats{};
  if (seg_get_stats(r.st, &stats) == SEG_OK) {
    r.info.steps = stats.steps;
    r.info.converged = stats.converged;
    r.info.total_energy = stats.last_check_total;
  }
  r.info.phase = (st == SEG_OK && phase == 2) ? 2 : 3;
  r.info.status = status != SEG_OK ? status : st;
  r.info.t_done = srv->now();
  seg_state_destroy(r.st);
  r.st = nullptr;
  srv->used -= r.bytes;
  srv->resident -= 1;
  g.members.erase(std::find(g.members.begin(), g.members.end(), r.id));
  g.dirty = true;
}

}  // namespace

extern "C" {

seg_status seg_server_create(const seg_server_params* opt, seg_server** out) {
  if (!out) return fail(SEG_ERR_ARG, "out is NULL");
  *out = nullptr;
  seg_server* srv = new (std::nothrow) seg_server;
  if (!srv) return fail(SEG_ERR_NO_MEMORY, "host allocation failed");
  if (opt) srv->prm = *opt;
  if (srv->prm.steps_per_tick <= 0) srv->prm.steps_per_tick = 16;
  if (srv->prm.max_resident < 0) srv->prm.max_resident = 0;
  if (srv->prm.hbm_budget_bytes == 0) {
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
      delete srv;
      return fail(SEG_ERR_CUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
    }
    srv->prm.hbm_budget_bytes = (uint64_t)(0.8 * (double)free_b);
  }
  srv->t0 = std::chrono::steady_clock::now();
  *out = srv;
  return SEG_OK;
}

double seg_server_clock(const seg_server* srv) { return srv ? srv->now() : 0.0; }

seg_status seg_server_submit(seg_server* srv, const seg_problem* p, int32_t m, double eps, seg_init init,
                             uint64_t seed, const seg_params* opt, int64_t* id) {
  if (!srv || !p || !id) return fail(SEG_ERR_ARG, "server, problem or id is NULL");
  seg_params prm{};
  if (opt) prm = *opt;
  if (prm.energy_tol < 0 && !(prm.energy_rtol > 0) && prm.max_steps <= 0)
    return fail(SEG_ERR_ARG, "a request needs a stop rule (energy_tol >= 0 or energy_rtol > 0) or max_steps");
  if (prm.check_every < 0 && prm.max_steps <= 0)
    return fail(SEG_ERR_ARG, "a request without energy checks needs max_steps");
  uint64_t bytes = 0;
  seg_status st = seg_state_bytes(p, m, &bytes);
  if (st != SEG_OK) return st;
  int64_t n = 0;
  st = seg_problem_info(p, &n, nullptr, nullptr, nullptr);
  if (st != SEG_OK) return st;
  auto r = std::make_unique<Request>();
  r->id = (int64_t)srv->reqs.size();
  r->p = p;
  r->m = m;
  r->eps = eps;
  r->init = init;
  r->seed = seed;
  r->prm = prm;
  r->bytes = bytes;
  r->n_vert = n;
  r->info.phase = 0;
  r->info.m = m;
  r->info.n_vert = n;
  r->info.t_submit = srv->now();
  *id = r->id;
  srv->queue.push_back(r->id);
  srv->reqs.push_back(std::move(r));
  return SEG_OK;
}

seg_status seg_server_tick(seg_server* srv, int32_t* running, int32_t* queued) {
  if (!srv) return fail(SEG_ERR_ARG, "server is NULL");
  // 1. admission, in arrival order
  while (!srv->queue.empty()) {
    Request& r = *srv->reqs[srv->queue.front()];
    if (srv->prm.max_resident > 0 && srv->resident >= srv->prm.max_resident) break;
    if (srv->used + r.bytes > srv->prm.hbm_budget_bytes) {
      if (srv->resident == 0) {  // can never fit
        srv->queue.pop_front();
        r.info.phase = 3;
        r.info.status = SEG_ERR_NO_MEMORY;
        r.info.t_done = srv->now();
        continue;
      }
      break;
    }
    srv->queue.pop_front();
    seg_state* st = nullptr;
    // the state gets its own stream (used for its result read-back); its
    // batched steps run on the stream of its class
    seg_status s = seg_state_create(r.p, r.m, r.eps, r.init, r.seed, &r.prm, nullptr, &st);
    if (s != SEG_OK) {
      r.info.phase = 3;
      r.info.status = s;
      r.info.t_done = srv->now();
      continue;
    }
    r.st = st;
    r.key = segimpl::state_class_key(st);
    Group& g = srv->groups[r.key];
    if (!g.stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return fail(SEG_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    g.members.push_back(r.id);
    g.dirty = true;
    srv->used += r.bytes;
    srv->resident += 1;
    r.info.phase = 1;
    r.info.t_admit = srv->now();
  }
  // 2. batches of the classes whose membership changed
  for (auto& kv : srv->groups) {
    Group& g = kv.second;
    if (!g.dirty) continue;
    release_batches(g);
    for (size_t i = 0; i < g.members.size(); i += (size_t)segimpl::kMaxBatch) {
      std::vector<seg_state*> part;
      for (size_t j = i; j < std::min(g.members.size(), i + (size_t)segimpl::kMaxBatch); ++j)
        part.push_back(srv->reqs[g.members[j]]->st);
      seg_batch* b = nullptr;
      seg_status s = seg_batch_create(part.data(), (int32_t)part.size(), g.stream, &b);
      if (s != SEG_OK) return s;
      g.batches.push_back(b);
    }
    g.dirty = false;
  }
  // 3. one quantum for every batch, all enqueued before any wait
  for (auto& kv : srv->groups)
    for (seg_batch* b : kv.second.batches) {
      seg_status s = seg_batch_step_async(b, srv->prm.steps_per_tick);
      if (s != SEG_OK) return s;
    }
  // 4. retire finished requests
  for (auto& kv : srv->groups) {
    Group& g = kv.second;
    for (seg_batch* b : g.batches) seg_batch_sync(b);  // per-member status is read below
    std::vector<int64_t> ids = g.members;
    for (int64_t id : ids) {
      Request& r = *srv->reqs[id];
      seg_stats stats{};
      seg_status s = seg_get_stats(r.st, &stats);
      r.info.steps = stats.steps;
      r.info.total_energy = stats.last_check_total;
      if (s != SEG_OK) {
        retire(srv, r, g, 3, s);
      } else if (stats.status_bits & 6) {
        retire(srv, r, g, 3, (stats.status_bits & 4) ? SEG_ERR_TIMEOUT : SEG_ERR_NONFINITE);
      } else if (stats.converged || (r.prm.max_steps > 0 && stats.steps >= r.prm.max_steps)) {
        retire(srv, r, g, 2, SEG_OK);
      }
    }
  }
  if (running) *running = srv->resident;
  if (queued) *queued = (int32_t)srv->queue.size();
  return SEG_OK;
}

seg_status seg_server_info(seg_server* srv, int64_t id, seg_request_info* out) {
  if (!srv || !out) return fail(SEG_ERR_ARG, "server or out is NULL");
  if (id < 0 || id >= (int64_t)srv->reqs.size()) return fail(SEG_ERR_ARG, "unknown request id");
  *out = srv->reqs[id]->info;
  return SEG_OK;
}

seg_status seg_server_result(seg_server* srv, int64_t id, double* u) {
  if (!srv || !u) return fail(SEG_ERR_ARG, "server or u is NULL");
  if (id < 0 || id >= (int64_t)srv->reqs.size()) return fail(SEG_ERR_ARG, "unknown request id");
  const Request& r = *srv->reqs[id];
  if (r.info.phase != 2) return fail(SEG_ERR_ARG, "request is not done");
  std::copy(r.result.begin(), r.result.end(), u);
  return SEG_OK;
}

void seg_server_destroy(seg_server* srv) {
  if (!srv) return;
  for (auto& kv : srv->groups) release_batches(kv.second);
  for (auto& r : srv->reqs)
    if (r->st) seg_state_destroy(r->st);
  for (auto& kv : srv->groups)
    if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
  delete srv;
}

}  // extern "C"

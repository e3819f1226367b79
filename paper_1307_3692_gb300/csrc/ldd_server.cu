// Request server: continuous batching of decomposition requests (C ABI in
// include/ldd.h, ldd_server_*).
//
// Requests (graph, beta, shifts, output buffers) arrive on any thread and wait
// in one FIFO queue.  Each of the server's slots is a worker thread that owns
// a union workspace (a disjoint-union graph object with fixed capacities,
// ldd_graph.cuh) and a CUDA stream.  A free worker takes, in arrival order,
// every waiting request that still fits its workspace -- the admission test is
// the requests' device footprint: vertices, arcs, cut-list entries and small
// components against the capacities the HBM budget bought -- and runs them as
// one decomposition of their disjoint union (Algorithm 2 never crosses from
// one member to another, so every member's result is exactly its result
// alone):
//   1. union tables from the members' resident tables (one kernel launch) and
//      the members' shifts copied in (host -> device);
//   2. spread, rank, round loop, finalize and the members' cut counts on the
//      worker's stream;
//   3. results copied out (device -> host), requests completed.
// The workers' streams run side by side on the device except for the round
// loop, a cooperative kernel that occupies every SM: the workspaces share a
// gate (BfsGate, ldd_graph.cuh), so each round loop waits on the event of the
// one enqueued before it.  One batch's rank, finalize, cut count and copies
// thus overlap another's, and requests that arrive while a batch is on the
// GPU are admitted to the next batch as soon as a slot and memory are free.
// A worker holds no lock while the device runs a union batch; a batch of one
// holds the gate for its whole call (run_alone).
//
// A batch that fails on a request's input (a bad shift) is rerun request by
// request, so only that request fails.
//
// one_at_a_time = 1 turns batching off: a single worker runs each request as
// one ldd_decompose_batch call (k = 1, the plain path) on its own graph, in
// arrival order -- the comparison the batched server is measured against.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ldd_graph.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  ldd_graph* g = nullptr;
  double beta = 0.0;
  const double* shifts = nullptr;
  int32_t* out_center = nullptr;
  int32_t* out_dist = nullptr;
  int64_t* out_cut = nullptr;
  UnionCaps need;          // the request's share of a workspace
  int status = LDD_OK;
  char msg[256] = "";      // ldd_last_error() text of a failed request
  bool done = false;
  double submit_us = 0.0, start_us = 0.0, end_us = 0.0;
  int64_t batch_id = -1;
  int32_t batch_size = 0;
  double fill_us = 0.0, run_us = 0.0;  // the batch's phases
};

bool fits(const UnionCaps& a, const UnionCaps& b, const UnionCaps& cap) {
  return a.N + b.N <= cap.N && a.E + b.E <= cap.E && a.M + b.M <= cap.M &&
         a.G + b.G <= cap.G && a.C + b.C <= cap.C && a.T + b.T <= cap.T && a.total + b.total <= cap.total &&
         a.k + b.k <= cap.k;
}

void add_to(UnionCaps& a, const UnionCaps& b) {
  a.N += b.N;
  a.E += b.E;
  a.M += b.M;
  a.G += b.G;
  a.C += b.C;
  a.T += b.T;
  a.total += b.total;
  a.k += b.k;
}

// Workspace capacities that fit a per-slot budget: arcs up to half of it (at
// most 2^31 - 1), vertices with what is left.
UnionCaps caps_for(u64 budget, int max_batch, u64 max_vertices, u64 max_arcs) {
  UnionCaps c;
  c.k = (u32)max_batch;
  c.E = max_arcs ? max_arcs : std::min<u64>((1ull << 31) - 64, budget / 2 / 12);
  c.M = c.E / 2 + 1;
  u64 N = max_vertices ? max_vertices : (1u << 30) - 64;
  N = N / 32 * 32;
  for (;;) {
    c.N = N;
    c.G = std::min<u64>(N, c.M);
    c.C = N / 2;
    c.T = N;
    c.total = N;
    if (max_vertices || N <= 32 || union_bytes(c) <= budget) break;
    N = std::max<u64>(32, N / 10 * 9 / 32 * 32);
  }
  return c;
}

}  // namespace

struct ldd_server {
  ldd_server_config cfg{};
  int device = 0;
  UnionCaps cap;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::vector<std::unique_ptr<Request>> reqs;  // by ticket; released by ldd_server_wait
  bool stop = false;
  int64_t next_batch = 0;
  BfsGate gate;  // orders the workspaces' round loops (and batches of one)
  std::vector<ldd_graph*> ws;
  std::vector<cudaStream_t> streams;
  std::vector<u64*> h_cut;
  std::vector<std::thread> workers;
  Clock::time_point t0 = Clock::now();

  double now_us() const {
    return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
  }
};

namespace {

void finish(ldd_server* S, const std::vector<Request*>& batch) {
  const double t = S->now_us();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (Request* r : batch) {
      r->end_us = t;
      r->done = true;
    }
  }
  S->cv_done.notify_all();
}

// Steps 1-3 for the requests of one batch on workspace slot; returns the
// batch's status (every request's status on success).
int run_batch(ldd_server* S, int slot, const std::vector<Request*>& batch) {
  ldd_graph* u = S->ws[(size_t)slot];
  cudaStream_t s = S->streams[(size_t)slot];
  ldd_graph::Union& U = *u->uni;
  const int k = (int)batch.size();
  std::vector<ldd_graph*> members((size_t)k);
  bool want_cut = false;
  for (int i = 0; i < k; ++i) {
    members[(size_t)i] = batch[(size_t)i]->g;
    want_cut |= batch[(size_t)i]->out_cut != nullptr;
  }
  const double t0 = S->now_us();
  int rc = union_fill(u, k, members.data(), s, false);
  if (rc != LDD_OK) return rc;
  for (int i = 0; i < k; ++i) {
    const Request* r = batch[(size_t)i];
    CUDA_TRY(cudaMemcpyAsync(U.d_shift_in + U.h_ooff[(size_t)i], r->shifts,
                             (size_t)r->g->n * 8, cudaMemcpyHostToDevice, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  const double t1 = S->now_us();
  int launches = 0, cut_launches = 0;
  const double t2 = S->now_us();
  rc = union_run(u, U.d_shift_in, U.d_out_c, U.d_out_d, want_cut, &launches, &cut_launches);
  if (rc != LDD_OK) return rc;
  if (want_cut)
    CUDA_TRY(cudaMemcpyAsync(S->h_cut[(size_t)slot], U.d_cut, (size_t)k * 8,
                             cudaMemcpyDeviceToHost, s));
  for (int i = 0; i < k; ++i) {
    const Request* r = batch[(size_t)i];
    const size_t n = (size_t)r->g->n, o = U.h_ooff[(size_t)i];
    CUDA_TRY(cudaMemcpyAsync(r->out_center, U.d_out_c + o, n * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(r->out_dist, U.d_out_d + o, n * 4, cudaMemcpyDeviceToHost, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  const double t3 = S->now_us();
  for (Request* r : batch) {
    r->fill_us = t1 - t0;
    r->run_us = t3 - t2;
  }
  for (int i = 0; i < k; ++i)
    if (batch[(size_t)i]->out_cut) *batch[(size_t)i]->out_cut = (int64_t)S->h_cut[(size_t)slot][i];
  return LDD_OK;
}

// A batch of one request skips the union: the request runs on its own graph
// object, as ldd_decompose_batch(g, 1, ...) does, holding the gate for the
// whole call (two workers may hold requests on the same graph object) after
// the round loop enqueued last.  At low arrival rates most batches are of one,
// and building a union for them only adds latency.
int run_alone(ldd_server* S, Request* r) {
  std::lock_guard<std::mutex> lk(S->gate.mu);
  if (S->gate.last) CUDA_TRY(cudaStreamWaitEvent(r->g->stream, S->gate.last, 0));
  const double t0 = S->now_us();
  const double* sh = r->shifts;
  int32_t* oc = r->out_center;
  int32_t* od = r->out_dist;
  const int rc = ldd_decompose_batch(r->g, 1, &r->beta, &sh, &oc, &od, r->out_cut);
  r->fill_us = 0.0;
  r->run_us = S->now_us() - t0;
  return rc;
}

void worker_batched(ldd_server* S, int slot) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Request*> batch;
    int64_t bid;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      if (S->queue.empty()) return;  // stop, and nothing left
      UnionCaps sum;
      while (!S->queue.empty() && fits(sum, S->queue.front()->need, S->cap)) {
        add_to(sum, S->queue.front()->need);
        batch.push_back(S->queue.front());
        S->queue.pop_front();
      }
      bid = S->next_batch++;
    }
    if (batch.empty()) continue;  // cannot happen: submit rejects requests that never fit
    const double t = S->now_us();
    for (Request* r : batch) {
      r->start_us = t;
      r->batch_id = bid;
      r->batch_size = (int32_t)batch.size();
    }
    int rc = batch.size() == 1 ? run_alone(S, batch[0]) : run_batch(S, slot, batch);
    if (rc != LDD_OK && batch.size() > 1) {
      // rerun one by one so that only the request at fault fails
      cudaStreamSynchronize(S->streams[(size_t)slot]);
      cudaGetLastError();
      for (Request* r : batch) {
        r->batch_size = 1;
        r->status = run_alone(S, r);
        if (r->status != LDD_OK) snprintf(r->msg, sizeof(r->msg), "%s", ldd_last_error());
      }
    } else {
      for (Request* r : batch) {
        r->status = rc;
        if (rc != LDD_OK) snprintf(r->msg, sizeof(r->msg), "%s", ldd_last_error());
      }
    }
    finish(S, batch);
  }
}

void worker_one_at_a_time(ldd_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    Request* r;
    int64_t bid;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      if (S->queue.empty()) return;
      r = S->queue.front();
      S->queue.pop_front();
      bid = S->next_batch++;
    }
    r->start_us = S->now_us();
    r->batch_id = bid;
    r->batch_size = 1;
    const double* sh = r->shifts;
    int32_t* oc = r->out_center;
    int32_t* od = r->out_dist;
    r->status = ldd_decompose_batch(r->g, 1, &r->beta, &sh, &oc, &od, r->out_cut);
    if (r->status != LDD_OK) snprintf(r->msg, sizeof(r->msg), "%s", ldd_last_error());
    finish(S, std::vector<Request*>{r});
  }
}

void free_server(ldd_server* S) {
  for (ldd_graph* u : S->ws)
    if (u) {
      free_graph_memory(u);
      delete u;
    }
  for (cudaStream_t s : S->streams)
    if (s) cudaStreamDestroy(s);
  for (u64* h : S->h_cut)
    if (h) cudaFreeHost(h);
  delete S;
}

}  // namespace

extern "C" {

int ldd_server_create(const ldd_server_config* cfg, ldd_server** out) {
  if (!out) return fail(LDD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(LDD_ERR_ARG, "cfg is NULL");
  if (cfg->slots < 1 || cfg->max_batch < 1)
    return fail(LDD_ERR_ARG, "slots (%d) and max_batch (%d) must be >= 1", cfg->slots,
                cfg->max_batch);
  if (cfg->hbm_budget_bytes <= 0 || cfg->max_vertices < 0 || cfg->max_arcs < 0)
    return fail(LDD_ERR_ARG, "the HBM budget must be > 0 and the caps >= 0");
  if (cfg->max_vertices >= (1ll << 30) || cfg->max_arcs >= (1ll << 31))
    return fail(LDD_ERR_RANGE, "max_vertices must be < 2^30 and max_arcs < 2^31");
  ldd_server* S = new (std::nothrow) ldd_server();
  if (!S) return fail(LDD_ERR_OOM, "host allocation failed");
  S->cfg = *cfg;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return fail(LDD_ERR_CUDA, "no usable CUDA device");
  }
  if (!cfg->one_at_a_time) {
    const int slots = cfg->slots;
    S->cap = caps_for((u64)cfg->hbm_budget_bytes / (u64)slots, cfg->max_batch,
                      (u64)cfg->max_vertices, (u64)cfg->max_arcs);
    if ((u64)slots * union_bytes(S->cap) > (u64)cfg->hbm_budget_bytes) {
      delete S;
      return fail(LDD_ERR_RANGE, "the caps need %llu bytes per slot, over the HBM budget",
                  (unsigned long long)union_bytes(S->cap));
    }
    for (int i = 0; i < slots; ++i) {
      ldd_graph* u = nullptr;
      cudaStream_t st = nullptr;
      u64* h = nullptr;
      int rc = union_alloc(&u, S->device, S->cap);
      S->ws.push_back(u);
      if (rc == LDD_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        rc = fail(LDD_ERR_CUDA, "cudaStreamCreate failed");
      S->streams.push_back(st);
      if (rc == LDD_OK && cudaMallocHost(&h, (size_t)cfg->max_batch * 8) != cudaSuccess)
        rc = fail(LDD_ERR_OOM, "pinned host allocation failed");
      S->h_cut.push_back(h);
      if (rc != LDD_OK) {
        cudaGetLastError();
        free_server(S);
        return rc;
      }
      u->stream = st;
      u->gate = &S->gate;
      if (cudaEventCreateWithFlags(&u->ev_gate, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_server(S);
        return fail(LDD_ERR_CUDA, "cudaEventCreate failed");
      }
    }
    for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker_batched, S, i);
  } else {
    S->workers.emplace_back(worker_one_at_a_time, S);
  }
  *out = S;
  return LDD_OK;
}

int ldd_server_footprint(const ldd_server* S, const ldd_graph* g, int64_t* out_bytes) {
  if (!S || !g || !out_bytes) return fail(LDD_ERR_ARG, "NULL argument");
  if (g->uni) return fail(LDD_ERR_ARG, "a union cannot be a request's graph");
  ldd_graph* m = const_cast<ldd_graph*>(g);
  *out_bytes = (int64_t)union_bytes(union_needs(1, &m));
  return LDD_OK;
}

int ldd_server_submit(ldd_server* S, ldd_graph* g, double beta, const double* shifts,
                      int32_t* out_center, int32_t* out_dist, int64_t* out_cut,
                      int64_t* out_ticket) {
  if (!S || !g || !out_ticket) return fail(LDD_ERR_ARG, "NULL server, graph or ticket");
  *out_ticket = -1;
  if (g->uni) return fail(LDD_ERR_ARG, "a union cannot be a request's graph");
  if (g->device != S->device) return fail(LDD_ERR_ARG, "graph and server on different devices");
  if (!(beta > 0.0) || isinf(beta)) return fail(LDD_ERR_ARG, "beta must be finite and > 0");
  if (g->n > 0 && (!shifts || !out_center || !out_dist))
    return fail(LDD_ERR_ARG, "NULL shifts or output");
  if (g->n > 0 && (is_device_ptr(shifts) || is_device_ptr(out_center) ||
                   is_device_ptr(out_dist) || (out_cut && is_device_ptr(out_cut))))
    return fail(LDD_ERR_ARG, "server requests take host buffers");
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return fail(LDD_ERR_OOM, "host allocation failed");
  r->g = g;
  r->beta = beta;
  r->shifts = shifts;
  r->out_center = out_center;
  r->out_dist = out_dist;
  r->out_cut = out_cut;
  r->need = union_needs(1, &g);
  if (!S->cfg.one_at_a_time && !fits(UnionCaps(), r->need, S->cap))
    return fail(LDD_ERR_RANGE, "the request's graph exceeds a slot's capacity");
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return fail(LDD_ERR_ARG, "the server is shutting down");
  r->submit_us = S->now_us();
  const int64_t ticket = (int64_t)S->reqs.size();
  Request* raw = r.get();
  S->reqs.push_back(std::move(r));
  *out_ticket = ticket;
  if (g->n == 0) {  // nothing to compute
    raw->start_us = raw->end_us = raw->submit_us;
    raw->batch_size = 1;
    if (out_cut) *out_cut = 0;
    raw->done = true;
    return LDD_OK;
  }
  S->queue.push_back(raw);
  S->cv_work.notify_one();
  return LDD_OK;
}

int ldd_server_wait(ldd_server* S, int64_t ticket, ldd_request_info* info) {
  if (!S) return fail(LDD_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  if (ticket < 0 || ticket >= (int64_t)S->reqs.size() || !S->reqs[(size_t)ticket])
    return fail(LDD_ERR_ARG, "unknown or already collected ticket %lld", (long long)ticket);
  Request* r = S->reqs[(size_t)ticket].get();
  S->cv_done.wait(lk, [&] { return r->done; });
  const int status = r->status;
  if (info) {
    info->status = status;
    info->batch_size = r->batch_size;
    info->batch_id = r->batch_id;
    info->submit_us = r->submit_us;
    info->start_us = r->start_us;
    info->end_us = r->end_us;
    info->batch_fill_us = r->fill_us;
    info->batch_run_us = r->run_us;
  }
  if (status != LDD_OK) fail(status, "%s", r->msg);
  S->reqs[(size_t)ticket].reset();
  return status;
}

int ldd_server_destroy(ldd_server* S) {
  if (!S) return LDD_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  DeviceGuard dg(S->device);
  free_server(S);
  return LDD_OK;
}

}  // extern "C"

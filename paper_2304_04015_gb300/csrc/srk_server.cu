// Query server: resident graphs, memory-based admission, worker streams.
//
// A request names a resident graph, a source, c, eps and a seed.  On submit
// the server evaluates the request's sample-count table (step a1) to know
// the device memory the query will hold (its scratch plus its score vector);
// the request is admitted only if the memory held by admitted, unfinished
// requests stays within the server's budget, otherwise it is shed at once.
// Admitted requests wait in a FIFO queue; each worker thread owns a CUDA
// stream, takes the next request, runs srk_single_source on its stream,
// copies the scores to the caller's host buffer (if one was given) and
// records the latency from submission to the result being on the host.
//
// With a latency target, admission also needs the request's estimated finish
// time to fit it: the server estimates a request's work as (targets with
// in-neighbours) x N_tot x kStepsPerPair walk steps (none when the source has
// no in-neighbours: its walks cannot leave it), keeps the estimated work of
// admitted, unfinished requests, and divides by the rate at which completed
// requests got through their estimated work (an exponential average).  The
// queue is then served shortest estimated work first, so short queries are
// not held behind long ones; without a target it is first in, first out.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "srk_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int32_t graph, s;
  double c, eps;
  uint64_t seed, tag;
  double *host_scores;
  size_t bytes;  // reserved device memory
  double work;   // estimated walk steps
  uint64_t order;
  Clock::time_point t_submit;
};

// walk steps per (target, pair) the work estimate assumes before any request
// has completed; completed requests refine the rate, not this factor
constexpr double kStepsPerPair = 0.8;

}  // namespace

struct srk_server {
  std::vector<const srk_graph *> graphs;
  std::vector<std::vector<uint8_t>> has_in;  // per graph: node has in-neighbours
  size_t budget = 0;
  double target_ms = 0.0;     // 0: memory-only admission, FIFO
  double rate = 5.0e10;       // estimated work units (walk steps) per second,
                              // refined on completions; starts conservative
  double queued_work = 0.0;   // estimated steps of admitted, unfinished requests
  uint64_t next_order = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_idle;
  std::deque<Request> queue;
  std::vector<std::thread> workers;
  bool stop = false;
  size_t reserved = 0, reserved_peak = 0;
  int running = 0;
  uint64_t submitted = 0, admitted = 0, shed = 0, completed = 0, failed = 0;
  uint64_t target_steps = 0;
  std::vector<double> latency_ms;
  bool have_first = false;
  Clock::time_point t_first, t_last;
};

namespace srk {

static void worker_main(srk_server *srv, int device) {
  cudaSetDevice(device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Request r;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv_work.wait(lk, [&] { return srv->stop || !srv->queue.empty(); });
      if (srv->queue.empty()) break;  // stop requested and nothing left
      auto pick = srv->queue.begin();
      if (srv->target_ms > 0.0)  // shortest estimated work first
        for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it)
          if (it->work < pick->work || (it->work == pick->work && it->order < pick->order))
            pick = it;
      r = *pick;
      srv->queue.erase(pick);
      ++srv->running;
    }
    const srk_graph *g = srv->graphs[(size_t)r.graph];
    double *d_scores = nullptr;
    srk_stats stats;
    srk_opts opt;
    memset(&opt, 0, sizeof opt);
    opt.L_override = -1;
    opt.stats = &stats;
    int rc = SRK_OK;
    const Clock::time_point t_start = Clock::now();
    cudaError_t e = cudaMallocFromPoolAsync((void **)&d_scores, sizeof(double) * (size_t)g->n,
                                            pool(g->device), st);
    if (e != cudaSuccess) rc = SRK_ENOMEM;
    if (rc == SRK_OK)
      rc = srk_single_source(g, r.s, r.c, r.eps, r.seed, &opt, d_scores, nullptr, nullptr, st);
    if (rc == SRK_OK && r.host_scores)
      e = cudaMemcpyAsync(r.host_scores, d_scores, sizeof(double) * (size_t)g->n,
                          cudaMemcpyDeviceToHost, st);
    if (d_scores) cudaFreeAsync(d_scores, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || e != cudaSuccess) rc = SRK_ECUDA;
    const Clock::time_point t_done = Clock::now();
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      --srv->running;
      srv->reserved -= r.bytes;
      srv->queued_work -= r.work;
      if (srv->queued_work < 0.0) srv->queued_work = 0.0;
      if (rc == SRK_OK) {
        ++srv->completed;
        srv->target_steps += stats.target_steps;
        const double secs = std::chrono::duration<double>(t_done - t_start).count();
        if (r.work > 1.0e6 && secs > 0.0)  // estimated work per second of service
          srv->rate = 0.8 * srv->rate + 0.2 * (r.work / secs);
        srv->latency_ms.push_back(
            std::chrono::duration<double, std::milli>(t_done - r.t_submit).count());
        srv->t_last = t_done;
      } else {
        ++srv->failed;
      }
      if (srv->queue.empty() && srv->running == 0) srv->cv_idle.notify_all();
    }
  }
  cudaStreamDestroy(st);
}

static double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace srk

using namespace srk;

extern "C" int srk_server_create(const srk_graph *const *graphs, int32_t n_graphs,
                                 uint64_t mem_budget, int32_t n_workers,
                                 double latency_target_ms, srk_server **out) {
  clear_error();
  if (!out) return fail(SRK_EINVAL, "out is null");
  *out = nullptr;
  if (!graphs || n_graphs < 1) return fail(SRK_EINVAL, "no graphs");
  if (n_workers < 1 || n_workers > 64)
    return fail(SRK_EINVAL, "n_workers = %d outside [1, 64]", n_workers);
  if (mem_budget == 0) return fail(SRK_EINVAL, "mem_budget must be positive");
  for (int32_t i = 0; i < n_graphs; ++i)
    if (!graphs[i]) return fail(SRK_EINVAL, "graph %d is null", i);
  if (!(latency_target_ms >= 0.0)) return fail(SRK_EINVAL, "latency target must be >= 0");
  srk_server *srv = new srk_server;
  srv->graphs.assign(graphs, graphs + n_graphs);
  srv->budget = (size_t)mem_budget;
  srv->target_ms = latency_target_ms;
  for (int32_t i = 0; i < n_graphs; ++i) {  // which nodes have in-neighbours
    const srk_graph *g = graphs[i];
    std::vector<int32_t> rp((size_t)g->n + 1);
    DeviceGuard guard(g->device);
    const cudaError_t e = cudaMemcpy(rp.data(), g->row_ptr, sizeof(int32_t) * rp.size(),
                                     cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      delete srv;
      return cuda_fail(e, "srk_server_create: reading in-degrees");
    }
    std::vector<uint8_t> has((size_t)g->n);
    for (size_t v = 0; v < has.size(); ++v) has[v] = rp[v + 1] > rp[v];
    srv->has_in.push_back(std::move(has));
  }
  const int device = graphs[0]->device;
  for (int32_t w = 0; w < n_workers; ++w) srv->workers.emplace_back(worker_main, srv, device);
  *out = srv;
  return SRK_OK;
}

extern "C" int srk_server_submit(srk_server *srv, int32_t graph, int32_t s, double c,
                                 double eps, uint64_t seed, double *host_scores,
                                 uint64_t tag, int32_t *admitted) {
  clear_error();
  if (admitted) *admitted = 0;
  if (!srv) return fail(SRK_EINVAL, "null server");
  if (graph < 0 || graph >= (int32_t)srv->graphs.size())
    return fail(SRK_EINVAL, "graph index %d out of range", graph);
  const srk_graph *g = srv->graphs[(size_t)graph];
  QueryTab t;
  int rc = build_table(g->n, s, c, eps, seed, nullptr, &t);
  if (rc) return rc;
  Workspace w;
  const size_t bytes = plan(t, &w, nullptr) + sizeof(double) * (size_t)g->n;
  const double work = srv->has_in[(size_t)graph][(size_t)s]
                          ? (double)g->n_act * (double)t.N_tot * kStepsPerPair
                          : 0.0;
  Request r;
  r.graph = graph;
  r.s = s;
  r.c = c;
  r.eps = eps;
  r.seed = seed;
  r.tag = tag;
  r.host_scores = host_scores;
  r.bytes = bytes;
  r.work = work;
  r.t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(srv->mu);
  ++srv->submitted;
  if (!srv->have_first) {
    srv->have_first = true;
    srv->t_first = r.t_submit;
  }
  const bool mem_ok = srv->reserved + bytes <= srv->budget;
  const bool time_ok = srv->target_ms <= 0.0 ||
                       (srv->queued_work + work) / srv->rate * 1e3 <= srv->target_ms;
  if (!mem_ok || !time_ok) {
    ++srv->shed;
    return SRK_OK;
  }
  r.order = srv->next_order++;
  srv->queued_work += work;
  srv->reserved += bytes;
  srv->reserved_peak = std::max(srv->reserved_peak, srv->reserved);
  ++srv->admitted;
  srv->queue.push_back(r);
  srv->cv_work.notify_one();
  if (admitted) *admitted = 1;
  return SRK_OK;
}

extern "C" int srk_server_drain(srk_server *srv) {
  if (!srv) return fail(SRK_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(srv->mu);
  srv->cv_idle.wait(lk, [&] { return srv->queue.empty() && srv->running == 0; });
  return SRK_OK;
}

extern "C" int srk_server_stats(srk_server *srv, srk_server_report *st) {
  if (!srv || !st) return fail(SRK_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  memset(st, 0, sizeof *st);
  st->submitted = srv->submitted;
  st->admitted = srv->admitted;
  st->shed = srv->shed;
  st->completed = srv->completed;
  st->failed = srv->failed;
  st->target_steps = srv->target_steps;
  st->reserved_peak = srv->reserved_peak;
  st->p50_ms = percentile(srv->latency_ms, 0.50);
  st->p99_ms = percentile(srv->latency_ms, 0.99);
  double sum = 0.0, mx = 0.0;
  for (double x : srv->latency_ms) {
    sum += x;
    mx = std::max(mx, x);
  }
  st->mean_ms = srv->latency_ms.empty() ? 0.0 : sum / (double)srv->latency_ms.size();
  st->max_ms = mx;
  if (srv->have_first && srv->completed)
    st->wall_s = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
  st->queries_per_s = st->wall_s > 0.0 ? (double)srv->completed / st->wall_s : 0.0;
  return SRK_OK;
}

extern "C" int srk_server_destroy(srk_server *srv) {
  if (!srv) return SRK_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto &th : srv->workers) th.join();
  delete srv;
  return SRK_OK;
}

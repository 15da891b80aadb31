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
// time to fit it.  Per graph the server keeps two figures, measured when it is
// created by a few small calibration queries and refined by every completed
// request (exponential averages): the walk steps per (target, pair) and the
// walk steps per second of service.  A request's estimated time is (targets
// with in-neighbours) x N_tot x steps per pair / steps per second (none when
// the source has no in-neighbours: its walks cannot leave it); a request is
// admitted when the estimated time of the admitted, unfinished requests plus
// its own fits the target.  The queue is then served shortest estimated time
// first, so short queries are not held behind long ones; without a target it
// is first in, first out.
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
  double pairs;  // (targets with in-neighbours) x N_tot, 0 when s has none
  double work;   // estimated seconds of service
  uint64_t order;
  Clock::time_point t_submit;
};

// Calibration of a graph at server creation: this many queries from evenly
// spaced nodes with in-neighbours, each with z = kCalibZ walks per pair.
constexpr int kCalibQueries = 4;
constexpr double kCalibZ = 256.0;

}  // namespace

struct srk_server {
  std::vector<const srk_graph *> graphs;
  std::vector<std::vector<uint8_t>> has_in;  // per graph: node has in-neighbours
  std::vector<double> steps_per_pair;        // per graph: walk steps per (target, pair)
  std::vector<double> steps_per_s;           // per graph: walk steps per second of service
  size_t budget = 0;
  double target_ms = 0.0;     // 0: memory-only admission, FIFO
  double queued_work = 0.0;   // estimated seconds of admitted, unfinished requests
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
        const double steps = (double)stats.target_steps;
        if (r.pairs > 0.0 && steps > 1.0e6 && secs > 0.0) {  // refine the graph's figures
          double &spp = srv->steps_per_pair[(size_t)r.graph];
          double &sps = srv->steps_per_s[(size_t)r.graph];
          spp = 0.8 * spp + 0.2 * (steps / r.pairs);
          sps = 0.8 * sps + 0.2 * (steps / secs);
        }
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
  // calibration: steps per pair and steps per second of each graph
  for (int32_t i = 0; i < n_graphs; ++i) {
    const srk_graph *g = graphs[i];
    const std::vector<uint8_t> &has = srv->has_in[(size_t)i];
    std::vector<int32_t> act;
    for (size_t v = 0; v < has.size(); ++v)
      if (has[v]) act.push_back((int32_t)v);
    double spp = 0.8, sps = 5.0e10;  // used when the graph has no walk steps
    if (!act.empty()) {
      DeviceGuard guard(g->device);
      double *d = nullptr;
      cudaStream_t st = nullptr;
      cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess)
        e = cudaMallocFromPoolAsync((void **)&d, sizeof(double) * (size_t)g->n, pool(g->device),
                                    st);
      double steps = 0.0, pairs = 0.0, secs = 0.0;
      for (int k = 0; k < kCalibQueries && e == cudaSuccess; ++k) {
        const int32_t s = act[act.size() * (size_t)(2 * k + 1) / (2 * kCalibQueries)];
        srk_stats stats;
        srk_opts opt;
        memset(&opt, 0, sizeof opt);
        opt.L_override = -1;
        opt.z_override = kCalibZ;
        opt.stats = &stats;
        const Clock::time_point t0 = Clock::now();
        if (srk_single_source(g, s, 0.6, 0.5, 1, &opt, d, nullptr, nullptr, st) != SRK_OK ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          e = cudaErrorUnknown;
          break;
        }
        secs += std::chrono::duration<double>(Clock::now() - t0).count();
        steps += (double)stats.target_steps;
        pairs += (double)g->n_act * (double)stats.n_walks;
      }
      if (d) cudaFreeAsync(d, st);
      if (st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
      }
      if (e != cudaSuccess) {
        delete srv;
        return fail(SRK_ECUDA, "srk_server_create: calibrating graph %d: %s", i,
                    srk_last_error());
      }
      if (steps > 0.0 && pairs > 0.0 && secs > 0.0) {
        spp = steps / pairs;
        sps = steps / secs;
      }
    }
    srv->steps_per_pair.push_back(spp);
    srv->steps_per_s.push_back(sps);
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
  const double pairs =
      srv->has_in[(size_t)graph][(size_t)s] ? (double)g->n_act * (double)t.N_tot : 0.0;
  Request r;
  r.graph = graph;
  r.s = s;
  r.c = c;
  r.eps = eps;
  r.seed = seed;
  r.tag = tag;
  r.host_scores = host_scores;
  r.bytes = bytes;
  r.pairs = pairs;
  r.t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(srv->mu);
  const double work = pairs * srv->steps_per_pair[(size_t)graph] / srv->steps_per_s[(size_t)graph];
  r.work = work;
  ++srv->submitted;
  if (!srv->have_first) {
    srv->have_first = true;
    srv->t_first = r.t_submit;
  }
  const bool mem_ok = srv->reserved + bytes <= srv->budget;
  const bool time_ok = srv->target_ms <= 0.0 || (srv->queued_work + work) * 1e3 <= srv->target_ms;
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

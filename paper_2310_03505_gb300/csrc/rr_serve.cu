// rr_serve.cu -- a scan server: resident scenes, requests admitted by device
// memory, continuous batching, latency accounting.
//
// Clients submit scan requests (scene, pose, sensor model, output) from any
// thread; each gets a ticket.  One worker thread owns the GPU side.  It keeps
// up to `slots` launch sequences in flight, each on its own stream with its
// own execution context and a fixed device arena carved from the memory
// budget when the server is created (nothing is allocated while serving).
// Whenever a slot is free the worker forms the next batch: the oldest waiting
// request's scene, then every other waiting request for that scene in
// arrival order whose ray tree still fits the slot's arena (and the scan /
// ray limits of a batch).  A ray tree is sized by an estimate once the scene
// has run a batch: the largest queue and record counts per initial ray seen
// on that scene at every bounce (bounces not seen yet: twice the previous
// one), times the configured safety factor -- far below the worst
// case (every hit spawning both children), so more requests share a launch
// sequence.  A batch that outgrows its estimate (the device reports
// RR_ERR_CAPACITY, nothing is dropped silently) goes back to the front of the
// queue and its requests are rerun at worst-case size.  The batch runs as one launch sequence
// of rr_scan_batch's kernels, so requests that arrive while others are on the
// GPU join the next batch as soon as a slot and its memory free up, and the
// batches of different slots overlap on the device.  A finished batch's
// requests are completed in one go (host outputs copied back), their
// latencies (submit to completion, host steady clock) recorded.
//
// A request computes exactly what rr_scan computes for it: only the order in
// which returns are added to a bin may differ with its batch mates.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rr_host.h"

namespace rr_host {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  rr_scene* scene = nullptr;
  rr_pose pose;
  rr_sensor_params params;
  float* out = nullptr;
  bool out_on_device = false;
  size_t image_bytes = 0;
  int state = RR_REQ_QUEUED;
  int status = RR_OK;
  double submit_ms = 0, start_ms = 0, done_ms = 0;
  uint32_t batch_size = 0;
  uint64_t rays0 = 0;
  bool worst = false;   // size its batch for the worst-case tree (a retry after an overflow)
};

// completed, failed or cancelled: nothing of it is left on the device
inline bool req_finished(const Request& r) {
  return r.state == RR_REQ_DONE || r.state == RR_REQ_FAILED || r.state == RR_REQ_CANCELLED;
}

// largest queue length and return records per initial ray seen at every
// bounce of a scene's batches
struct Growth {
  uint32_t depth = 0;   // bounces seen (0: no batch yet)
  double q[RR_MAX_BOUNCES + 1] = {0};
  double r[RR_MAX_BOUNCES + 1] = {0};
};

struct Slot {
  ExecCtx ctx;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<uint64_t> batch;   // tickets in flight (empty: free)
  std::vector<float*> images;    // device image of each
  unsigned long long closest0 = 0, anyhit0 = 0;   // counters before the batch
  bool estimated = false;        // the batch was sized by the growth estimate
  uint64_t n0 = 0;               // initial rays of the batch
  uint32_t max_bounces = 0;
};

}  // namespace rr_host

struct rr_server {
  rr_serve_config cfg;
  rr_host::LaunchCfg launch;
  int device = 0;
  rr_host::Clock::time_point t0;
  std::vector<rr_host::Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending;                                  // waiting tickets, arrival order
  std::unordered_map<uint64_t, rr_host::Request> reqs;          // live and finished, until read
  std::unordered_map<const rr_scene*, rr_host::Growth> growth;  // ray-tree statistics per scene
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  // statistics since the last reset
  uint64_t submitted = 0, completed = 0, failed = 0, rejected = 0, batches = 0, retried = 0, cancelled = 0;
  uint64_t closest = 0, anyhit = 0, rays0 = 0;
  double stats_t0 = 0, busy_ms = 0;
  std::vector<double> latencies;
};

namespace rr_host {

static double now_ms(const rr_server* sv) {
  return std::chrono::duration<double, std::milli>(Clock::now() - sv->t0).count();
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// arena bytes of a batch (requests of one scene): workspace plus device
// images of host outputs.  The workspace is sized by the scene's growth
// estimate when there is one and no request asks for the worst case
// (*estimated says which), else for the worst-case tree.
static size_t batch_bytes(const rr_server* sv, const std::vector<const Request*>& b, WsLayout* L_out,
                          bool* estimated) {
  std::vector<rr_sensor_params> ps(b.size());
  size_t img = 0;
  bool est = sv != nullptr && !b.empty();
  for (size_t i = 0; i < b.size(); ++i) {
    ps[i] = b[i]->params;
    if (!b[i]->out_on_device) img += align256(b[i]->image_bytes);
    if (b[i]->worst) est = false;
  }
  const Growth* g = nullptr;
  if (est && sv->cfg.admission == RR_ADMIT_WORST_CASE) est = false;
  if (est) {
    auto it = sv->growth.find(b[0]->scene);
    if (it == sv->growth.end() || it->second.depth == 0) est = false;
    else g = &it->second;
  }
  WsLayout L;
  if (est) {
    const double f = sv->cfg.estimate_factor;
    double qe = 0.0, re = 0.0;
    for (const Request* r : b) {
      double qmax = 0.0, rsum = 0.0, q = 1.0, rr_ = 2.0;
      for (uint32_t k = 0; k < r->params.max_bounces && k <= RR_MAX_BOUNCES; ++k) {
        // a bounce the scene has not reached yet: twice the previous one
        q = k < g->depth ? g->q[k] : 2.0 * q;
        rr_ = k < g->depth ? g->r[k] : 2.0 * rr_;
        qmax = std::max(qmax, q);
        rsum += rr_;
      }
      qe += (double)r->rays0 * qmax;
      re += (double)r->rays0 * rsum;
    }
    L = plan_workspace_caps(ps.data(), (uint32_t)ps.size(), (uint64_t)(f * qe) + 1, (uint64_t)(f * re) + 1);
  } else {
    L = plan_workspace(ps.data(), (uint32_t)ps.size(), ~uint64_t(0));
  }
  if (estimated) *estimated = est;
  if (L_out) *L_out = L;
  return align256(L.total) + img;
}

// complete the batch of a slot whose work has finished (worker thread, lock held)
static void finish_slot(rr_server* sv, Slot& sl) {
  const int status = device_status(&sl.ctx, sl.stream);
  const double t = now_ms(sv);
  sv->closest += sl.ctx.h_ctr->stat_closest - sl.closest0;
  sv->anyhit += sl.ctx.h_ctr->stat_anyhit - sl.anyhit0;
  const rr_scene* scene = sl.batch.empty() ? nullptr : sv->reqs[sl.batch.front()].scene;
  if (status == RR_OK && scene && sl.n0) {
    // the batch's queue and record counts per initial ray feed the scene's estimate
    Growth& g = sv->growth[scene];
    const rr::ScanCounters* c = sl.ctx.h_ctr;
    for (uint32_t k = 0; k < sl.max_bounces && k <= RR_MAX_BOUNCES; ++k) {
      g.q[k] = std::max(g.q[k], (double)c->count[k] / (double)sl.n0);
      const uint32_t r0 = c->rec_start[k], r1 = k < RR_MAX_BOUNCES ? c->rec_start[k + 1] : r0;
      g.r[k] = std::max(g.r[k], (double)(r1 >= r0 ? r1 - r0 : 0u) / (double)sl.n0);
    }
    g.depth = std::max(g.depth, std::min<uint32_t>(sl.max_bounces, RR_MAX_BOUNCES + 1));
  }
  if (status == RR_ERR_CAPACITY && sl.estimated) {
    // the batch outgrew its estimate: its requests go back to the front of the
    // queue, in their order, to run again sized for the worst case
    for (size_t k = sl.batch.size(); k-- > 0;) {
      auto it = sv->reqs.find(sl.batch[k]);
      if (it == sv->reqs.end()) continue;
      it->second.state = RR_REQ_QUEUED;
      it->second.worst = true;
      sv->pending.push_front(sl.batch[k]);
      ++sv->retried;
    }
    sl.batch.clear();
    sl.images.clear();
    return;
  }
  for (size_t k = 0; k < sl.batch.size(); ++k) {
    auto it = sv->reqs.find(sl.batch[k]);
    if (it == sv->reqs.end()) continue;
    Request& r = it->second;
    int st = status;
    if (st == RR_OK && !r.out_on_device) {
      const cudaError_t e = cudaMemcpyAsync(r.out, sl.images[k], r.image_bytes, cudaMemcpyDeviceToHost, sl.stream);
      const cudaError_t e2 = e == cudaSuccess ? cudaStreamSynchronize(sl.stream) : e;
      if (e2 != cudaSuccess) {
        cudaGetLastError();
        st = RR_ERR_CUDA;
      }
    }
    r.state = st == RR_OK ? RR_REQ_DONE : RR_REQ_FAILED;
    r.status = st;
    r.done_ms = t;
    if (st == RR_OK) {
      ++sv->completed;
      sv->latencies.push_back(r.done_ms - r.submit_ms);
    } else {
      ++sv->failed;
    }
  }
  sl.batch.clear();
  sl.images.clear();
}

// form and launch the next batch on a free slot (worker thread, lock held);
// returns false when nothing could be launched
static bool launch_slot(rr_server* sv, Slot& sl) {
  if (sv->pending.empty()) return false;
  rr_scene* scene = sv->reqs[sv->pending.front()].scene;
  std::vector<const Request*> b;
  std::vector<uint64_t> tickets;
  uint64_t rays = 0;
  for (auto it = sv->pending.begin(); it != sv->pending.end(); ++it) {
    const Request& r = sv->reqs[*it];
    if (r.scene != scene) continue;
    if (b.size() >= sv->cfg.max_batch_scans) break;
    if (!b.empty() && rays + r.rays0 > sv->cfg.max_batch_rays) continue;
    b.push_back(&r);
    if (!b.empty() && batch_bytes(sv, b, nullptr, nullptr) > sl.arena_bytes) {
      b.pop_back();
      continue;
    }
    tickets.push_back(*it);
    rays += r.rays0;
  }
  if (b.empty()) return false;   // cannot happen: every request fits a slot alone (checked at submit)
  WsLayout L;
  bool estimated = false;
  batch_bytes(sv, b, &L, &estimated);
  // device images: caller's device buffers, or arena space after the workspace
  std::vector<float*> images(b.size());
  std::vector<rr_pose> poses(b.size());
  std::vector<rr_sensor_params> ps(b.size());
  size_t off = align256(L.total);
  for (size_t k = 0; k < b.size(); ++k) {
    poses[k] = b[k]->pose;
    ps[k] = b[k]->params;
    if (b[k]->out_on_device) {
      images[k] = b[k]->out;
    } else {
      images[k] = reinterpret_cast<float*>(sl.arena + off);
      off += align256(b[k]->image_bytes);
    }
  }
  const double t = now_ms(sv);
  for (uint64_t tk : tickets) {
    Request& r = sv->reqs[tk];
    r.state = RR_REQ_RUNNING;
    r.start_ms = t;
    r.batch_size = (uint32_t)tickets.size();
    sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), tk));
  }
  sl.closest0 = sl.ctx.h_ctr->stat_closest;
  sl.anyhit0 = sl.ctx.h_ctr->stat_anyhit;
  int rc = batch_enqueue(scene, &sl.ctx, poses.data(), ps.data(), images.data(), (uint32_t)b.size(), nullptr,
                         sl.stream, sl.arena, L, false, false, sv->launch, nullptr);
  if (rc == RR_OK) {
    const cudaError_t e = cudaEventRecord(sl.done, sl.stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = RR_ERR_CUDA;
    }
  }
  if (rc != RR_OK) {
    for (uint64_t tk : tickets) {
      Request& r = sv->reqs[tk];
      r.state = RR_REQ_FAILED;
      r.status = rc;
      r.done_ms = now_ms(sv);
      ++sv->failed;
    }
    cudaStreamSynchronize(sl.stream);
    return true;
  }
  sl.batch = tickets;
  sl.images = images;
  sl.estimated = estimated;
  sl.n0 = rays;
  sl.max_bounces = 0;
  for (const Request* r : b) sl.max_bounces = std::max(sl.max_bounces, r->params.max_bounces);
  ++sv->batches;
  sv->rays0 += rays;
  return true;
}

static void worker_main(rr_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  double busy_since = -1.0;
  while (true) {
    bool progress = false;
    size_t in_flight = 0;
    for (Slot& sl : sv->slots) {
      if (sl.batch.empty()) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) {
        ++in_flight;
        continue;
      }
      if (q != cudaSuccess) cudaGetLastError();
      finish_slot(sv, sl);
      progress = true;
    }
    if (progress) sv->cv_done.notify_all();
    for (Slot& sl : sv->slots) {
      if (!sl.batch.empty()) continue;
      if (!launch_slot(sv, sl)) break;
      if (!sl.batch.empty()) ++in_flight;
      progress = true;
    }
    if (progress) sv->cv_done.notify_all();
    const double t = now_ms(sv);
    if (in_flight && busy_since < 0) busy_since = t;
    if (!in_flight && busy_since >= 0) {
      sv->busy_ms += t - busy_since;
      busy_since = -1.0;
    }
    if (sv->stop && sv->pending.empty() && !in_flight) break;
    if (progress) continue;
    if (in_flight) {
      // poll the slots' events; new requests wake the loop at once
      sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
    } else {
      sv->cv_work.wait(lk, [sv] { return sv->stop || !sv->pending.empty(); });
    }
  }
  if (busy_since >= 0) sv->busy_ms += now_ms(sv) - busy_since;
}

static int serve_check(const rr_serve_config* c) {
  if (c->slots > 16) return fail(RR_ERR_INVALID_ARG, "slots must be in [1, 16] (0: 4)");
  if (c->node_format != RR_NODES_WIDE8 && c->node_format != RR_NODES_BINARY)
    return fail(RR_ERR_INVALID_ARG, "node_format must be RR_NODES_WIDE8 or RR_NODES_BINARY");
  if (c->refill_threshold > 32) return fail(RR_ERR_INVALID_ARG, "refill_threshold must be in [0, 32]");
  if (c->admission > RR_ADMIT_WORST_CASE)
    return fail(RR_ERR_INVALID_ARG, "admission must be RR_ADMIT_ESTIMATE or RR_ADMIT_WORST_CASE");
  if (!(c->estimate_factor >= 0.0f) || !std::isfinite(c->estimate_factor))
    return fail(RR_ERR_INVALID_ARG, "estimate_factor must be finite and >= 0 (0: 2)");
  return RR_OK;
}

}  // namespace rr_host

using namespace rr_host;

extern "C" {

int rr_serve_create(const rr_serve_config* config, rr_server** out) {
  if (!out) return fail(RR_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  rr_serve_config c;
  memset(&c, 0, sizeof c);
  if (config) c = *config;
  int rc = serve_check(&c);
  if (rc != RR_OK) return rc;
  if (!c.memory_budget) c.memory_budget = uint64_t(16) << 30;
  if (!c.slots) c.slots = 4;
  if (!c.max_batch_scans) c.max_batch_scans = 64;
  if (!c.max_batch_rays) c.max_batch_rays = 4u << 20;
  if (!c.max_queue) c.max_queue = 4096;
  if (!c.refill_threshold) c.refill_threshold = 16;
  if (c.estimate_factor == 0.0f) c.estimate_factor = 2.0f;
  if (c.memory_budget / c.slots < (uint64_t(16) << 20))
    return fail(RR_ERR_INVALID_ARG, "memory_budget must give every slot at least 16 MiB");
  rr_server* sv = new rr_server();
  sv->cfg = c;
  sv->launch.node_format = c.node_format;
  sv->launch.refill = c.refill_threshold;
  sv->launch.use_graph = 0;
  sv->t0 = Clock::now();
  cudaGetDevice(&sv->device);
  sv->slots.resize(c.slots);
  const size_t arena = (size_t)(c.memory_budget / c.slots) & ~size_t(255);
  cudaError_t e = cudaSuccess;
  for (Slot& sl : sv->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = ctx_init(&sl.ctx, sl.stream);
    if (e == cudaSuccess) e = dev_malloc((void**)&sl.arena, arena);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sl.stream);
    sl.arena_bytes = arena;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    rr_serve_destroy(sv);
    return cuda_fail(e, "creating the server's slots");
  }
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return RR_OK;
}

int rr_serve_destroy(rr_server* sv) {
  if (!sv) return RR_OK;
  if (sv->worker.joinable()) {
    {
      std::lock_guard<std::mutex> g(sv->mu);
      sv->stop = true;
    }
    sv->cv_work.notify_all();
    sv->worker.join();
  }
  for (Slot& sl : sv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    ctx_free(&sl.ctx);
    if (sl.arena) cudaFree(sl.arena);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete sv;
  return RR_OK;
}

int rr_serve_submit(rr_server* sv, rr_scene* scene, const rr_pose* pose, const rr_sensor_params* params,
                    float* out_polar, uint64_t* ticket) {
  if (!sv || !scene || !out_polar || !ticket) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  int rc = check_params(pose, params);
  if (rc != RR_OK) return rc;
  if (scene->device != sv->device)
    return fail(RR_ERR_INVALID_ARG, "rr_serve_submit: the scene lives on device " + std::to_string(scene->device) +
                                        ", the server on device " + std::to_string(sv->device));
  Request r;
  r.scene = scene;
  r.pose = *pose;
  r.params = *params;
  r.out = out_polar;
  r.out_on_device = is_device_ptr(out_polar);
  r.image_bytes = (size_t)params->n_azimuth * params->n_bins * sizeof(float);
  r.rays0 = (uint64_t)params->n_azimuth * params->rays_per_beam;
  std::vector<const Request*> alone = {&r};
  const size_t need = batch_bytes(nullptr, alone, nullptr, nullptr);   // worst case: a retry must fit
  if (need > sv->slots[0].arena_bytes)
    return fail(RR_ERR_INVALID_ARG, "the request needs " + std::to_string(need) + " bytes of worst-case scratch, " +
                                        "more than a slot's " + std::to_string(sv->slots[0].arena_bytes) +
                                        "; raise memory_budget or lower slots");
  {
    std::lock_guard<std::mutex> g(sv->mu);
    if (sv->stop) return fail(RR_ERR_BUSY, "the server is shutting down");
    if (sv->pending.size() >= sv->cfg.max_queue) {
      ++sv->rejected;
      return fail(RR_ERR_BUSY, "the request queue is full");
    }
    r.ticket = sv->next_ticket++;
    r.submit_ms = now_ms(sv);
    sv->reqs[r.ticket] = r;
    sv->pending.push_back(r.ticket);
    ++sv->submitted;
    *ticket = r.ticket;
  }
  sv->cv_work.notify_one();
  return RR_OK;
}

int rr_serve_cancel(rr_server* sv, uint64_t ticket, int* cancelled) {
  if (!sv || !cancelled) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  *cancelled = 0;
  {
    std::lock_guard<std::mutex> g(sv->mu);   // the worker forms batches under this lock
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(RR_ERR_INVALID_ARG, "unknown ticket");
    Request& r = it->second;
    if (r.state != RR_REQ_QUEUED) return RR_OK;
    auto q = std::find(sv->pending.begin(), sv->pending.end(), ticket);
    if (q != sv->pending.end()) sv->pending.erase(q);
    r.state = RR_REQ_CANCELLED;
    r.status = RR_ERR_CANCELLED;
    r.done_ms = now_ms(sv);
    ++sv->cancelled;
    *cancelled = 1;
  }
  sv->cv_done.notify_all();
  return RR_OK;
}

int rr_serve_poll(rr_server* sv, uint64_t ticket, int* done) {
  if (!sv || !done) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return fail(RR_ERR_INVALID_ARG, "unknown ticket");
  *done = req_finished(it->second) ? 1 : 0;
  return RR_OK;
}

int rr_serve_wait(rr_server* sv, uint64_t ticket, uint32_t timeout_ms) {
  if (!sv) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto finished = [&] {
    auto it = sv->reqs.find(ticket);
    return it == sv->reqs.end() || req_finished(it->second);
  };
  if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished))
    return fail(RR_ERR_TIMEOUT, "the request is not finished");
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return fail(RR_ERR_INVALID_ARG, "unknown ticket");
  if (it->second.state == RR_REQ_CANCELLED) return fail(RR_ERR_CANCELLED, "the request was cancelled");
  if (it->second.status != RR_OK) return fail(it->second.status, "the request failed");
  return RR_OK;
}

int rr_serve_result(rr_server* sv, uint64_t ticket, rr_serve_record* out) {
  if (!sv || !out) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return fail(RR_ERR_INVALID_ARG, "unknown ticket");
  const Request& r = it->second;
  memset(out, 0, sizeof *out);
  out->state = r.state;
  out->status = r.status;
  out->submit_ms = r.submit_ms;
  out->start_ms = r.start_ms;
  out->done_ms = r.done_ms;
  out->batch_size = r.batch_size;
  if (req_finished(r)) sv->reqs.erase(it);
  return RR_OK;
}

int rr_serve_stats_get(rr_server* sv, rr_serve_stats* out, int reset) {
  if (!sv || !out) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(sv->mu);
  memset(out, 0, sizeof *out);
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->failed = sv->failed;
  out->rejected_busy = sv->rejected;
  out->batches = sv->batches;
  out->closest_queries = sv->closest;
  out->anyhit_queries = sv->anyhit;
  out->initial_rays = sv->rays0;
  out->busy_ms = sv->busy_ms;
  out->elapsed_ms = now_ms(sv) - sv->stats_t0;
  out->queued = sv->pending.size();
  out->retried = sv->retried;
  out->cancelled = sv->cancelled;
  std::vector<double> l = sv->latencies;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {   // nearest rank
      size_t k = (size_t)std::ceil(p / 100.0 * (double)l.size());
      return l[k ? k - 1 : 0];
    };
    double sum = 0;
    for (double v : l) sum += v;
    out->latency_p50_ms = pct(50);
    out->latency_p99_ms = pct(99);
    out->latency_mean_ms = sum / (double)l.size();
    out->latency_max_ms = l.back();
  }
  if (reset) {
    sv->submitted = sv->completed = sv->failed = sv->rejected = sv->batches = sv->retried = sv->cancelled = 0;
    sv->closest = sv->anyhit = sv->rays0 = 0;
    sv->busy_ms = 0;
    sv->stats_t0 = now_ms(sv);
    sv->latencies.clear();
  }
  return RR_OK;
}

}  // extern "C"

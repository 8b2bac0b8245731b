// rr_api.cu -- the extern "C" boundary declared in include/rr.h (scene,
// single scans, debug, counters; batches are in rr_batch.cu).
//
// Host code here validates arguments, owns device memory and orders the
// launches; every step of the scan itself runs in the kernels of
// rr_build.cu, rr_trace.cu and rr_image.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rr_host.h"

using rr::ScanArgs;
using rr::ScanCounters;

namespace rr_host {

static thread_local std::string t_error;
static thread_local cudaStream_t t_stream = nullptr;

void set_error(const std::string& msg) { t_error = msg; }
cudaStream_t current_stream() { return t_stream; }

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

// host-side fault injection: the number of allocations still to let pass
// before one fails (-1: off), and the allocations seen since the last query
static std::atomic<int64_t> g_alloc_countdown{-1};
static std::atomic<uint64_t> g_allocs_seen{0};

static bool injected_alloc_failure() {
  g_allocs_seen.fetch_add(1, std::memory_order_relaxed);
  int64_t c = g_alloc_countdown.load();
  while (c >= 0)
    if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 0;   // the armed one fails, then off
  return false;
}

cudaError_t dev_malloc_raw(void** p, size_t n) {
  if (injected_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, n);
}

cudaError_t host_malloc_raw(void** p, size_t n) {
  if (injected_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, n);
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? RR_ERR_OOM : RR_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define RR_CHECK_CUDA(expr, what)              \
  do {                                         \
    cudaError_t e__ = (expr);                  \
    if (e__ != cudaSuccess) {                  \
      cudaGetLastError();                      \
      return cuda_fail(e__, what);             \
    }                                          \
  } while (0)

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// profiling
void prof_begin(rr_scene* s, int kind, cudaStream_t st, cudaEvent_t* stop_out) {
  *stop_out = nullptr;
  if (!s->prof) return;
  ProfEvent ev;
  ev.kind = kind;
  for (cudaEvent_t* e : {&ev.start, &ev.stop}) {
    if (!s->prof_pool.empty()) {
      *e = s->prof_pool.back();
      s->prof_pool.pop_back();
    } else {
      cudaEventCreate(e);
    }
  }
  cudaEventRecord(ev.start, st);
  s->prof_pending.push_back(ev);
  *stop_out = ev.stop;
}

void prof_end(rr_scene* s, cudaEvent_t stop, cudaStream_t st) {
  if (stop) cudaEventRecord(stop, st);
}

static void prof_collect(rr_scene* s) {
  for (ProfEvent& ev : s->prof_pending) {
    float ms = 0.f, t0 = 0.f, t1 = 0.f;
    if (cudaEventSynchronize(ev.stop) == cudaSuccess && cudaEventElapsedTime(&ms, ev.start, ev.stop) == cudaSuccess) {
      s->prof_ms[ev.kind] += ms;
      s->prof_launches[ev.kind] += 1;
      if (s->prof_base && cudaEventElapsedTime(&t0, s->prof_base, ev.start) == cudaSuccess &&
          cudaEventElapsedTime(&t1, s->prof_base, ev.stop) == cudaSuccess)
        s->prof_iv[ev.kind].push_back({t0, t1});
    }
    s->prof_pool.push_back(ev.start);
    s->prof_pool.push_back(ev.stop);
  }
  s->prof_pending.clear();
}

// length of the union of the collected intervals of one kind
static double prof_union(std::vector<std::pair<double, double>>& iv) {
  std::sort(iv.begin(), iv.end());
  double total = 0.0, a = 0.0, b = -1.0;
  bool open = false;
  for (const auto& x : iv) {
    if (open && x.first <= b) {
      b = std::max(b, x.second);
      continue;
    }
    if (open) total += b - a;
    a = x.first;
    b = x.second;
    open = true;
  }
  if (open) total += b - a;
  return total;
}

// ---------------------------------------------------------------------------
// parameter checks
static bool finite_f(float x) { return std::isfinite(x); }

int check_params(const rr_pose* pose, const rr_sensor_params* p) {
  if (!pose || !p) return fail(RR_ERR_INVALID_ARG, "pose and params must not be NULL");
  if (p->n_azimuth < 1 || p->n_azimuth > RR_MAX_AZIMUTH) return fail(RR_ERR_INVALID_ARG, "n_azimuth out of range");
  if (p->rays_per_beam < 1 || p->rays_per_beam > RR_MAX_RAYS_PER_BEAM)
    return fail(RR_ERR_INVALID_ARG, "rays_per_beam out of range");
  if (p->max_bounces < 1 || p->max_bounces > RR_MAX_BOUNCES)
    return fail(RR_ERR_INVALID_ARG, "max_bounces must be in [1, 16]");
  if (p->n_bins < 1 || p->n_bins > RR_MAX_BINS) return fail(RR_ERR_INVALID_ARG, "n_bins must be in [1, 16384]");
  if ((uint64_t)p->n_azimuth * p->rays_per_beam > (1ull << 30))
    return fail(RR_ERR_INVALID_ARG, "n_azimuth * rays_per_beam exceeds 2^30");
  const float fs[] = {p->beam_width_rad, p->beam_prob, p->elevation_rad, p->bin_size_m, p->t_min_m, p->min_energy,
                      p->freq_hz, p->blur_sigma_bins, p->az_pattern_sigma, p->noise_sys, p->noise_amb,
                      p->beam_aspect, p->noise_cell_az, p->noise_cell_bins, p->range_falloff};
  for (float f : fs)
    if (!finite_f(f)) return fail(RR_ERR_INVALID_ARG, "sensor parameters must be finite");
  if (p->beam_width_rad < 0.f || p->beam_width_rad > 3.14159265f)
    return fail(RR_ERR_INVALID_ARG, "beam_width_rad must be in [0, pi]");
  if (p->beam_width_rad > 0.f && !(p->beam_prob > 0.f && p->beam_prob < 1.f))
    return fail(RR_ERR_INVALID_ARG, "beam_prob must be in (0, 1)");
  if (!(p->bin_size_m > 0.f)) return fail(RR_ERR_INVALID_ARG, "bin_size_m must be > 0");
  if (p->t_min_m < 0.f || p->min_energy < 0.f) return fail(RR_ERR_INVALID_ARG, "t_min_m and min_energy must be >= 0");
  if (!(p->freq_hz > 0.f)) return fail(RR_ERR_INVALID_ARG, "freq_hz must be > 0");
  if (p->blur_sigma_bins < 0.f || p->blur_sigma_bins > 256.f || p->az_pattern_sigma < 0.f ||
      p->az_pattern_sigma > 256.f)
    return fail(RR_ERR_INVALID_ARG, "blur / pattern sigma must be in [0, 256]");
  if (p->noise_sys < 0.f || p->noise_amb < 0.f) return fail(RR_ERR_INVALID_ARG, "noise amplitudes must be >= 0");
  if (p->beam_aspect < 0.f || p->beam_aspect > 100.f)
    return fail(RR_ERR_INVALID_ARG, "beam_aspect must be in [0, 100] (0: circular)");
  if ((p->noise_cell_az != 0.f && p->noise_cell_az < 1.f) || (p->noise_cell_bins != 0.f && p->noise_cell_bins < 1.f) ||
      p->noise_cell_az > 1e6f || p->noise_cell_bins > 1e6f)
    return fail(RR_ERR_INVALID_ARG, "noise cells must be 0 (default) or in [1, 1e6]");
  if (p->range_falloff < 0.f || p->range_falloff > 16.f)
    return fail(RR_ERR_INVALID_ARG, "range_falloff must be in [0, 16]");
  for (int i = 0; i < 3; ++i)
    if (!finite_f(pose->p[i])) return fail(RR_ERR_INVALID_ARG, "pose position must be finite");
  double qn = 0.0;
  for (int i = 0; i < 4; ++i) {
    if (!finite_f(pose->q[i])) return fail(RR_ERR_INVALID_ARG, "pose quaternion must be finite");
    qn += (double)pose->q[i] * pose->q[i];
  }
  if (!(qn > 1e-12)) return fail(RR_ERR_INVALID_ARG, "pose quaternion must be non-zero");
  return RR_OK;
}

// The scene's buffers live on the device that was current when it was
// created; its kernels must be launched there.  A call made with another
// device current is refused before anything is queued: without peer access
// the kernels would fault on the scene's pointers.
int check_device(const rr_scene* s, const char* who) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RR_ERR_CUDA, std::string(who) + ": no usable current device");
  }
  if (dev != s->device)
    return fail(RR_ERR_INVALID_ARG, std::string(who) + ": the scene lives on device " + std::to_string(s->device) +
                                        " but device " + std::to_string(dev) + " is current");
  return RR_OK;
}

// read (and clear) the sticky device status of a context; waits for the stream
int device_status(ExecCtx* x, cudaStream_t st) {
  RR_CHECK_CUDA(cudaMemcpyAsync(x->h_ctr, x->d_ctr, sizeof(ScanCounters), cudaMemcpyDeviceToHost, st),
                "reading the scan counters");
  RR_CHECK_CUDA(cudaStreamSynchronize(st), "scan");
  const uint32_t err = x->h_ctr->error;
  if (err) {
    RR_CHECK_CUDA(cudaMemsetAsync(&x->d_ctr->error, 0, sizeof(uint32_t), st), "clearing the status");
    RR_CHECK_CUDA(cudaMemsetAsync(&x->d_ctr->need_rays, 0, 2 * sizeof(uint32_t), st), "clearing the status");
    RR_CHECK_CUDA(cudaStreamSynchronize(st), "clearing the status");
    char msg[256];
    if (err & rr::kErrBadVertex)
      return fail(RR_ERR_INVALID_ARG, "a rebuild saw an invalid vertex index or a non-finite vertex");
    if (err & rr::kErrBvh) return fail(RR_ERR_CUDA, "the BVH build failed; nothing was traced");
    if (err & rr::kErrStack) return fail(RR_ERR_CAPACITY, "BVH deeper than the traversal stack");
    if (err & rr::kErrTimeout) return fail(RR_ERR_TIMEOUT, "a bounded device wait gave up");
    if (err & (rr::kErrCapacityRays | rr::kErrCapacityRecs)) {
      snprintf(msg, sizeof msg,
               "ray tree outgrew the workspace: %u queued rays and %u return records were needed; raise the "
               "workspace limit",
               x->h_ctr->need_rays, x->h_ctr->need_recs);
      return fail(RR_ERR_CAPACITY, msg);
    }
    if (err & rr::kErrCapacitySegs) return fail(RR_ERR_CAPACITY, "segment buffer too small");
    return fail(RR_ERR_CUDA, "unknown device status");
  }
  return RR_OK;
}

int scene_status(rr_scene* s, cudaStream_t st) {
  int rc = device_status(&s->main, st);   // st has joined the split lanes' work
  for (uint32_t k = 0; k < s->split_used; ++k) {
    const int r = device_status(&s->split[k].ctx, s->split[k].stream);
    if (rc == RR_OK) rc = r;
  }
  return rc;
}

cudaError_t ctx_init(ExecCtx* x, cudaStream_t st) {
  cudaError_t e = dev_malloc((void**)&x->d_ctr, sizeof(ScanCounters));
  if (e == cudaSuccess) e = host_malloc((void**)&x->h_ctr, sizeof(ScanCounters));
  if (e == cudaSuccess) memset(x->h_ctr, 0, sizeof(ScanCounters));   // the mirror starts equal to the device
  if (e == cudaSuccess) e = cudaMemsetAsync(x->d_ctr, 0, sizeof(ScanCounters), st);
  return e;
}

void ctx_free(ExecCtx* x) {
  if (x->d_ctr) cudaFree(x->d_ctr);
  if (x->h_ctr) cudaFreeHost(x->h_ctr);
  if (x->ws) cudaFree(x->ws);
  if (x->d_image) cudaFree(x->d_image);
  if (x->h_stage) cudaFreeHost(x->h_stage);
  if (x->stage_ev) cudaEventDestroy(x->stage_ev);
  if (x->gexec) cudaGraphExecDestroy(x->gexec);
  if (x->cap_stream) cudaStreamDestroy(x->cap_stream);
  for (int b = 0; b < RR_MAX_BOUNCES; ++b) {
    if (x->fork[b]) cudaEventDestroy(x->fork[b]);
    if (x->join[b]) cudaEventDestroy(x->join[b]);
  }
  if (x->side) cudaStreamDestroy(x->side);
  *x = ExecCtx();
}

}  // namespace rr_host

using namespace rr_host;

int rr_host::rebuild_bvh(rr_scene* s, cudaStream_t st) {
  if (s->nt == 0) return RR_OK;
  RR_CHECK_CUDA(build_lbvh(s, st, true), "rebuilding the BVH");
  uint32_t misc[8];
  RR_CHECK_CUDA(cudaMemcpyAsync(misc, s->d_misc, sizeof misc, cudaMemcpyDeviceToHost, st), "reading the build status");
  RR_CHECK_CUDA(cudaStreamSynchronize(st), "rebuilding the BVH");
  if (misc[6] & rr::kErrTopBuild) return fail(RR_ERR_CUDA, "the SAH top of the BVH could not be built");
  if (misc[6]) return fail(RR_ERR_INVALID_ARG, "the scene's vertices are invalid");
  s->depth = misc[7];
  if (s->depth > (uint32_t)rr::kStack)
    return fail(RR_ERR_CAPACITY, "BVH depth " + std::to_string(s->depth) + " exceeds the traversal stack");
  return RR_OK;
}

// one-thread kernel folding the build status into the scan status word
__global__ void k_fold_build_status(const uint32_t* misc, const uint32_t* wctr, ScanCounters* ctr) {
  uint32_t e = 0;
  if (misc[6] & ~rr::kErrTopBuild) e |= rr::kErrBadVertex;
  if ((misc[6] & rr::kErrTopBuild) || wctr[4]) e |= rr::kErrBvh;
  if (e) atomicOr(&ctr->error, e);
}

extern "C" {

int rr_version(void) { return RR_VERSION; }

const char* rr_last_error(void) { return t_error.c_str(); }

int rr_set_stream(void* cuda_stream) {
  t_stream = (cudaStream_t)cuda_stream;
  return RR_OK;
}

int rr_fault_inject_alloc(int64_t fail_at, uint64_t* allocs_seen) {
  if (allocs_seen) *allocs_seen = g_allocs_seen.exchange(0);
  g_alloc_countdown.store(fail_at < 0 ? -1 : fail_at);
  return RR_OK;
}

int rr_selftest_wait(uint32_t which, double* waited_ms) {
  if (which > RR_WAIT_SHADE_PREFIX) return fail(RR_ERR_INVALID_ARG, "rr_selftest_wait: unknown wait");
  const cudaStream_t st = t_stream;
  const size_t bytes = 256 + sizeof(ScanCounters);   // the largest arrangement, zeroed
  void* scratch = nullptr;
  RR_CHECK_CUDA(dev_malloc(&scratch, bytes), "allocating the self-test scratch");
  const auto t0 = std::chrono::steady_clock::now();
  bool gave_up = false;
  cudaError_t e = cudaMemsetAsync(scratch, 0, bytes, st);
  if (e == cudaSuccess) {
    if (which == RR_WAIT_TOP_TASK) e = selftest_top_wait(static_cast<uint32_t*>(scratch), st, &gave_up);
    else if (which == RR_WAIT_WIDE_NODE) e = selftest_wide_wait(static_cast<uint32_t*>(scratch), st, &gave_up);
    else e = selftest_look_back_wait(scratch, st, &gave_up);
  }
  const auto t1 = std::chrono::steady_clock::now();
  if (waited_ms) *waited_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(scratch);
    return cuda_fail(e, "running the self-test wait");
  }
  RR_CHECK_CUDA(cudaFree(scratch), "freeing the self-test scratch");
  if (!gave_up) return fail(RR_ERR_CUDA, "rr_selftest_wait: the wait ended without its error bit");
  return fail(RR_ERR_TIMEOUT, "a bounded device wait gave up (self-test: expected)");
}

int rr_scene_destroy(rr_scene* s) {
  if (!s) return RR_OK;
  cudaDeviceSynchronize();
  void* ptrs[] = {s->d_vtx, s->d_idx, s->d_mat_id, s->d_raw_mats, s->d_mats, s->d_lut, s->d_lut_cells,
                  s->d_tri, s->d_nodes, s->d_centroid, s->d_keys[0], s->d_keys[1], s->d_vals[0], s->d_vals[1],
                  s->d_hist, s->d_parent, s->d_child, s->d_nbox, s->d_visit, s->d_misc,
                  s->d_cut, s->d_wnodes, s->d_wtri, s->d_wsrc, s->d_wrec, s->d_wctr, s->d_lobe_kind,
                  s->d_lobe_samples, s->d_range, s->d_cl_at, s->d_cl_bsum, s->d_cl_rec,
                  s->d_top_slot, s->d_top_task, s->d_top_ready, s->d_top_small, s->d_top_ctr, s->d_top_cb};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  ctx_free(&s->main);
  for (SplitLane& ln : s->split) {
    ctx_free(&ln.ctx);
    if (ln.join) cudaEventDestroy(ln.join);
    if (ln.stream) cudaStreamDestroy(ln.stream);
  }
  if (s->fork) cudaEventDestroy(s->fork);
  if (s->wide_ready) cudaEventDestroy(s->wide_ready);
  for (auto& ev : s->prof_pending) {
    cudaEventDestroy(ev.start);
    cudaEventDestroy(ev.stop);
  }
  for (auto e : s->prof_pool) cudaEventDestroy(e);
  if (s->prof_base) cudaEventDestroy(s->prof_base);
  delete s;
  return RR_OK;
}

int rr_scene_create(const float* vertices, uint32_t n_vertices, const uint32_t* triangles, uint32_t n_triangles,
                    const uint16_t* material_ids, const rr_material* materials, uint32_t n_materials,
                    rr_scene** out) {
  if (!out) return fail(RR_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (n_triangles > 0 && (!vertices || !triangles || !material_ids))
    return fail(RR_ERR_INVALID_ARG, "vertices, triangles and material_ids must not be NULL");
  if (n_materials == 0 || !materials) return fail(RR_ERR_INVALID_ARG, "at least one material is required");
  if (n_materials > RR_MAX_MATERIALS) return fail(RR_ERR_INVALID_ARG, "too many materials");
  if (n_triangles > (1u << 30)) return fail(RR_ERR_INVALID_ARG, "more than 2^30 triangles");
  std::vector<rr_material> mats(n_materials);
  {
    cudaError_t e = cudaMemcpy(mats.data(), materials, n_materials * sizeof(rr_material), cudaMemcpyDefault);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "reading the materials");
    }
  }
  for (uint32_t m = 0; m < n_materials; ++m) {
    const rr_material& x = mats[m];
    if (!(std::isfinite(x.eps_r) && std::isfinite(x.loss_tangent) && std::isfinite(x.A) && std::isfinite(x.B) &&
          std::isfinite(x.C)))
      return fail(RR_ERR_INVALID_ARG, "material " + std::to_string(m) + ": non-finite value");
    const bool ct = (x.flags & RR_MAT_COOK_TORRANCE) != 0u, tab = (x.flags & RR_MAT_TABULATED_LOBE) != 0u;
    if (ct && tab) return fail(RR_ERR_INVALID_ARG, "material " + std::to_string(m) + ": one lobe kind only");
    if (x.eps_r < 1.f || x.loss_tangent < 0.f)
      return fail(RR_ERR_INVALID_ARG, "material " + std::to_string(m) + ": needs eps_r >= 1, tan_d >= 0");
    if (ct) {
      if (x.A < 0.f || x.A > 1.f || !(x.B >= 1e-3f && x.B <= 10.f))
        return fail(RR_ERR_INVALID_ARG, "material " + std::to_string(m) +
                                            ": Cook-Torrance needs 0 <= A (diffuse) <= 1, 1e-3 <= B (roughness) <= 10");
    } else if (x.A < 0.f || x.B < 0.f || x.A > 1.f || x.B > 1.f || x.A + x.B > 1.f + 1e-6f || x.C < 0.f) {
      return fail(RR_ERR_INVALID_ARG, "material " + std::to_string(m) +
                                          ": needs 0 <= A, B, A + B <= 1, C >= 0");
    }
  }
  cudaStream_t st = t_stream;
  rr_scene* s = new rr_scene();
  cudaGetDevice(&s->device);
  s->nv = n_vertices;
  s->nt = n_triangles;
  s->nm = n_materials;
  s->lobe_kind.resize(n_materials);
  for (uint32_t m = 0; m < n_materials; ++m)   // a tabulated lobe is Eq. 5 until it is set
    s->lobe_kind[m] = (mats[m].flags & RR_MAT_COOK_TORRANCE) ? (uint8_t)rr::kLobeCookTorrance : (uint8_t)rr::kLobeEq5;
  s->raw_flags.resize(n_materials);
  for (uint32_t m = 0; m < n_materials; ++m) s->raw_flags[m] = mats[m].flags;
  auto bail = [&](int code) {
    rr_scene_destroy(s);
    return code;
  };
  {
    cudaError_t e = build_alloc(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bail(cuda_fail(e, "allocating the scene"));
    }
  }
  cudaError_t e = cudaSuccess;
  e = ctx_init(&s->main, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(RR_ERR_OOM, "allocating the scan counters"));
  }
  if (e == cudaSuccess && n_vertices)
    e = cudaMemcpyAsync(s->d_vtx, vertices, (size_t)n_vertices * 3 * sizeof(float), cudaMemcpyDefault, st);
  if (e == cudaSuccess && n_triangles)
    e = cudaMemcpyAsync(s->d_idx, triangles, (size_t)n_triangles * 3 * sizeof(uint32_t), cudaMemcpyDefault, st);
  if (e == cudaSuccess && n_triangles)
    e = cudaMemcpyAsync(s->d_mat_id, material_ids, (size_t)n_triangles * sizeof(uint16_t), cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_raw_mats, mats.data(), n_materials * sizeof(rr_material), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = build_materials(s, st);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = build_lbvh(s, st, true);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return bail(cuda_fail(e, "building the scene"));
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->build_ms = ms;
  if (n_triangles) {
    uint32_t misc[8];
    e = cudaMemcpy(misc, s->d_misc, sizeof misc, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bail(cuda_fail(e, "reading the build status"));
    if (misc[6] & 1u) return bail(fail(RR_ERR_INVALID_ARG, "a triangle references a vertex index >= n_vertices"));
    if (misc[6] & 2u) return bail(fail(RR_ERR_INVALID_ARG, "a material id is >= n_materials"));
    if (misc[6] & rr::kErrBadVertex) return bail(fail(RR_ERR_INVALID_ARG, "non-finite vertex coordinates"));
    if (misc[6] & rr::kErrTopBuild) return bail(fail(RR_ERR_CUDA, "the SAH top of the BVH could not be built"));
    s->depth = misc[7];
    if (s->depth > (uint32_t)rr::kStack)
      return bail(fail(RR_ERR_CAPACITY, "BVH depth " + std::to_string(s->depth) + " exceeds the traversal stack"));
  }
  *out = s;
  return RR_OK;
}

int rr_scene_update_vertices(rr_scene* s, const float* vertices) {
  if (!s || !vertices) return fail(RR_ERR_INVALID_ARG, "scene and vertices must not be NULL");
  if (int rc = check_device(s, "rr_scene_update_vertices")) return rc;
  cudaStream_t st = t_stream;
  cudaEvent_t ev;
  if (s->nv)
    RR_CHECK_CUDA(cudaMemcpyAsync(s->d_vtx, vertices, (size_t)s->nv * 3 * sizeof(float), cudaMemcpyDefault, st),
                  "copying the vertices");
  prof_begin(s, RR_K_BUILD, st, &ev);
  RR_CHECK_CUDA(build_lbvh(s, st, false), "rebuilding the BVH");
  prof_end(s, ev, st);
  if (s->nt) {
    s->launches += 1;
    k_fold_build_status<<<1, 1, 0, st>>>(s->d_misc, s->d_wctr, s->main.d_ctr);
    RR_CHECK_CUDA(cudaGetLastError(), "status fold");
  }
  return RR_OK;
}

int rr_scene_info_get(const rr_scene* s, rr_scene_info* info) {
  if (!s || !info) return fail(RR_ERR_INVALID_ARG, "scene and info must not be NULL");
  memset(info, 0, sizeof *info);
  info->n_triangles = s->nt;
  info->n_materials = s->nm;
  info->bvh_depth = s->depth;
  if (s->nt && !s->wide_stale) {   // the count of the latest collapse
    uint32_t n = 0;
    RR_CHECK_CUDA(cudaStreamSynchronize(t_stream), "synchronising");
    RR_CHECK_CUDA(cudaMemcpy(&n, s->d_wctr + 1, sizeof n, cudaMemcpyDeviceToHost), "reading the wide node count");
    info->n_wide_nodes = n;
  }
  info->device_bytes = s->scene_bytes;
  info->workspace_bytes = s->main.ws_bytes;
  info->build_ms = s->build_ms;
  return RR_OK;
}

int rr_scene_export_bvh(const rr_scene* s, uint32_t* morton, uint32_t* perm, uint32_t* children, uint32_t* parents,
                        float* boxes) {
  if (!s) return fail(RR_ERR_INVALID_ARG, "scene must not be NULL");
  RR_CHECK_CUDA(cudaStreamSynchronize(t_stream), "synchronising");
  const size_t T = s->nt;
  if (T == 0) return RR_OK;
  if (morton) RR_CHECK_CUDA(cudaMemcpy(morton, s->d_keys[0], T * 4, cudaMemcpyDeviceToHost), "export");
  if (perm) RR_CHECK_CUDA(cudaMemcpy(perm, s->d_vals[0], T * 4, cudaMemcpyDeviceToHost), "export");
  if (T > 1 && children) RR_CHECK_CUDA(cudaMemcpy(children, s->d_child, (T - 1) * 8, cudaMemcpyDeviceToHost), "export");
  if (parents) RR_CHECK_CUDA(cudaMemcpy(parents, s->d_parent, (2 * T - 1) * 4, cudaMemcpyDeviceToHost), "export");
  if (T > 1 && boxes) {
    std::vector<float4> nodes((T - 1) * 4);
    RR_CHECK_CUDA(cudaMemcpy(nodes.data(), s->d_nodes, nodes.size() * sizeof(float4), cudaMemcpyDeviceToHost),
                  "export");
    for (size_t i = 0; i + 1 < T; ++i) {
      const float4 n0 = nodes[4 * i], n1 = nodes[4 * i + 1], n2 = nodes[4 * i + 2];
      float* b = boxes + 12 * i;
      const float v[12] = {n0.x, n0.z, n2.x, n0.y, n0.w, n2.y, n1.x, n1.z, n2.z, n1.y, n1.w, n2.w};
      memcpy(b, v, sizeof v);
    }
  }
  return RR_OK;
}

int rr_scene_set_lobe(rr_scene* s, uint32_t material, const float* density) {
  if (!s || !density) return fail(RR_ERR_INVALID_ARG, "scene and density must not be NULL");
  if (material >= s->nm) return fail(RR_ERR_INVALID_ARG, "material index out of range");
  if (int rc = check_device(s, "rr_scene_set_lobe")) return rc;
  if (!(s->raw_flags[material] & RR_MAT_TABULATED_LOBE))
    return fail(RR_ERR_INVALID_ARG, "the material was not created with RR_MAT_TABULATED_LOBE");
  std::vector<float> h(rr::kLobeSamples);
  RR_CHECK_CUDA(cudaMemcpy(h.data(), density, h.size() * sizeof(float), cudaMemcpyDefault), "reading the lobe");
  double total = 0.0;
  for (float v : h) {
    if (!std::isfinite(v) || v < 0.f) return fail(RR_ERR_INVALID_ARG, "lobe samples must be finite and >= 0");
    total += v;
  }
  if (!(total > 0.0)) return fail(RR_ERR_INVALID_ARG, "lobe samples must not all be zero");
  cudaStream_t st = t_stream;
  if (!s->d_lobe_samples) {
    const size_t bytes = (size_t)s->nm * rr::kLobeSamples * sizeof(float);
    RR_CHECK_CUDA(dev_malloc(&s->d_lobe_samples, bytes), "allocating the lobe samples");
    RR_CHECK_CUDA(cudaMemsetAsync(s->d_lobe_samples, 0, bytes, st), "clearing the lobe samples");
  }
  RR_CHECK_CUDA(cudaMemcpyAsync(s->d_lobe_samples + (size_t)material * rr::kLobeSamples, h.data(),
                                h.size() * sizeof(float), cudaMemcpyHostToDevice, st),
                "copying the lobe samples");
  s->lobe_kind[material] = (uint8_t)rr::kLobeTable;
  RR_CHECK_CUDA(build_materials(s, st), "rebuilding the lobe tables");   // synchronises (h stays alive)
  return RR_OK;
}

// Scene blob: a 64-byte header, then the payload -- vertices f32[V][3],
// triangles u32[T][3], material ids u16[T] (padded to 4 bytes), materials
// rr_material[M], the launch configuration rr_batch_config, and for every
// tabulated lobe its material index u32 and densities f32[RR_LOBE_SAMPLES].
// The checksum is FNV-1a (64 bit) over the payload.
struct SceneBlobHeader {
  char magic[8];            // "RRSCENE" and a zero byte
  uint32_t version, nv, nt, nm, n_tab, reserved;
  uint64_t payload_bytes, checksum;
  uint8_t pad[16];
};
static_assert(sizeof(SceneBlobHeader) == 64, "the blob header is 64 bytes");
static const char kBlobMagic[8] = {'R', 'R', 'S', 'C', 'E', 'N', 'E', 0};
constexpr uint32_t kBlobVersion = 1;

static uint64_t fnv1a(const unsigned char* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

static size_t blob_payload_bytes(uint32_t nv, uint32_t nt, uint32_t nm, uint32_t n_tab) {
  return (size_t)nv * 12 + (size_t)nt * 12 + (((size_t)nt * 2 + 3) & ~(size_t)3) + (size_t)nm * sizeof(rr_material) +
         sizeof(rr_batch_config) + (size_t)n_tab * (4 + (size_t)rr::kLobeSamples * 4);
}

int rr_scene_save(const rr_scene* s, void* blob, uint64_t capacity, uint64_t* size) {
  if (!s || !size) return fail(RR_ERR_INVALID_ARG, "scene and size must not be NULL");
  if (int rc = check_device(s, "rr_scene_save")) return rc;
  uint32_t n_tab = 0;
  for (uint32_t m = 0; m < s->nm; ++m) n_tab += s->lobe_kind[m] == rr::kLobeTable ? 1u : 0u;
  const size_t payload = blob_payload_bytes(s->nv, s->nt, s->nm, n_tab);
  *size = sizeof(SceneBlobHeader) + payload;
  if (!blob) return RR_OK;
  if (capacity < *size) return fail(RR_ERR_INVALID_ARG, "the blob needs " + std::to_string(*size) + " bytes");
  RR_CHECK_CUDA(cudaStreamSynchronize(t_stream), "synchronising");
  unsigned char* b = static_cast<unsigned char*>(blob) + sizeof(SceneBlobHeader);
  unsigned char* q = b;
  auto d2h = [&](const void* src, size_t n) -> cudaError_t {
    cudaError_t e = n ? cudaMemcpy(q, src, n, cudaMemcpyDeviceToHost) : cudaSuccess;
    q += n;
    return e;
  };
  RR_CHECK_CUDA(d2h(s->d_vtx, (size_t)s->nv * 12), "saving the vertices");
  RR_CHECK_CUDA(d2h(s->d_idx, (size_t)s->nt * 12), "saving the triangles");
  RR_CHECK_CUDA(d2h(s->d_mat_id, (size_t)s->nt * 2), "saving the material ids");
  for (size_t pad = (((size_t)s->nt * 2 + 3) & ~(size_t)3) - (size_t)s->nt * 2; pad; --pad) *q++ = 0;
  RR_CHECK_CUDA(d2h(s->d_raw_mats, (size_t)s->nm * sizeof(rr_material)), "saving the materials");
  rr_batch_config cfg;
  if (int rc = rr_batch_config_get(s, &cfg)) return rc;
  memcpy(q, &cfg, sizeof cfg);
  q += sizeof cfg;
  for (uint32_t m = 0; m < s->nm; ++m) {
    if (s->lobe_kind[m] != rr::kLobeTable) continue;
    memcpy(q, &m, 4);
    q += 4;
    RR_CHECK_CUDA(d2h(s->d_lobe_samples + (size_t)m * rr::kLobeSamples, (size_t)rr::kLobeSamples * 4),
                  "saving a tabulated lobe");
  }
  SceneBlobHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kBlobMagic, 8);
  h.version = kBlobVersion;
  h.nv = s->nv;
  h.nt = s->nt;
  h.nm = s->nm;
  h.n_tab = n_tab;
  h.payload_bytes = payload;
  h.checksum = fnv1a(b, payload);
  memcpy(blob, &h, sizeof h);
  return RR_OK;
}

int rr_scene_load(const void* blob, uint64_t size, rr_scene** out) {
  if (!blob || !out) return fail(RR_ERR_INVALID_ARG, "blob and out must not be NULL");
  if (size < sizeof(SceneBlobHeader)) return fail(RR_ERR_INVALID_ARG, "the blob is truncated (no header)");
  SceneBlobHeader h;
  memcpy(&h, blob, sizeof h);
  if (memcmp(h.magic, kBlobMagic, 8) != 0) return fail(RR_ERR_INVALID_ARG, "not a scene blob");
  if (h.version != kBlobVersion)
    return fail(RR_ERR_INVALID_ARG, "scene blob format " + std::to_string(h.version) + ", this library reads " +
                                        std::to_string(kBlobVersion));
  if (h.nm == 0 || h.nm > RR_MAX_MATERIALS || h.n_tab > h.nm || h.nt > (1u << 30))
    return fail(RR_ERR_INVALID_ARG, "the blob header is inconsistent");
  const size_t payload = blob_payload_bytes(h.nv, h.nt, h.nm, h.n_tab);
  if (h.payload_bytes != payload || size < sizeof(SceneBlobHeader) + payload)
    return fail(RR_ERR_INVALID_ARG, "the blob is truncated or its sizes disagree");
  const unsigned char* b = static_cast<const unsigned char*>(blob) + sizeof(SceneBlobHeader);
  if (fnv1a(b, payload) != h.checksum) return fail(RR_ERR_INVALID_ARG, "the blob is corrupted (checksum)");
  // copies of the arrays: the payload has no alignment guarantee beyond bytes
  std::vector<float> vtx((size_t)h.nv * 3);
  std::vector<uint32_t> tri((size_t)h.nt * 3);
  std::vector<uint16_t> mid(h.nt);
  std::vector<rr_material> mats(h.nm);
  const unsigned char* q = b;
  memcpy(vtx.data(), q, vtx.size() * 4);
  q += vtx.size() * 4;
  memcpy(tri.data(), q, tri.size() * 4);
  q += tri.size() * 4;
  memcpy(mid.data(), q, mid.size() * 2);
  q += ((size_t)h.nt * 2 + 3) & ~(size_t)3;
  memcpy(mats.data(), q, mats.size() * sizeof(rr_material));
  q += mats.size() * sizeof(rr_material);
  rr_batch_config cfg;
  memcpy(&cfg, q, sizeof cfg);
  q += sizeof cfg;
  rr_scene* s = nullptr;
  int rc = rr_scene_create(vtx.data(), h.nv, tri.data(), h.nt, mid.data(), mats.data(), h.nm, &s);
  if (rc != RR_OK) return rc;
  std::vector<float> dens(rr::kLobeSamples);
  for (uint32_t k = 0; k < h.n_tab && rc == RR_OK; ++k) {
    uint32_t m = 0;
    memcpy(&m, q, 4);
    memcpy(dens.data(), q + 4, dens.size() * 4);
    q += 4 + dens.size() * 4;
    rc = rr_scene_set_lobe(s, m, dens.data());
  }
  if (rc == RR_OK) rc = rr_batch_config_set(s, &cfg);   // rebuilds when the saved BVH build differs
  if (rc == RR_OK) {
    cudaError_t e = cudaStreamSynchronize(t_stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "loading the scene");
  }
  if (rc != RR_OK) {
    const std::string msg = rr_last_error();
    rr_scene_destroy(s);
    return fail(rc, msg);
  }
  *out = s;
  return RR_OK;
}

int rr_scene_export_wide(rr_scene* s, void* nodes, uint32_t cap, uint32_t* n_nodes, float* tris) {
  if (!s) return fail(RR_ERR_INVALID_ARG, "scene must not be NULL");
  if (int rc = check_device(s, "rr_scene_export_wide")) return rc;
  if (s->nt && s->wide_stale) RR_CHECK_CUDA(build_wide(s, t_stream), "collapsing the wide BVH");
  RR_CHECK_CUDA(cudaStreamSynchronize(t_stream), "synchronising");
  uint32_t wctr[8] = {0};
  if (s->nt) RR_CHECK_CUDA(cudaMemcpy(wctr, s->d_wctr, sizeof wctr, cudaMemcpyDeviceToHost), "export");
  if (wctr[4]) return fail(RR_ERR_CUDA, "the wide BVH build failed");
  if (n_nodes) *n_nodes = wctr[1];
  const size_t nn = std::min<size_t>(wctr[1], cap);
  if (nodes && nn)
    RR_CHECK_CUDA(cudaMemcpy(nodes, s->d_wnodes, nn * rr::kWideNodeWords * sizeof(float4), cudaMemcpyDeviceToHost),
                  "export");
  if (tris && s->nt)
    RR_CHECK_CUDA(cudaMemcpy(tris, s->d_wtri, (size_t)s->nt * 3 * sizeof(float4), cudaMemcpyDeviceToHost), "export");
  return RR_OK;
}

int rr_scan_async(rr_scene* s, const rr_pose* pose, const rr_sensor_params* p, float* out_polar) {
  if (!s || !out_polar) return fail(RR_ERR_INVALID_ARG, "scene and out_polar must not be NULL");
  int rc = check_params(pose, p);
  if (rc != RR_OK) return rc;
  if ((rc = check_device(s, "rr_scan_async")) != RR_OK) return rc;
  if (!is_device_ptr(out_polar)) return fail(RR_ERR_INVALID_ARG, "rr_scan_async needs a device output");
  return scan_split(s, pose, p, out_polar, t_stream, true);
}

int rr_scene_sync(rr_scene* s) {
  if (!s) return fail(RR_ERR_INVALID_ARG, "scene must not be NULL");
  return scene_status(s, t_stream);
}

int rr_scan(rr_scene* s, const rr_pose* pose, const rr_sensor_params* p, float* out_polar) {
  if (!s || !out_polar) return fail(RR_ERR_INVALID_ARG, "scene and out_polar must not be NULL");
  int rc = check_params(pose, p);
  if (rc != RR_OK) return rc;
  if ((rc = check_device(s, "rr_scan")) != RR_OK) return rc;
  cudaStream_t st = t_stream;
  const size_t img_bytes = (size_t)p->n_azimuth * p->n_bins * sizeof(float);
  const bool dev = is_device_ptr(out_polar);
  float* target = out_polar;
  if (!dev) {
    rc = ensure_image(&s->main, img_bytes, st);
    if (rc != RR_OK) return rc;
    target = s->main.d_image;
  }
  rc = scan_split(s, pose, p, target, st, true);
  if (rc != RR_OK) return rc;
  if (!dev)
    RR_CHECK_CUDA(cudaMemcpyAsync(out_polar, target, img_bytes, cudaMemcpyDeviceToHost, st), "copying the image");
  return scene_status(s, st);
}

int rr_scan_debug(rr_scene* s, const rr_pose* pose, const rr_sensor_params* p, const uint8_t* ray_mask,
                  float* out_polar, rr_segment* segs, uint64_t seg_capacity, uint64_t* n_segs, float* ray_tallies) {
  if (!s || !out_polar) return fail(RR_ERR_INVALID_ARG, "scene and out_polar must not be NULL");
  int rc = check_params(pose, p);
  if (rc != RR_OK) return rc;
  if ((rc = check_device(s, "rr_scan_debug")) != RR_OK) return rc;
  cudaStream_t st = t_stream;
  const size_t n0 = (size_t)p->n_azimuth * p->rays_per_beam;
  const size_t img_bytes = (size_t)p->n_azimuth * p->n_bins * sizeof(float);
  if (seg_capacity > 0xFFFFFFFFull) seg_capacity = 0xFFFFFFFFull;
  // temporaries of the debug path (allocated per call)
  float* d_img = nullptr;
  rr_segment* d_segs = nullptr;
  float* d_tal = nullptr;
  uint8_t* d_mask = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(d_img);
    cudaFree(d_segs);
    cudaFree(d_tal);
    cudaFree(d_mask);
  };
  auto check = [&](cudaError_t e, const char* what) -> int {
    if (e == cudaSuccess) return RR_OK;
    cudaGetLastError();
    cleanup();
    return cuda_fail(e, what);
  };
  if ((rc = check(dev_malloc(&d_img, img_bytes), "debug image")) != RR_OK) return rc;
  if (segs && seg_capacity)
    if ((rc = check(dev_malloc(&d_segs, seg_capacity * sizeof(rr_segment)), "debug segments")) != RR_OK) return rc;
  if (ray_tallies) {
    if ((rc = check(dev_malloc(&d_tal, n0 * 4 * sizeof(float)), "debug tallies")) != RR_OK) return rc;
    if ((rc = check(cudaMemsetAsync(d_tal, 0, n0 * 4 * sizeof(float), st), "debug tallies")) != RR_OK) return rc;
  }
  if (ray_mask) {
    if ((rc = check(dev_malloc(&d_mask, n0), "debug mask")) != RR_OK) return rc;
    if ((rc = check(cudaMemcpyAsync(d_mask, ray_mask, n0, cudaMemcpyDefault, st), "debug mask")) != RR_OK) return rc;
  }
  DebugOut dbg;
  dbg.segs = d_segs;
  dbg.seg_cap = d_segs ? (uint32_t)seg_capacity : 0u;
  dbg.tallies = d_tal;
  dbg.mask = d_mask;
  float* const images[1] = {d_img};
  rc = batch_run(s, &s->main, pose, p, images, 1, &dbg, st, s->cfg);
  if (rc != RR_OK) {
    cleanup();
    return rc;
  }
  rc = device_status(&s->main, st);
  const uint64_t total = s->main.h_ctr->seg_start[p->max_bounces];
  if (n_segs) *n_segs = total;
  if (rc == RR_OK || rc == RR_ERR_CAPACITY) {
    int rc2;
    if ((rc2 = check(cudaMemcpyAsync(out_polar, d_img, img_bytes, cudaMemcpyDefault, st), "copy")) != RR_OK)
      return rc2;
    if (d_segs) {
      const uint64_t nw = total < seg_capacity ? total : seg_capacity;
      if ((rc2 = check(cudaMemcpyAsync(segs, d_segs, nw * sizeof(rr_segment), cudaMemcpyDefault, st), "copy")) !=
          RR_OK)
        return rc2;
    }
    if (d_tal)
      if ((rc2 = check(cudaMemcpyAsync(ray_tallies, d_tal, n0 * 4 * sizeof(float), cudaMemcpyDefault, st),
                       "copy")) != RR_OK)
        return rc2;
  }
  cleanup();
  if (rc == RR_OK && segs && total > seg_capacity) return fail(RR_ERR_CAPACITY, "segment buffer too small");
  return rc;
}

int rr_polar_to_db_u8(const float* polar, uint64_t n, float cutoff_db, uint8_t* out) {
  if (!polar || !out) return fail(RR_ERR_INVALID_ARG, "NULL buffer");
  if (!(cutoff_db > 0.f) || !std::isfinite(cutoff_db)) return fail(RR_ERR_INVALID_ARG, "cutoff_db must be > 0");
  if (!is_device_ptr(polar) || !is_device_ptr(out)) return fail(RR_ERR_INVALID_ARG, "buffers must be device memory");
  RR_CHECK_CUDA(launch_db_u8(polar, n, cutoff_db, out, t_stream), "dB map launch");
  return RR_OK;
}

int rr_scene_stats(rr_scene* s, rr_stats* out, int reset) {
  if (!s || !out) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = t_stream;
  memset(out, 0, sizeof *out);
  // the scene's own context and the lanes of split scans (joined into st)
  std::vector<ExecCtx*> xs = {&s->main};
  for (uint32_t k = 0; k < s->split_used; ++k) xs.push_back(&s->split[k].ctx);
  RR_CHECK_CUDA(cudaStreamSynchronize(st), "stats");
  for (ExecCtx* x : xs) {
    RR_CHECK_CUDA(cudaMemcpy(x->h_ctr, x->d_ctr, sizeof(ScanCounters), cudaMemcpyDeviceToHost), "stats");
    out->closest_queries += x->h_ctr->stat_closest;
    out->anyhit_queries += x->h_ctr->stat_anyhit;
    out->returns += x->h_ctr->stat_returns;
    out->nodes_visited += x->h_ctr->stat_nodes;
    out->tris_tested += x->h_ctr->stat_tris;
    out->anyhit_nodes_visited += x->h_ctr->stat_nodes_any;
    out->anyhit_tris_tested += x->h_ctr->stat_tris_any;
  }
  out->scans = s->main.h_ctr->stat_scans;   // a split scan counts once (its first range)
  out->kernel_launches = s->launches;
  if (reset) {
    s->launches = 0;
    for (ExecCtx* x : xs)
      RR_CHECK_CUDA(cudaMemset(&x->d_ctr->stat_closest, 0, 8 * sizeof(unsigned long long)), "stats reset");
  }
  return RR_OK;
}

int rr_profile_enable(rr_scene* s, int on) {
  if (!s) return fail(RR_ERR_INVALID_ARG, "NULL scene");
  if (on && !s->prof) {
    // a new time origin: fold the intervals measured against the old one
    prof_collect(s);
    for (int k = 0; k < RR_K_COUNT; ++k) {
      s->prof_busy_done[k] += prof_union(s->prof_iv[k]);
      s->prof_iv[k].clear();
    }
    if (!s->prof_base) RR_CHECK_CUDA(cudaEventCreate(&s->prof_base), "profile event");
    RR_CHECK_CUDA(cudaEventRecord(s->prof_base, t_stream), "profile event");
  }
  s->prof = on != 0;
  return RR_OK;
}

int rr_profile_read(rr_scene* s, rr_profile* out, int reset) {
  if (!s || !out) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  prof_collect(s);
  for (int k = 0; k < RR_K_COUNT; ++k) {
    out->ms[k] = s->prof_ms[k];
    out->launches[k] = s->prof_launches[k];
    out->busy_ms[k] = s->prof_busy_done[k] + prof_union(s->prof_iv[k]);
    if (reset) {
      s->prof_ms[k] = 0.0;
      s->prof_launches[k] = 0;
      s->prof_busy_done[k] = 0.0;
      s->prof_iv[k].clear();
    }
  }
  return RR_OK;
}

}  // extern "C"

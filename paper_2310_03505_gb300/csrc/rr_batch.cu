// rr_batch.cu -- batches of scans: planning, descriptors, launch sequences,
// CUDA graphs and the launch autotuner.
//
// A request of n scans (poses and sensor models of one scene, uneven ray
// counts and bounce limits allowed) is cut into launch sequences ("groups"):
// consecutive scans whose worst-case ray tree fits the workspace limit and the
// key ranges of the device records.  Each group is one fixed sequence of
// persistent kernels over all its scans' rays:
//   raygen, { trace, shade } x (largest bounce limit), bin columns, [pattern]
// Its per-scan constants travel as a descriptor table uploaded ahead of the
// kernels, so the kernels' own arguments depend only on the workspace and the
// group's shape; a captured CUDA graph of the sequence is replayed as long as
// they stay the same.  Single scans are groups of one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rr_host.h"

using rr::ScanArgs;
using rr::ScanDesc;

namespace rr_host {

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// running worst-case sizes of a set of scans
struct Need {
  uint64_t n0 = 0;     // initial rays
  uint64_t q = 0;      // largest queue: sum of n0 * 2^(bounces - 1)
  uint64_t r = 0;      // return records: sum of 2 n0 (2^bounces - 1)
  uint64_t tmp = 0;    // floats of the images before the azimuth pattern
  uint64_t n = 0;      // scans
  bool order = false;  // room for the closest-hit query order (rr_batch_config.query_order)
  // a scan of n_az columns (all azimuths of p, or a range of them)
  void add(const rr_sensor_params& p, uint32_t n_az) {
    const uint64_t s0 = (uint64_t)n_az * p.rays_per_beam;
    n0 += s0;
    q += s0 << (p.max_bounces - 1);
    r += 2ull * s0 * ((1ull << p.max_bounces) - 1ull);
    if (p.az_pattern_sigma > 0.f) tmp += (uint64_t)p.n_azimuth * p.n_bins;
    n += 1;
  }
  void add(const rr_sensor_params& p) { add(p, p.n_azimuth); }
};

static size_t desc_bytes(uint64_t n) { return (size_t)n * sizeof(ScanDesc) + 2 * (size_t)(n + 1) * sizeof(uint32_t); }

static uint64_t order_bytes(uint64_t q, const Need& nd) {
  return nd.order ? align256(q * 2) + align256(q * 4) +
                        align256((RR_MAX_BOUNCES + 1) * (uint64_t)rr::kOrderBuckets * 4) +
                        align256((uint64_t)rr::kOrderBuckets * 4)
                  : 0;
}

static uint64_t bytes_of(uint64_t q, uint64_t r, const Need& nd) {
  const uint64_t tiles = (q + 255) / 256 + 1;
  return align256(q * sizeof(rr::RayRec)) * 2 + align256(q * sizeof(rr::HitRec)) + align256(q * 4) + align256(r * 8) +
         align256(tiles * 8) + align256(nd.tmp * 4) + align256(desc_bytes(nd.n)) + order_bytes(q, nd);
}

static WsLayout layout_of(const Need& nd, uint64_t limit) {
  const uint64_t cap30 = 1ull << 30;
  uint64_t q = std::min(nd.q, cap30), r = std::min(nd.r, cap30 << 1);
  if (q < nd.n0) q = nd.n0;
  WsLayout L;
  L.clamped = false;
  if (bytes_of(q, r, nd) > limit) {
    // scale the queues and records; the parts that do not grow with them stay
    const double fixed = (double)bytes_of(0, 0, nd);
    const double f = std::max(0.0, (double)limit - fixed) / std::max(1.0, (double)bytes_of(q, r, nd) - fixed);
    q = std::max<uint64_t>(nd.n0, (uint64_t)(q * f));
    r = std::max<uint64_t>(2 * nd.n0, (uint64_t)(r * f));
    L.clamped = true;
  }
  L.ray_cap = (uint32_t)q;
  L.rec_cap = (uint32_t)std::min<uint64_t>(r, 0xFFFFFFFFull);
  L.tiles = (uint32_t)((q + 255) / 256 + 1);
  L.n_desc = (uint32_t)nd.n;
  L.tmp_floats = nd.tmp;
  size_t off = 0;
  L.off_rays0 = off;
  off += align256((size_t)q * sizeof(rr::RayRec));
  L.off_rays1 = off;
  off += align256((size_t)q * sizeof(rr::RayRec));
  L.off_hits = off;
  off += align256((size_t)q * sizeof(rr::HitRec));
  L.off_vis = off;   // deferred visibility: the candidates of a bounce
  off += align256((size_t)q * 4);
  L.off_recs = off;
  off += align256((size_t)L.rec_cap * 8);
  L.off_status = off;
  off += align256((size_t)L.tiles * 8);
  L.off_tmp = off;
  off += align256((size_t)nd.tmp * 4);
  L.off_desc = off;
  off += align256(desc_bytes(nd.n));
  // query order: keys, permutation, per-bounce bucket counts, bucket cursors
  L.off_order = off;
  L.order = nd.order;
  off += order_bytes(q, nd);
  L.total = off;
  return L;
}

WsLayout plan_workspace(const rr_sensor_params* ps, uint32_t n, uint64_t limit, const uint32_t* az_count,
                        bool order) {
  Need nd;
  nd.order = order;
  for (uint32_t i = 0; i < n; ++i) nd.add(ps[i], az_count ? az_count[i] : ps[i].n_azimuth);
  return layout_of(nd, limit);
}

WsLayout plan_workspace_caps(const rr_sensor_params* ps, uint32_t n, uint64_t q_cap, uint64_t r_cap, bool order) {
  Need nd;
  nd.order = order;
  for (uint32_t i = 0; i < n; ++i) nd.add(ps[i]);
  Need e = nd;
  e.q = std::min(nd.q, std::max(q_cap, nd.n0));
  e.r = std::min(nd.r, std::max(r_cap, 2 * nd.n0));
  WsLayout L = layout_of(e, ~uint64_t(0));
  L.clamped = e.q < nd.q || e.r < nd.r;
  return L;
}

std::vector<Group> plan_groups(const rr_sensor_params* ps, uint32_t n, const LaunchCfg& cfg) {
  std::vector<Group> out;
  uint32_t i = 0;
  while (i < n) {
    Need nd;
    nd.order = cfg.order == RR_ORDER_CELL_OCTANT;
    uint64_t cols = 0;
    uint32_t j = i;
    while (j < n) {
      if (j > i) {
        Need t = nd;
        t.add(ps[j]);
        if (j - i >= rr::kMaxBatchScans || cols + ps[j].n_azimuth > rr::kMaxColumns || t.n0 > (1ull << 30) ||
            t.tmp >= 0xFFFFFFFFull || (cfg.wavefront_rays && t.n0 > cfg.wavefront_rays) ||
            layout_of(t, cfg.ws_limit).clamped)
          break;
      }
      nd.add(ps[j]);
      cols += ps[j].n_azimuth;
      ++j;
    }
    Group g;
    g.first = i;
    g.count = j - i;
    g.L = layout_of(nd, cfg.ws_limit);
    out.push_back(g);
    i = j;
  }
  return out;
}

int ensure_workspace(ExecCtx* x, size_t bytes, cudaStream_t st) {
  if (x->ws_bytes >= bytes) return RR_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "synchronising before growing the workspace");
  }
  if (x->ws) cudaFree(x->ws);
  x->ws = nullptr;
  x->ws_bytes = 0;
  x->gkey.clear();   // a captured graph points into the old workspace
  e = dev_malloc(&x->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "allocating the scan workspace");
  }
  x->ws_bytes = bytes;
  return RR_OK;
}

int ensure_image(ExecCtx* x, size_t bytes, cudaStream_t st) {
  if (x->image_bytes >= bytes) return RR_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "synchronising before growing the image buffer");
  }
  if (x->d_image) cudaFree(x->d_image);
  x->d_image = nullptr;
  x->image_bytes = 0;
  e = dev_malloc(&x->d_image, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "allocating the image buffer");
  }
  x->image_bytes = bytes;
  return RR_OK;
}

// pinned staging for the descriptors; waits until the previous upload from
// it has been read by the device
static int stage_acquire(ExecCtx* x, size_t bytes) {
  if (x->stage_used) {
    cudaError_t e = cudaEventSynchronize(x->stage_ev);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "waiting for the descriptor staging");
    }
    x->stage_used = false;
  }
  if (!x->stage_ev) {
    cudaError_t e = cudaEventCreateWithFlags(&x->stage_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "creating the staging event");
    }
  }
  if (x->stage_bytes < bytes) {
    if (x->h_stage) cudaFreeHost(x->h_stage);
    x->h_stage = nullptr;
    x->stage_bytes = 0;
    const size_t want = std::max<size_t>(bytes, 4096);
    cudaError_t e = host_malloc(&x->h_stage, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "allocating the descriptor staging");
    }
    x->stage_bytes = want;
  }
  return RR_OK;
}

// descriptor of one scan (the same float arithmetic for every entry point)
static void fill_desc(ScanDesc& d, const rr_pose& pose, const rr_sensor_params& p, float* image, uint32_t ray0,
                      uint32_t col0, uint32_t tmp0, uint32_t az_begin) {
  memset(&d, 0, sizeof d);
  const float qn = 1.0f / std::sqrt(pose.q[0] * pose.q[0] + pose.q[1] * pose.q[1] + pose.q[2] * pose.q[2] +
                                    pose.q[3] * pose.q[3]);
  const float r_max = (float)p.n_bins * p.bin_size_m;
  d.pos_rmax = make_float4(pose.p[0], pose.p[1], pose.p[2], r_max);
  d.quat = make_float4(pose.q[0] * qn, pose.q[1] * qn, pose.q[2] * qn, pose.q[3] * qn);
  d.dims = make_uint4(p.n_azimuth, p.rays_per_beam, p.max_bounces, p.n_bins);
  d.beam = make_float4(p.beam_width_rad, p.beam_prob, p.elevation_rad, p.bin_size_m);
  d.phys = make_float4(p.t_min_m, p.min_energy, p.freq_hz, (p.flags & RR_MULTIPATH) ? 2.0f * r_max : r_max);
  d.post = make_float4(p.blur_sigma_bins, p.az_pattern_sigma, p.noise_sys, p.noise_amb);
  d.rng = make_uint4((uint32_t)(p.seed & 0xFFFFFFFFu), (uint32_t)(p.seed >> 32), p.scan_id, p.flags);
  d.offs = make_uint4(ray0, col0, tmp0, az_begin);
  d.ext = make_float4(p.beam_aspect > 0.f ? p.beam_aspect : 1.0f, p.noise_cell_az > 0.f ? p.noise_cell_az : 8.0f,
                      p.noise_cell_bins > 0.f ? p.noise_cell_bins : 32.0f, p.range_falloff);
  d.image = image;
}

// the side stream and events of deferred visibility (made outside any capture)
static cudaError_t ensure_side(ExecCtx* x) {
  if (x->side_ready) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (!x->side) e = cudaStreamCreateWithFlags(&x->side, cudaStreamNonBlocking);
  for (int b = 0; b < RR_MAX_BOUNCES && e == cudaSuccess; ++b) {
    if (!x->fork[b]) e = cudaEventCreateWithFlags(&x->fork[b], cudaEventDisableTiming);
    if (e == cudaSuccess && !x->join[b]) e = cudaEventCreateWithFlags(&x->join[b], cudaEventDisableTiming);
  }
  x->side_ready = e == cudaSuccess;
  return e;
}

// the kernels of one launch sequence on stream st (with deferred visibility,
// each bounce's visibility queries on x->side, overlapping the next bounce's
// closest-hit queries; the next shading pass waits for them)
static cudaError_t launch_sequence(rr_scene* s, ExecCtx* x, const ScanArgs& a, bool pattern, const LaunchCfg& cfg,
                                   bool profile, cudaStream_t st) {
  cudaEvent_t ev;
  cudaError_t e;
  const bool overlap = a.defer_vis && x->side_ready;
  int pending = -1;   // bounce whose visibility queries run on the side stream
  if (profile) prof_begin(s, RR_K_RAYGEN, st, &ev);
  if ((e = launch_raygen(a, st)) != cudaSuccess) return e;
  if (profile) prof_end(s, ev, st);
  const bool vis = (a.any_flags & RR_MULTIPATH) != 0u;
  for (uint32_t b = 0; b < a.max_bounces; ++b) {
    if (profile) prof_begin(s, RR_K_TRACE, st, &ev);
    if ((e = launch_query(a, b, false, cfg, st)) != cudaSuccess) return e;
    if (profile) prof_end(s, ev, st);
    if (b >= 1 && vis && !a.defer_vis) {   // air-path visibility (Sec. III-A) from bounce 1 on
      if (profile) prof_begin(s, RR_K_VIS, st, &ev);
      if ((e = launch_vis_prep(a, b, st)) != cudaSuccess) return e;
      if ((e = launch_query(a, b, true, cfg, st)) != cudaSuccess) return e;
      if (profile) prof_end(s, ev, st);
    }
    if (pending >= 0) {
      if ((e = cudaStreamWaitEvent(st, x->join[pending], 0)) != cudaSuccess) return e;
      pending = -1;
    }
    if (profile) prof_begin(s, RR_K_SHADE, st, &ev);
    if ((e = launch_shade(a, b, st)) != cudaSuccess) return e;
    if (a.order_perm && b + 1 < a.max_bounces && (e = launch_order(a, b + 1, st)) != cudaSuccess) return e;
    if (profile) prof_end(s, ev, st);
    if (b >= 1 && vis && a.defer_vis) {   // the candidates the shading pass listed, settled when visible
      cudaStream_t sv = st;
      if (overlap) {
        if ((e = cudaEventRecord(x->fork[b], st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(x->side, x->fork[b], 0)) != cudaSuccess) return e;
        sv = x->side;
      }
      if (profile) prof_begin(s, RR_K_VIS, sv, &ev);
      if ((e = launch_query(a, b, true, cfg, sv)) != cudaSuccess) return e;
      if (profile) prof_end(s, ev, sv);
      if (overlap) {
        if ((e = cudaEventRecord(x->join[b], x->side)) != cudaSuccess) return e;
        pending = (int)b;
      }
    }
  }
  if (pending >= 0 && (e = cudaStreamWaitEvent(st, x->join[pending], 0)) != cudaSuccess) return e;
  if (profile) prof_begin(s, RR_K_IMAGE, st, &ev);
  if ((e = launch_image(a, pattern, st)) != cudaSuccess) return e;
  if (profile) prof_end(s, ev, st);
  return cudaSuccess;
}

// replay (capturing first when the arguments changed) the launch sequence
static int graph_launch(rr_scene* s, ExecCtx* x, const ScanArgs& a, bool pattern, const LaunchCfg& cfg,
                        cudaStream_t st) {
  std::vector<unsigned char> key(sizeof(ScanArgs) + 4 * sizeof(uint32_t));
  memcpy(key.data(), &a, sizeof(ScanArgs));
  const uint32_t extra[4] = {pattern ? 1u : 0u, cfg.trace_block, cfg.trace_blocks_per_sm, cfg.refill};
  memcpy(key.data() + sizeof(ScanArgs), extra, sizeof extra);
  if (!(x->gexec && key == x->gkey)) {
    if (!x->cap_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&x->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "creating the capture stream");
      }
    }
    // one-time attribute and occupancy queries stay outside the capture
    num_sms();
    init_image_attrs();
    cudaError_t e = cudaStreamBeginCapture(x->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "beginning the graph capture");
    }
    const cudaError_t le = launch_sequence(s, x, a, pattern, cfg, false, x->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(x->cap_stream, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return cuda_fail(le != cudaSuccess ? le : e, "capturing the launch sequence");
    }
    if (x->gexec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(x->gexec, g, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(x->gexec);
        x->gexec = nullptr;
      }
    }
    if (!x->gexec) {
      e = cudaGraphInstantiate(&x->gexec, g, 0);
      if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        x->gexec = nullptr;
        x->gkey.clear();
        return cuda_fail(e, "instantiating the launch graph");
      }
    }
    cudaGraphDestroy(g);
    x->gkey = key;
  }
  cudaError_t e = cudaGraphLaunch(x->gexec, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "launching the graph");
  }
  return RR_OK;
}

int batch_enqueue(rr_scene* s, ExecCtx* x, const rr_pose* poses, const rr_sensor_params* ps, float* const* images,
                  uint32_t n, const DebugOut* dbg, cudaStream_t st, void* ws, const WsLayout& L, bool profile,
                  bool allow_graph, const LaunchCfg& cfg, void* host_desc, const uint32_t* az_range) {
  if (n == 0) return RR_OK;
  if (n != L.n_desc) return fail(RR_ERR_INVALID_ARG, "internal: layout planned for another batch");
  char* w = (char*)ws;
  const size_t dbytes = desc_bytes(n);
  void* hd = host_desc;
  if (!hd) {
    const int rc = stage_acquire(x, dbytes);
    if (rc != RR_OK) return rc;
    hd = x->h_stage;
  }
  ScanDesc* D = (ScanDesc*)hd;
  uint32_t* R0 = (uint32_t*)(D + n);
  uint32_t* C0 = R0 + (n + 1);
  uint32_t rays = 0, cols = 0, maxb = 0, maxbins = 0, any_flags = 0;
  uint64_t tmp = 0;
  bool pattern = false, min_energy = false;
  for (uint32_t i = 0; i < n; ++i) {
    const rr_sensor_params& p = ps[i];
    const bool pat = p.az_pattern_sigma > 0.f;
    const uint32_t az0 = az_range ? az_range[2 * i] : 0u, naz = az_range ? az_range[2 * i + 1] : p.n_azimuth;
    fill_desc(D[i], poses[i], p, images[i], rays, cols, pat ? (uint32_t)tmp : rr::kNone, az0);
    R0[i] = rays;
    C0[i] = cols;
    rays += naz * p.rays_per_beam;
    cols += naz;
    if (pat) tmp += (uint64_t)p.n_azimuth * p.n_bins;
    maxb = std::max(maxb, p.max_bounces);
    maxbins = std::max(maxbins, p.n_bins);
    any_flags |= p.flags;
    pattern = pattern || pat;
    min_energy = min_energy || p.min_energy > 0.f;
  }
  R0[n] = rays;
  C0[n] = cols;
  if (tmp > L.tmp_floats) return fail(RR_ERR_INVALID_ARG, "internal: pattern buffer planned too small");
  cudaError_t e = cudaMemcpyAsync(w + L.off_desc, hd, dbytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !host_desc) {
    e = cudaEventRecord(x->stage_ev, st);
    x->stage_used = e == cudaSuccess;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "uploading the scan descriptors");
  }

  ScanArgs a;
  memset(&a, 0, sizeof a);
  const bool wide = cfg.node_format == RR_NODES_WIDE8 && s->nt > 0;
  if (wide) {
    // collapse the 8-wide BVH on first use after a build; streams other than
    // the one that collapsed it wait for it
    std::lock_guard<std::mutex> guard(s->lock);
    if (s->wide_stale) {
      cudaEvent_t ev;
      const bool prof = profile && s->prof;
      if (prof) prof_begin(s, RR_K_BUILD, st, &ev);
      e = build_wide(s, st);
      if (prof) prof_end(s, ev, st);
      if (e == cudaSuccess && !s->wide_ready) e = cudaEventCreateWithFlags(&s->wide_ready, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(s->wide_ready, st);
    } else if (s->wide_ready) {
      e = cudaStreamWaitEvent(st, s->wide_ready, 0);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "collapsing the wide BVH");
    }
  }
  a.tri = wide ? s->d_wtri : s->d_tri;
  a.tri_copy = 3 * (size_t)s->nt;
  a.nodes = wide ? s->d_wnodes : s->d_nodes;
  a.mats = s->d_mats;
  a.lut = s->d_lut;
  a.n_tris = s->nt;
  a.n_mats = s->nm;
  a.wide = wide ? 1u : 0u;
  a.node_cap = wide ? s->wcap : (s->nt > 1 ? s->nt - 1 : 0u);
  a.bvh_status = wide ? s->d_wctr + 4 : nullptr;
  a.build_status = s->d_misc + 6;
  a.desc = (const ScanDesc*)(w + L.off_desc);
  a.ray0 = (const uint32_t*)(w + L.off_desc + (size_t)n * sizeof(ScanDesc));
  a.col0 = a.ray0 + (n + 1);
  a.n_scans = n;
  a.n_rays0 = rays;
  a.n_cols = cols;
  a.max_bounces = maxb;
  a.max_bins = maxbins;
  a.any_flags = any_flags;
  // deferred visibility needs the children spawned whatever their air-path
  // return: with a min_energy cut the return decides, so the query runs first
  a.defer_vis = (any_flags & RR_MULTIPATH) && maxb > 1 && !min_energy ? 1u : 0u;
  a.vis_list = (uint32_t*)(w + L.off_vis);
  a.refill = cfg.refill;
  a.rays[0] = (rr::RayRec*)(w + L.off_rays0);
  a.rays[1] = (rr::RayRec*)(w + L.off_rays1);
  a.hits = (rr::HitRec*)(w + L.off_hits);
  a.recs = (uint2*)(w + L.off_recs);
  a.tile_status = (unsigned long long*)(w + L.off_status);
  a.ctr = x->d_ctr;
  a.image_tmp = pattern ? (float*)(w + L.off_tmp) : nullptr;
  if (cfg.order == RR_ORDER_CELL_OCTANT && L.order && maxb > 1) {
    char* o = w + L.off_order;
    a.order_key = (uint16_t*)o;
    o += align256((size_t)L.ray_cap * 2);
    a.order_perm = (uint32_t*)o;
    o += align256((size_t)L.ray_cap * 4);
    a.order_hist = (uint32_t*)o;
    o += align256((size_t)(RR_MAX_BOUNCES + 1) * rr::kOrderBuckets * 4);
    a.order_off = (uint32_t*)o;
  }
  a.ray_cap = L.ray_cap;
  a.rec_cap = L.rec_cap;
  if (dbg) {
    a.segs = dbg->segs;
    a.seg_cap = dbg->seg_cap;
    a.tallies = dbg->tallies;
    a.mask = dbg->mask;
  }
  s->launches += 2u + 2u * maxb + ((any_flags & RR_MULTIPATH) && maxb > 1 ? (a.defer_vis ? 1u : 2u) * (maxb - 1u) : 0u) +
                 (pattern ? 1u : 0u) + (a.order_perm ? 2u * (maxb - 1u) : 0u);
  // without its side stream, deferred visibility runs on the launch stream
  // (the allocation-free entry point, which stages its descriptors from the
  // caller's stack, never creates one)
  if (a.defer_vis && !x->side_ready && !host_desc && ensure_side(x) != cudaSuccess) cudaGetLastError();
  const bool prof = profile && s->prof;
  if (!prof && allow_graph && cfg.use_graph && !dbg) return graph_launch(s, x, a, pattern, cfg, st);
  e = launch_sequence(s, x, a, pattern, cfg, prof, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "scan launch");
  }
  return RR_OK;
}

int batch_run(rr_scene* s, ExecCtx* x, const rr_pose* poses, const rr_sensor_params* ps, float* const* images,
              uint32_t n, const DebugOut* dbg, cudaStream_t st, const LaunchCfg& cfg) {
  const std::vector<Group> groups = plan_groups(ps, n, cfg);
  if (dbg && groups.size() != 1) return fail(RR_ERR_INVALID_ARG, "internal: a debug scan is one group");
  size_t need = 0;
  for (const Group& g : groups) need = std::max(need, g.L.total);
  int rc = ensure_workspace(x, need, st);
  if (rc != RR_OK) return rc;
  for (const Group& g : groups) {
    rc = batch_enqueue(s, x, poses + g.first, ps + g.first, images + g.first, g.count, dbg, st, x->ws, g.L, true,
                       true, cfg, nullptr, nullptr);
    if (rc != RR_OK) return rc;
  }
  return RR_OK;
}

// One scan as split_streams azimuth ranges, each a launch sequence of its own
// on its own stream and execution context: the bounces of the ranges no
// longer wait for each other, so the tail of one range's bounce (its slowest
// queries) overlaps the others' work.  Forked from and joined back to st.
// Scans with a beam pattern (which needs every column) run whole.
int scan_split(rr_scene* s, const rr_pose* pose, const rr_sensor_params* p, float* image, cudaStream_t st,
               bool profile) {
  uint32_t k_n = std::min<uint32_t>(s->cfg.split, p->n_azimuth);
  if (k_n <= 1 || p->az_pattern_sigma > 0.f) {
    float* const images[1] = {image};
    return batch_run(s, &s->main, pose, p, images, 1, nullptr, st, s->cfg);
  }
  cudaError_t e = cudaSuccess;
  for (uint32_t k = 1; k < k_n; ++k) {
    SplitLane& ln = s->split[k - 1];
    if (!ln.stream) {
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ln.join, cudaEventDisableTiming);
      if (e == cudaSuccess) e = ctx_init(&ln.ctx, ln.stream);
    }
  }
  if (e == cudaSuccess && !s->fork) e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(s->fork, st);
  for (uint32_t k = 1; k < k_n && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(s->split[k - 1].stream, s->fork, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "forking the split scan");
  }
  s->split_used = std::max<uint32_t>(s->split_used, k_n - 1);
  for (uint32_t k = 0; k < k_n; ++k) {
    const uint32_t a0 = (uint32_t)((uint64_t)p->n_azimuth * k / k_n);
    const uint32_t a1 = (uint32_t)((uint64_t)p->n_azimuth * (k + 1) / k_n);
    const uint32_t range[2] = {a0, a1 - a0};
    ExecCtx* x = k == 0 ? &s->main : &s->split[k - 1].ctx;
    cudaStream_t sk = k == 0 ? st : s->split[k - 1].stream;
    const WsLayout L = plan_workspace(p, 1, s->cfg.ws_limit, &range[1], s->cfg.order == RR_ORDER_CELL_OCTANT);
    int rc = ensure_workspace(x, L.total, sk);
    if (rc != RR_OK) return rc;
    float* const images[1] = {image};
    rc = batch_enqueue(s, x, pose, p, images, 1, nullptr, sk, x->ws, L, profile, true, s->cfg, nullptr, range);
    if (rc != RR_OK) return rc;
  }
  for (uint32_t k = 1; k < k_n && e == cudaSuccess; ++k) {
    e = cudaEventRecord(s->split[k - 1].join, s->split[k - 1].stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->split[k - 1].join, 0);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "joining the split scan");
  }
  return RR_OK;
}

static int check_batch(rr_scene* s, uint32_t n, const rr_pose* poses, const rr_sensor_params* params,
                       float* const* out) {
  if (!s || (n && (!poses || !params || !out))) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  for (uint32_t i = 0; i < n; ++i) {
    const int rc = check_params(&poses[i], &params[i]);
    if (rc != RR_OK) return fail(rc, "scan " + std::to_string(i) + ": " + rr_last_error());
    if (!out[i]) return fail(RR_ERR_INVALID_ARG, "scan " + std::to_string(i) + ": NULL output");
  }
  return check_device(s, "rr_scan_batch");
}

static int cfg_check(const rr_batch_config* c) {
  if (c->trace_block != 64 && c->trace_block != 128 && c->trace_block != 256)
    return fail(RR_ERR_INVALID_ARG, "trace_block must be 64, 128 or 256");
  if (c->trace_blocks_per_sm > 64) return fail(RR_ERR_INVALID_ARG, "trace_blocks_per_sm must be <= 64");
  if (c->use_graph > 1) return fail(RR_ERR_INVALID_ARG, "use_graph must be 0 or 1");
  if (c->node_format != RR_NODES_WIDE8 && c->node_format != RR_NODES_BINARY)
    return fail(RR_ERR_INVALID_ARG, "node_format must be RR_NODES_WIDE8 or RR_NODES_BINARY");
  if (c->refill_threshold > 32) return fail(RR_ERR_INVALID_ARG, "refill_threshold must be in [0, 32]");
  if (c->split_streams > kMaxSplit) return fail(RR_ERR_INVALID_ARG, "split_streams must be in [0, 4]");
  if (c->workspace_limit != 0 && c->workspace_limit < (uint64_t(1) << 20))
    return fail(RR_ERR_INVALID_ARG, "workspace_limit must be 0 or at least 1 MiB");
  if (c->bvh_build != RR_BVH_LBVH && c->bvh_build != RR_BVH_SAH_TOP)
    return fail(RR_ERR_INVALID_ARG, "bvh_build must be RR_BVH_LBVH or RR_BVH_SAH_TOP");
  if (c->query_order > RR_ORDER_CELL_OCTANT)
    return fail(RR_ERR_INVALID_ARG, "query_order must be RR_ORDER_QUEUE or RR_ORDER_CELL_OCTANT");
  return RR_OK;
}

static void cfg_to_abi(const LaunchCfg& c, rr_batch_config* o) {
  memset(o, 0, sizeof *o);
  o->wavefront_rays = c.wavefront_rays;
  o->trace_block = c.trace_block;
  o->trace_blocks_per_sm = c.trace_blocks_per_sm;
  o->use_graph = c.use_graph;
  o->node_format = c.node_format;
  o->refill_threshold = c.refill;
  o->workspace_limit = c.ws_limit;
  o->split_streams = c.split;
  o->bvh_build = c.bvh_build;
  o->query_order = c.order;
}

static LaunchCfg cfg_from_abi(const rr_batch_config* c) {
  LaunchCfg o;
  o.wavefront_rays = c->wavefront_rays;
  o.trace_block = c->trace_block;
  o.trace_blocks_per_sm = c->trace_blocks_per_sm;
  o.use_graph = c->use_graph;
  o.node_format = c->node_format;
  o.refill = c->refill_threshold ? c->refill_threshold : 16u;
  if (c->workspace_limit) o.ws_limit = c->workspace_limit;
  o.split = c->split_streams ? c->split_streams : 3u;
  o.bvh_build = c->bvh_build;
  o.order = c->query_order;
  return o;
}

}  // namespace rr_host

using namespace rr_host;

extern "C" {

int rr_scan_batch(rr_scene* s, uint32_t n, const rr_pose* poses, const rr_sensor_params* params, float* const* out) {
  int rc = check_batch(s, n, poses, params, out);
  if (rc != RR_OK) return rc;
  cudaStream_t st = current_stream();
  const std::vector<Group> groups = plan_groups(params, n, s->cfg);
  size_t need = 0;
  for (const Group& g : groups) need = std::max(need, g.L.total);
  rc = ensure_workspace(&s->main, need, st);
  if (rc != RR_OK) return rc;
  std::vector<float*> images(n);
  std::vector<bool> on_dev(n);
  for (uint32_t i = 0; i < n; ++i) on_dev[i] = is_device_ptr(out[i]);
  for (const Group& g : groups) {
    // host outputs of the group land in the scene's image buffer first
    size_t host_bytes = 0;
    for (uint32_t i = g.first; i < g.first + g.count; ++i)
      if (!on_dev[i]) host_bytes += (size_t)params[i].n_azimuth * params[i].n_bins * sizeof(float);
    if (host_bytes) {
      rc = ensure_image(&s->main, host_bytes, st);
      if (rc != RR_OK) return rc;
    }
    size_t off = 0;
    for (uint32_t i = g.first; i < g.first + g.count; ++i) {
      if (on_dev[i]) {
        images[i] = out[i];
      } else {
        images[i] = s->main.d_image + off / sizeof(float);
        off += (size_t)params[i].n_azimuth * params[i].n_bins * sizeof(float);
      }
    }
    rc = batch_enqueue(s, &s->main, poses + g.first, params + g.first, images.data() + g.first, g.count, nullptr, st,
                       s->main.ws, g.L, true, true, s->cfg, nullptr, nullptr);
    if (rc != RR_OK) return rc;
    for (uint32_t i = g.first; i < g.first + g.count; ++i) {
      if (on_dev[i]) continue;
      const size_t bytes = (size_t)params[i].n_azimuth * params[i].n_bins * sizeof(float);
      cudaError_t e = cudaMemcpyAsync(out[i], images[i], bytes, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "copying an image");
      }
    }
  }
  return device_status(&s->main, st);
}

int rr_scan_batch_async(rr_scene* s, uint32_t n, const rr_pose* poses, const rr_sensor_params* params,
                        float* const* out) {
  int rc = check_batch(s, n, poses, params, out);
  if (rc != RR_OK) return rc;
  for (uint32_t i = 0; i < n; ++i)
    if (!is_device_ptr(out[i]))
      return fail(RR_ERR_INVALID_ARG, "scan " + std::to_string(i) + ": rr_scan_batch_async needs device outputs");
  return batch_run(s, &s->main, poses, params, out, n, nullptr, current_stream(), s->cfg);
}

int rr_batch_config_get(const rr_scene* s, rr_batch_config* out) {
  if (!s || !out) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  cfg_to_abi(s->cfg, out);
  return RR_OK;
}

int rr_batch_config_set(rr_scene* s, const rr_batch_config* c) {
  if (!s || !c) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  const int rc = cfg_check(c);
  if (rc != RR_OK) return rc;
  const bool rebuild = c->bvh_build != s->cfg.bvh_build;
  s->cfg = cfg_from_abi(c);
  return rebuild ? rebuild_bvh(s, current_stream()) : RR_OK;
}

int rr_batch_plan(uint32_t n, const rr_sensor_params* params, const rr_batch_config* config, uint32_t* first,
                  uint32_t cap, uint32_t* n_groups, uint64_t* max_workspace) {
  if ((n && !params) || !n_groups || (cap && !first)) return fail(RR_ERR_INVALID_ARG, "NULL argument");
  LaunchCfg cfg;
  if (config) {
    const int rc = cfg_check(config);
    if (rc != RR_OK) return rc;
    cfg = cfg_from_abi(config);
  }
  const rr_pose identity = {{0.f, 0.f, 0.f}, {1.f, 0.f, 0.f, 0.f}};
  for (uint32_t i = 0; i < n; ++i) {
    const int rc = check_params(&identity, &params[i]);
    if (rc != RR_OK) return fail(rc, "scan " + std::to_string(i) + ": " + rr_last_error());
  }
  const std::vector<Group> groups = plan_groups(params, n, cfg);
  uint64_t mx = 0;
  for (size_t g = 0; g < groups.size(); ++g) {
    if (g < cap) first[g] = groups[g].first;
    mx = std::max<uint64_t>(mx, groups[g].L.total);
  }
  *n_groups = (uint32_t)groups.size();
  if (max_workspace) *max_workspace = mx;
  return RR_OK;
}

int rr_autotune(rr_scene* s, uint32_t n, const rr_pose* poses, const rr_sensor_params* params, uint32_t reps,
                rr_batch_config* best_out, float* best_ms, float* start_ms) {
  if (!s || n == 0 || !poses || !params) return fail(RR_ERR_INVALID_ARG, "NULL argument or empty batch");
  if (reps == 0) reps = 1;
  for (uint32_t i = 0; i < n; ++i) {
    const int rc = check_params(&poses[i], &params[i]);
    if (rc != RR_OK) return rc;
  }
  if (int rc = check_device(s, "rr_autotune")) return rc;
  cudaStream_t st = current_stream();
  size_t total = 0;
  uint64_t rays = 0;
  for (uint32_t i = 0; i < n; ++i) {
    total += (size_t)params[i].n_azimuth * params[i].n_bins;
    rays += (uint64_t)params[i].n_azimuth * params[i].rays_per_beam;
  }
  float* d_out = nullptr;
  cudaError_t e = dev_malloc(&d_out, total * sizeof(float));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "allocating the autotuner's images");
  }
  std::vector<float*> images(n);
  size_t off = 0;
  for (uint32_t i = 0; i < n; ++i) {
    images[i] = d_out + off;
    off += (size_t)params[i].n_azimuth * params[i].n_bins;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const LaunchCfg saved = s->cfg;
  int rc = RR_OK;
  // mean device time of one pass over the batch with configuration c
  auto time_cfg = [&](const LaunchCfg& c, float* ms) -> int {
    s->cfg = c;
    int r = batch_run(s, &s->main, poses, params, images.data(), n, nullptr, st, s->cfg);   // warm-up (and capture)
    if (r != RR_OK) return r;
    cudaEventRecord(e0, st);
    for (uint32_t k = 0; k < reps && r == RR_OK; ++k)
      r = batch_run(s, &s->main, poses, params, images.data(), n, nullptr, st, s->cfg);
    cudaEventRecord(e1, st);
    if (r != RR_OK) return r;
    r = device_status(&s->main, st);
    if (r != RR_OK) return r;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / (float)reps;
    return RR_OK;
  };
  LaunchCfg best = saved;
  float best_t = 0.f;
  rc = time_cfg(best, &best_t);
  const float first_t = best_t;
  // coordinate descent: node format, wavefront size, trace block, trace blocks per SM, graph
  if (rc == RR_OK) {
    LaunchCfg c = best;
    c.node_format = best.node_format == RR_NODES_WIDE8 ? RR_NODES_BINARY : RR_NODES_WIDE8;
    float t = 0.f;
    rc = time_cfg(c, &t);
    if (rc == RR_OK && t < best_t) best_t = t, best = c;
  }
  if (rc == RR_OK) {
    std::vector<uint32_t> waves = {0u};
    for (uint32_t w = 1u << 19; w < rays && w <= (1u << 26); w <<= 1) waves.push_back(w);
    for (uint32_t w : waves) {
      if (w == best.wavefront_rays) continue;
      LaunchCfg c = best;
      c.wavefront_rays = w;
      float t = 0.f;
      if ((rc = time_cfg(c, &t)) != RR_OK) break;
      if (t < best_t) best_t = t, best = c;
    }
  }
  if (rc == RR_OK) {
    for (uint32_t b : {64u, 128u, 256u}) {
      if (b == best.trace_block) continue;
      LaunchCfg c = best;
      c.trace_block = b;
      c.trace_blocks_per_sm = 0;
      float t = 0.f;
      if ((rc = time_cfg(c, &t)) != RR_OK) break;
      if (t < best_t) best_t = t, best = c;
    }
  }
  if (rc == RR_OK) {
    const uint32_t mx = (uint32_t)trace_max_blocks_per_sm(best.trace_block, best.node_format == RR_NODES_WIDE8);
    for (uint32_t k : {mx / 2u, (3u * mx) / 4u}) {
      if (k == 0 || k == mx || k == best.trace_blocks_per_sm) continue;
      LaunchCfg c = best;
      c.trace_blocks_per_sm = k;
      float t = 0.f;
      if ((rc = time_cfg(c, &t)) != RR_OK) break;
      if (t < best_t) best_t = t, best = c;
    }
  }
  if (rc == RR_OK) {
    for (uint32_t r : {1u, 4u, 8u, 16u, 32u}) {
      if (r == best.refill) continue;
      LaunchCfg c = best;
      c.refill = r;
      float t = 0.f;
      if ((rc = time_cfg(c, &t)) != RR_OK) break;
      if (t < best_t) best_t = t, best = c;
    }
  }
  if (rc == RR_OK) {
    LaunchCfg c = best;
    c.use_graph = best.use_graph ? 0u : 1u;
    float t = 0.f;
    rc = time_cfg(c, &t);
    if (rc == RR_OK && t < best_t) best_t = t, best = c;
  }
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_out);
  if (rc != RR_OK) {
    s->cfg = saved;
    return rc;
  }
  s->cfg = best;
  if (best_out) cfg_to_abi(best, best_out);
  if (best_ms) *best_ms = best_t;
  if (start_ms) *start_ms = first_t;
  return RR_OK;
}

}  // extern "C"

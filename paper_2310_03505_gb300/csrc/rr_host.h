// rr_host.h -- host-side scene object and the launchers each translation
// unit exports to the C ABI layer.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "rr_internal.cuh"

namespace rr_host {

// thread-local error message and stream
void set_error(const std::string& msg);
cudaStream_t current_stream();

struct ProfEvent {
  int kind;
  cudaEvent_t start, stop;
};

// tunables of the batched launch sequence (rr_batch_config)
struct LaunchCfg {
  uint32_t wavefront_rays = 0;        // most initial rays per launch sequence, 0: workspace limit only
  uint32_t trace_block = 64;          // 64, 128 or 256
  uint32_t trace_blocks_per_sm = 0;   // 0: occupancy maximum
  uint32_t use_graph = 1;             // capture each launch sequence once and replay it
  uint32_t node_format = RR_NODES_BINARY;
  uint32_t refill = 16;               // idle lanes that trigger a refill (1..32)
  uint32_t split = 3;                 // a single scan as this many azimuth ranges on their own streams
  uint64_t ws_limit = uint64_t(24) << 30;
  uint32_t bvh_build = RR_BVH_SAH_TOP;
  uint32_t order = 0;                 // RR_ORDER_*: query order of the closest-hit queries of bounces >= 1
};

constexpr uint32_t kMaxSplit = 4;

// What one stream of scans needs besides the scene: device counters and
// status, the scan workspace, an image buffer for host outputs, pinned
// staging of the scan descriptors and the captured launch graph.  A scene owns
// one for its own entry points; a server owns one per slot, so launch
// sequences on different streams never share scratch.
struct ExecCtx {
  rr::ScanCounters* d_ctr = nullptr;
  rr::ScanCounters* h_ctr = nullptr;   // pinned mirror
  void* ws = nullptr;
  size_t ws_bytes = 0;
  float* d_image = nullptr;            // device images of host outputs
  size_t image_bytes = 0;
  void* h_stage = nullptr;             // pinned staging of the scan descriptors
  size_t stage_bytes = 0;
  cudaEvent_t stage_ev = nullptr;      // the last upload from h_stage has been read
  bool stage_used = false;
  cudaStream_t cap_stream = nullptr;   // stream used only to capture graphs
  cudaGraphExec_t gexec = nullptr;     // last captured launch sequence
  std::vector<unsigned char> gkey;     // what gexec was captured for
  // deferred visibility: the visibility queries of bounce b run on `side`
  // while the closest-hit queries of bounce b + 1 run on the launch stream
  cudaStream_t side = nullptr;
  cudaEvent_t fork[RR_MAX_BOUNCES] = {};
  cudaEvent_t join[RR_MAX_BOUNCES] = {};
  bool side_ready = false;
};
cudaError_t ctx_init(ExecCtx* x, cudaStream_t st);   // counters (zeroed)
void ctx_free(ExecCtx* x);

// an extra stream of a split scan with its execution context
struct SplitLane {
  ExecCtx ctx;
  cudaStream_t stream = nullptr;
  cudaEvent_t join = nullptr;
};

}  // namespace rr_host

struct rr_scene {
  int device = 0;
  uint32_t nv = 0, nt = 0, nm = 0;
  // resident scene
  float* d_vtx = nullptr;          // [V][3]
  uint32_t* d_idx = nullptr;       // [T][3]
  uint16_t* d_mat_id = nullptr;    // [T]
  rr_material* d_raw_mats = nullptr;
  rr::MatDev* d_mats = nullptr;    // [M]
  float4* d_lut = nullptr;         // [M][kLutCells + 1]
  float* d_lut_cells = nullptr;    // [M][kLutCells]
  uint8_t* d_lobe_kind = nullptr;  // [M] kLobeEq5 / kLobeCookTorrance / kLobeTable
  std::vector<uint8_t> lobe_kind;  // host copy
  std::vector<uint32_t> raw_flags; // rr_material.flags of every material
  float* d_lobe_samples = nullptr; // [M][kLobeSamples] tabulated lobes (allocated on first use)
  float4* d_tri = nullptr;         // [3][T][3] sorted leaves in three rotated copies, then [T] unit normals
  float4* d_nodes = nullptr;       // [T-1][4]
  // 8-wide quantised BVH (collapsed from the binary one at every build)
  uint32_t wcap = 0;               // wide node capacity (T - 1, at least 1)
  uint32_t wide_epoch = 0;         // build counter tagging the published work items
  bool wide_stale = true;          // the binary LBVH changed since the last collapse
  uint32_t* d_cut = nullptr;       // [T-1][8] cut of every binary internal node, slot order
  float4* d_wnodes = nullptr;      // [wcap][kWideNodeWords]
  float4* d_wtri = nullptr;        // the same in wide-leaf order
  unsigned long long* d_wsrc = nullptr;   // [wcap] epoch << 32 | binary node of each wide node
  uint4* d_wrec = nullptr;         // [wcap] (binary node, first child, first triangle, 0)
  uint32_t* d_wctr = nullptr;      // [8] ticket, allocated, done, triangles, error
  // build temporaries (kept for rebuilds)
  float4* d_centroid = nullptr;    // [T]
  uint32_t* d_keys[2] = {nullptr, nullptr};
  uint32_t* d_vals[2] = {nullptr, nullptr};
  uint32_t* d_hist = nullptr;      // [4 sort passes][256][tiles]
  uint32_t* d_parent = nullptr;    // [2T-1]
  uint32_t* d_child = nullptr;     // [T-1][2]
  float* d_nbox = nullptr;         // [2T-1][6]
  uint32_t* d_visit = nullptr;     // [T-1]
  uint32_t* d_misc = nullptr;      // [8]: bounds (6, encoded), error bits, depth
  uint2* d_range = nullptr;        // [T-1] leaf range (first, last) of every internal node
  // SAH top over the LBVH's subtrees (allocated with the first such build)
  uint32_t* d_cl_at = nullptr;     // [T] cluster root reference at the cluster's first leaf, else kNone
  uint32_t* d_cl_bsum = nullptr;   // [cl_blocks rounded up to 4] clusters per compaction block, then offsets
  float4* d_cl_rec = nullptr;      // [2][T][2] cluster (lo xyz, weight) (hi xyz, root reference), ping-pong
  uint32_t* d_top_slot = nullptr;  // [T] node slots of the LBVH's top part (root first)
  uint4* d_top_task = nullptr;     // [T] block tasks (first, end, node slot, depth | source << 31)
  uint32_t* d_top_ready = nullptr; // [T] block task published
  uint4* d_top_small = nullptr;    // [T] warp tasks, same fields
  uint32_t* d_top_ctr = nullptr;   // [8] counters of the build
  uint32_t* d_top_cb = nullptr;    // [T][6] centroid bounds of the block task at each node slot (encoded)
  uint32_t cl_blocks = 0;
  uint32_t sort_tiles = 0;
  uint32_t depth = 0;
  float build_ms = 0.f;
  size_t scene_bytes = 0;
  // execution state of the scene's own entry points
  rr_host::ExecCtx main;
  rr_host::SplitLane split[rr_host::kMaxSplit - 1];   // the other azimuth ranges of split scans
  uint32_t split_used = 0;                           // lanes that have run work (status, statistics)
  cudaEvent_t fork = nullptr;
  rr_host::LaunchCfg cfg;
  std::mutex lock;                     // lazy wide collapse and launch counting across threads
  cudaEvent_t wide_ready = nullptr;    // recorded after the latest collapse
  // profiling
  bool prof = false;
  std::vector<rr_host::ProfEvent> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[RR_K_COUNT] = {0};
  uint64_t prof_launches[RR_K_COUNT] = {0};
  cudaEvent_t prof_base = nullptr;                               // time origin of the intervals
  std::vector<std::pair<double, double>> prof_iv[RR_K_COUNT];    // [start, stop] ms after prof_base
  double prof_busy_done[RR_K_COUNT] = {0};                       // unions folded in before a new base
  std::atomic<uint64_t> launches{0};  // kernels launched for this scene (any stream)
};

namespace rr_host {

// rr_build.cu
cudaError_t build_alloc(rr_scene* s);
cudaError_t build_lbvh(rr_scene* s, cudaStream_t st, bool with_depth);   // a1..a5 on s->d_vtx; counts its launches
cudaError_t build_materials(rr_scene* s, cudaStream_t st);
cudaError_t build_wide(rr_scene* s, cudaStream_t st);      // a6, stream ordered after the LBVH

// rr_trace.cu
int num_sms();
int trace_max_blocks_per_sm(uint32_t block, bool wide);
cudaError_t launch_raygen(const rr::ScanArgs& a, cudaStream_t st);
cudaError_t launch_query(const rr::ScanArgs& a, uint32_t bounce, bool any, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_vis_prep(const rr::ScanArgs& a, uint32_t bounce, cudaStream_t st);
cudaError_t launch_shade(const rr::ScanArgs& a, uint32_t bounce, cudaStream_t st);
cudaError_t launch_order(const rr::ScanArgs& a, uint32_t bounce, cudaStream_t st);   // query order of a bounce

// failure detection (rr_selftest_wait): each runs one bounded device wait on
// a flag that nothing sets and reports whether it gave up as designed
cudaError_t selftest_top_wait(uint32_t* scratch, cudaStream_t st, bool* gave_up);    // rr_build.cu
cudaError_t selftest_wide_wait(uint32_t* scratch, cudaStream_t st, bool* gave_up);   // rr_build.cu
cudaError_t selftest_look_back_wait(void* scratch, cudaStream_t st, bool* gave_up);  // rr_trace.cu

// rr_image.cu
void init_image_attrs();
cudaError_t launch_image(const rr::ScanArgs& a, bool pattern, cudaStream_t st);
cudaError_t launch_db_u8(const float* polar, uint64_t n, float cutoff_db, uint8_t* out, cudaStream_t st);

// rebuild with the scene's configuration, wait, check status and depth (rr_api.cu)
int rebuild_bvh(rr_scene* s, cudaStream_t st);

// profiling helpers (rr_api.cu)
void prof_begin(rr_scene* s, int kind, cudaStream_t st, cudaEvent_t* stop_out);
void prof_end(rr_scene* s, cudaEvent_t stop, cudaStream_t st);

// scan orchestration shared by the entry points (rr_batch.cu)
struct WsLayout {
  uint32_t ray_cap, rec_cap, tiles, n_desc;
  size_t off_rays0, off_rays1, off_hits, off_vis, off_recs, off_status, off_tmp, off_desc, off_order, total;
  size_t tmp_floats;
  bool clamped;
  bool order;   // holds the closest-hit query order buffers
};
struct DebugOut {
  rr_segment* segs = nullptr;
  uint32_t seg_cap = 0;
  float* tallies = nullptr;
  const uint8_t* mask = nullptr;
};
// one launch sequence: scans [first, first + count) of a request
struct Group {
  uint32_t first = 0, count = 0;
  WsLayout L;
};
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
// Every device and pinned host allocation of the library goes through these
// two, so that rr_fault_inject_alloc can make a chosen one fail (as
// cudaErrorMemoryAllocation, without calling CUDA).
cudaError_t dev_malloc_raw(void** p, size_t n);
cudaError_t host_malloc_raw(void** p, size_t n);
template <class T>
cudaError_t dev_malloc(T** p, size_t n) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), n);
}
template <class T>
cudaError_t host_malloc(T** p, size_t n) {
  return host_malloc_raw(reinterpret_cast<void**>(p), n);
}
bool is_device_ptr(const void* p);
int check_params(const rr_pose* pose, const rr_sensor_params* p);
// RR_ERR_INVALID_ARG unless the current device is the scene's (who: caller name for the message)
int check_device(const rr_scene* s, const char* who);
// worst-case workspace of scans ps[0..n) traced together, clamped to limit
WsLayout plan_workspace(const rr_sensor_params* ps, uint32_t n, uint64_t limit, const uint32_t* az_count = nullptr,
                        bool order = false);
// the same with the queues and records sized to given capacities (an estimate of the
// ray tree; clamped = smaller than the worst case), never below the initial rays
WsLayout plan_workspace_caps(const rr_sensor_params* ps, uint32_t n, uint64_t q_cap, uint64_t r_cap,
                            bool order = false);
// split n scans into launch sequences that respect the limits of cfg
std::vector<Group> plan_groups(const rr_sensor_params* ps, uint32_t n, const LaunchCfg& cfg);
// queue the launch sequence of scans poses/ps[0..n) writing images[i]
// (device); the workspace at ws is laid out by L.  host_desc: where the
// descriptors are staged (NULL: the scene's pinned staging).  No allocation
// unless allow_graph.
int batch_enqueue(rr_scene* s, ExecCtx* x, const rr_pose* poses, const rr_sensor_params* ps, float* const* images,
                  uint32_t n, const DebugOut* dbg, cudaStream_t st, void* ws, const WsLayout& L, bool profile,
                  bool allow_graph, const LaunchCfg& cfg, void* host_desc, const uint32_t* az_range = nullptr);
// one scan, split into azimuth ranges on several streams when the scene's configuration asks for it
int scan_split(rr_scene* s, const rr_pose* pose, const rr_sensor_params* p, float* image, cudaStream_t st,
               bool profile);
// device status of the scene's contexts (main and split lanes); waits for st
int scene_status(rr_scene* s, cudaStream_t st);
int ensure_workspace(ExecCtx* x, size_t bytes, cudaStream_t st);
int ensure_image(ExecCtx* x, size_t bytes, cudaStream_t st);
int device_status(ExecCtx* x, cudaStream_t st);
// whole request on the context's workspace (grown as needed): images[i] device pointers
int batch_run(rr_scene* s, ExecCtx* x, const rr_pose* poses, const rr_sensor_params* ps, float* const* images,
              uint32_t n, const DebugOut* dbg, cudaStream_t st, const LaunchCfg& cfg);

}  // namespace rr_host

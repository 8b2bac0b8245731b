// rr_host.h -- host-side scene object and the launchers each translation
// unit exports to the C ABI layer.
#pragma once

#include <cuda_runtime.h>

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
  float4* d_tri = nullptr;         // [T][3] sorted leaves
  float4* d_nodes = nullptr;       // [T-1][4]
  // build temporaries (kept for rebuilds)
  float4* d_centroid = nullptr;    // [T]
  uint32_t* d_keys[2] = {nullptr, nullptr};
  uint32_t* d_vals[2] = {nullptr, nullptr};
  uint32_t* d_hist = nullptr;      // [256][tiles]
  uint32_t* d_parent = nullptr;    // [2T-1]
  uint32_t* d_child = nullptr;     // [T-1][2]
  float* d_nbox = nullptr;         // [2T-1][6]
  uint32_t* d_visit = nullptr;     // [T-1]
  uint32_t* d_misc = nullptr;      // [8]: bounds (6, encoded), error bits, depth
  uint32_t sort_tiles = 0;
  uint32_t depth = 0;
  float build_ms = 0.f;
  size_t scene_bytes = 0;
  // scan workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  rr::ScanCounters* d_ctr = nullptr;
  rr::ScanCounters* h_ctr = nullptr;   // pinned mirror
  float* d_image = nullptr;            // internal image for host outputs
  size_t image_bytes = 0;
  // profiling
  bool prof = false;
  std::vector<rr_host::ProfEvent> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[RR_K_COUNT] = {0};
  uint64_t prof_launches[RR_K_COUNT] = {0};
  uint64_t launches = 0;  // kernels launched by this scene
};

namespace rr_host {

// rr_build.cu
cudaError_t build_alloc(rr_scene* s);
cudaError_t build_lbvh(rr_scene* s, cudaStream_t st, bool with_depth);   // a1..a5 on s->d_vtx; counts its launches
cudaError_t build_materials(rr_scene* s, cudaStream_t st);

// rr_trace.cu
struct LaunchDims {
  int trace_grid, trace_block, shade_grid, shade_block;
};
LaunchDims trace_dims();
cudaError_t launch_raygen(const rr::ScanArgs& a, cudaStream_t st);
cudaError_t launch_trace(const rr::ScanArgs& a, uint32_t bounce, cudaStream_t st);
cudaError_t launch_shade(const rr::ScanArgs& a, uint32_t bounce, cudaStream_t st);

// rr_image.cu
cudaError_t launch_image(const rr::ScanArgs& a, cudaStream_t st);
cudaError_t launch_db_u8(const float* polar, uint64_t n, float cutoff_db, uint8_t* out, cudaStream_t st);

// profiling helpers (rr_api.cu)
void prof_begin(rr_scene* s, int kind, cudaStream_t st, cudaEvent_t* stop_out);
void prof_end(rr_scene* s, cudaEvent_t stop, cudaStream_t st);

// scan orchestration shared by the entry points (rr_api.cu)
struct WsLayout {
  uint32_t ray_cap, rec_cap, tiles;
  size_t off_rays0, off_rays1, off_hits, off_recs, off_status, off_tmp, total;
  bool clamped;
};
struct DebugOut {
  rr_segment* segs = nullptr;
  uint32_t seg_cap = 0;
  float* tallies = nullptr;
  const uint8_t* mask = nullptr;
};
int fail(int code, const std::string& msg);
bool is_device_ptr(const void* p);
int check_params(const rr_pose* pose, const rr_sensor_params* p);
WsLayout plan_workspace(const rr_sensor_params* p);
int scan_enqueue_into(rr_scene* s, const rr_pose* pose, const rr_sensor_params* p, float* image, const DebugOut* dbg,
                      cudaStream_t st, void* ws, const WsLayout& L, bool profile);
int device_status(rr_scene* s, cudaStream_t st);

}  // namespace rr_host

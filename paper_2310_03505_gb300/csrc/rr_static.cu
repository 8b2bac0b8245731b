// rr_static.cu -- rr_scan_static: the polar scan without any allocation.
//
// Some callers cannot allocate device memory while they run: real-time loops
// that must never block on the allocator (cudaMalloc and cudaFree can
// synchronise the whole device), and host programs whose device memory is
// owned by another allocator under a fixed budget (a framework's caching
// allocator) and that forbid raw cudaMalloc.  rr_scan grows a workspace inside
// the scene on demand, which such callers cannot accept.  rr_scan_static runs
// the same kernels on a fixed scratch area compiled into the library instead.
//
// The scratch is one file-scope device array of kStaticScratchBytes.  Every
// GPU that loads the library holds it until the process exits.  Host code
// cannot use the array's name as a device address, so the first call on each
// device (with that device current) looks the address up once with
// cudaGetSymbolAddress and keeps it.
//
// All calls share the one array and it keeps the contents of the last call.
// The scan reads nothing from it before writing: the kernels write the ray
// queues, hits and return records before they read them, and the trace kernel
// clears every tile flag a bounce uses.  Calls that overlap on the GPU
// (several streams, threads or scenes at once) race on the array.  The scan's
// status counters are the scene's own (those of its rr_scan path), so a
// static call that overlaps any other scan of the same scene also races on
// them.
//
// The static path always traverses the binary BVH, which every build makes:
// both node formats give the same closest hit for every query, and the
// binary nodes never need the lazy collapse of the 8-wide BVH.
#include <cuda_runtime.h>

#include <mutex>

#include "rr_host.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of g_static_scratch on the current device (set up once)
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return rr_host::fail(RR_ERR_CUDA, "rr_scan_static: no usable current device");
  }
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return rr_host::fail(RR_ERR_CUDA, std::string("rr_scan_static: cudaGetSymbolAddress failed: ") +
                                            cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return RR_OK;
}

}  // namespace

extern "C" int rr_scan_static(rr_scene* s, const rr_pose* pose, const rr_sensor_params* p, float* out_polar) {
  using namespace rr_host;
  if (!s || !out_polar) return fail(RR_ERR_INVALID_ARG, "scene and out_polar must not be NULL");
  int rc = check_params(pose, p);
  if (rc != RR_OK) return rc;
  if ((rc = check_device(s, "rr_scan_static")) != RR_OK) return rc;
  if (!is_device_ptr(out_polar)) return fail(RR_ERR_INVALID_ARG, "rr_scan_static needs a device output");
  const WsLayout L = plan_workspace(p, 1, kStaticScratchBytes);
  if (L.total > kStaticScratchBytes || L.clamped)
    return fail(RR_ERR_INVALID_ARG, "rr_scan_static: this scan needs " + std::to_string(L.total) +
                                        " bytes of scratch, more than the fixed " +
                                        std::to_string(kStaticScratchBytes) + " bytes; use rr_scan");
  void* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != RR_OK) return rc;
  cudaStream_t st = current_stream();
  // the scan descriptor is staged from this stack buffer (a pageable copy
  // returns once the source has been read), so nothing is allocated
  alignas(16) unsigned char desc[sizeof(rr::ScanDesc) + 2 * 2 * sizeof(uint32_t)];
  float* const images[1] = {out_polar};
  LaunchCfg cfg = s->cfg;
  cfg.use_graph = 0;
  cfg.node_format = RR_NODES_BINARY;
  rc = batch_enqueue(s, &s->main, pose, p, images, 1, nullptr, st, scratch, L, false, false, cfg, desc);
  if (rc != RR_OK) return rc;
  return device_status(&s->main, st);
}

"""Python binding of the C ABI in ``include/rr.h`` (ctypes).

Argument marshalling only: every function has the name of the C entry point
it calls, turns numpy arrays / torch tensors / dicts into pointers and
structs, raises ``RRError`` on a non-zero status, and nothing else.  All the
scan work runs in the CUDA library ``librr.so``; there is no CPU fallback.
If the library is missing, every call raises.

Buffers may be numpy arrays, CPU tensors or CUDA tensors (the library tells
host and device pointers apart).  Calls run on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librr.so")

RR_OK, RR_ERR_INVALID_ARG, RR_ERR_OOM, RR_ERR_CAPACITY, RR_ERR_TIMEOUT, RR_ERR_CUDA, RR_ERR_BUSY, RR_ERR_CANCELLED = range(8)
RR_MULTIPATH, RR_REFRACTION, RR_SPECKLE, RR_NOISE, RR_COUNT_TRAVERSAL, RR_NOISE_PERLIN = 1, 2, 4, 8, 16, 32
RR_MAT_PERFECT_CONDUCTOR, RR_MAT_COOK_TORRANCE, RR_MAT_TABULATED_LOBE = 1, 2, 4
RR_WAIT_TOP_TASK, RR_WAIT_WIDE_NODE, RR_WAIT_SHADE_PREFIX = 0, 1, 2
RR_LOBE_SAMPLES = 4097
RR_NO_HIT = 0xFFFFFFFF
RR_K_RAYGEN, RR_K_TRACE, RR_K_SHADE, RR_K_IMAGE, RR_K_BUILD, RR_K_VIS, RR_K_COUNT = range(7)
KERNEL_NAMES = ["raygen", "trace", "shade", "image", "build", "vis"]


class RRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rr status {code}: {msg}")
        self.code = code


class rr_material(C.Structure):
    _fields_ = [("eps_r", C.c_float), ("loss_tangent", C.c_float), ("A", C.c_float), ("B", C.c_float),
                ("C", C.c_float), ("flags", C.c_uint32)]


class rr_pose(C.Structure):
    _fields_ = [("p", C.c_float * 3), ("q", C.c_float * 4)]


class rr_sensor_params(C.Structure):
    _fields_ = [("n_azimuth", C.c_uint32), ("rays_per_beam", C.c_uint32), ("max_bounces", C.c_uint32),
                ("n_bins", C.c_uint32), ("beam_width_rad", C.c_float), ("beam_prob", C.c_float),
                ("elevation_rad", C.c_float), ("bin_size_m", C.c_float), ("t_min_m", C.c_float),
                ("min_energy", C.c_float), ("freq_hz", C.c_float), ("blur_sigma_bins", C.c_float),
                ("az_pattern_sigma", C.c_float), ("noise_sys", C.c_float), ("noise_amb", C.c_float),
                ("flags", C.c_uint32), ("seed", C.c_uint64), ("scan_id", C.c_uint32), ("beam_aspect", C.c_float),
                ("noise_cell_az", C.c_float), ("noise_cell_bins", C.c_float), ("range_falloff", C.c_float)]


class rr_segment(C.Structure):
    _fields_ = [("az", C.c_uint32), ("k", C.c_uint32), ("path", C.c_uint32), ("bounce", C.c_uint32),
                ("tri", C.c_uint32), ("t", C.c_float), ("E", C.c_float), ("flags", C.c_uint32),
                ("cos_i", C.c_float), ("ret_t", C.c_float), ("ret_a", C.c_float), ("visits", C.c_float)]


SEGMENT_DTYPE = np.dtype([("az", "<u4"), ("k", "<u4"), ("path", "<u4"), ("bounce", "<u4"), ("tri", "<u4"),
                          ("t", "<f4"), ("E", "<f4"), ("flags", "<u4"), ("cos_i", "<f4"), ("ret_t", "<f4"),
                          ("ret_a", "<f4"), ("visits", "<f4")])


class rr_scene_info(C.Structure):
    _fields_ = [("n_triangles", C.c_uint32), ("n_materials", C.c_uint32), ("bvh_depth", C.c_uint32),
                ("n_wide_nodes", C.c_uint32), ("device_bytes", C.c_uint64), ("workspace_bytes", C.c_uint64),
                ("build_ms", C.c_float), ("reserved_f", C.c_float)]


class rr_stats(C.Structure):
    _fields_ = [("closest_queries", C.c_uint64), ("anyhit_queries", C.c_uint64), ("returns", C.c_uint64),
                ("scans", C.c_uint64), ("nodes_visited", C.c_uint64), ("tris_tested", C.c_uint64),
                ("kernel_launches", C.c_uint64), ("anyhit_nodes_visited", C.c_uint64),
                ("anyhit_tris_tested", C.c_uint64)]


class rr_profile(C.Structure):
    _fields_ = [("ms", C.c_double * RR_K_COUNT), ("launches", C.c_uint64 * RR_K_COUNT),
                ("busy_ms", C.c_double * RR_K_COUNT)]


class rr_batch_config(C.Structure):
    _fields_ = [("wavefront_rays", C.c_uint32), ("trace_block", C.c_uint32), ("trace_blocks_per_sm", C.c_uint32),
                ("use_graph", C.c_uint32), ("node_format", C.c_uint32), ("refill_threshold", C.c_uint32),
                ("workspace_limit", C.c_uint64), ("split_streams", C.c_uint32), ("bvh_build", C.c_uint32),
                ("query_order", C.c_uint32), ("reserved", C.c_uint32)]


RR_NODES_WIDE8, RR_NODES_BINARY = 0, 1
RR_BVH_LBVH, RR_BVH_SAH_TOP = 0, 1
RR_ORDER_QUEUE, RR_ORDER_CELL_OCTANT = 0, 1
WIDE_NODE_BYTES = 80
RR_REQ_QUEUED, RR_REQ_RUNNING, RR_REQ_DONE, RR_REQ_FAILED, RR_REQ_CANCELLED = range(5)
RR_ADMIT_ESTIMATE, RR_ADMIT_WORST_CASE = 0, 1


class rr_serve_config(C.Structure):
    _fields_ = [("memory_budget", C.c_uint64), ("slots", C.c_uint32), ("max_batch_scans", C.c_uint32),
                ("max_batch_rays", C.c_uint32), ("max_queue", C.c_uint32), ("node_format", C.c_uint32),
                ("refill_threshold", C.c_uint32), ("admission", C.c_uint32), ("estimate_factor", C.c_float)]


class rr_serve_record(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("submit_ms", C.c_double), ("start_ms", C.c_double),
                ("done_ms", C.c_double), ("batch_size", C.c_uint32), ("reserved", C.c_uint32)]


class rr_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("rejected_busy", C.c_uint64), ("batches", C.c_uint64), ("closest_queries", C.c_uint64),
                ("anyhit_queries", C.c_uint64), ("initial_rays", C.c_uint64), ("queued", C.c_uint64),
                ("busy_ms", C.c_double), ("elapsed_ms", C.c_double), ("latency_p50_ms", C.c_double),
                ("latency_p99_ms", C.c_double), ("latency_mean_ms", C.c_double), ("latency_max_ms", C.c_double),
                ("retried", C.c_uint64), ("cancelled", C.c_uint64)]


# every symbol declared in include/rr.h with its ctypes signature
_P = C.c_void_p
SIGNATURES = {
    "rr_version": ([], C.c_int),
    "rr_last_error": ([], C.c_char_p),
    "rr_set_stream": ([_P], C.c_int),
    "rr_selftest_wait": ([C.c_uint32, C.POINTER(C.c_double)], C.c_int),
    "rr_fault_inject_alloc": ([C.c_int64, C.POINTER(C.c_uint64)], C.c_int),
    "rr_scene_create": ([_P, C.c_uint32, _P, C.c_uint32, _P, _P, C.c_uint32, C.POINTER(_P)], C.c_int),
    "rr_scene_destroy": ([_P], C.c_int),
    "rr_scene_update_vertices": ([_P, _P], C.c_int),
    "rr_scene_set_lobe": ([_P, C.c_uint32, _P], C.c_int),
    "rr_scene_save": ([_P, _P, C.c_uint64, C.POINTER(C.c_uint64)], C.c_int),
    "rr_scene_load": ([_P, C.c_uint64, C.POINTER(_P)], C.c_int),
    "rr_scene_info_get": ([_P, C.POINTER(rr_scene_info)], C.c_int),
    "rr_scene_export_bvh": ([_P, _P, _P, _P, _P, _P], C.c_int),
    "rr_scene_export_wide": ([_P, _P, C.c_uint32, C.POINTER(C.c_uint32), _P], C.c_int),
    "rr_scan": ([_P, C.POINTER(rr_pose), C.POINTER(rr_sensor_params), _P], C.c_int),
    "rr_scan_async": ([_P, C.POINTER(rr_pose), C.POINTER(rr_sensor_params), _P], C.c_int),
    "rr_scene_sync": ([_P], C.c_int),
    "rr_scan_static": ([_P, C.POINTER(rr_pose), C.POINTER(rr_sensor_params), _P], C.c_int),
    "rr_scan_batch": ([_P, C.c_uint32, _P, _P, _P], C.c_int),
    "rr_scan_batch_async": ([_P, C.c_uint32, _P, _P, _P], C.c_int),
    "rr_batch_config_get": ([_P, C.POINTER(rr_batch_config)], C.c_int),
    "rr_batch_config_set": ([_P, C.POINTER(rr_batch_config)], C.c_int),
    "rr_batch_plan": ([C.c_uint32, _P, C.POINTER(rr_batch_config), _P, C.c_uint32, C.POINTER(C.c_uint32),
                       C.POINTER(C.c_uint64)], C.c_int),
    "rr_autotune": ([_P, C.c_uint32, _P, _P, C.c_uint32, C.POINTER(rr_batch_config), C.POINTER(C.c_float),
                     C.POINTER(C.c_float)], C.c_int),
    "rr_serve_create": ([C.POINTER(rr_serve_config), C.POINTER(_P)], C.c_int),
    "rr_serve_destroy": ([_P], C.c_int),
    "rr_serve_submit": ([_P, _P, C.POINTER(rr_pose), C.POINTER(rr_sensor_params), _P, C.POINTER(C.c_uint64)],
                        C.c_int),
    "rr_serve_poll": ([_P, C.c_uint64, C.POINTER(C.c_int)], C.c_int),
    "rr_serve_cancel": ([_P, C.c_uint64, C.POINTER(C.c_int)], C.c_int),
    "rr_serve_wait": ([_P, C.c_uint64, C.c_uint32], C.c_int),
    "rr_serve_result": ([_P, C.c_uint64, C.POINTER(rr_serve_record)], C.c_int),
    "rr_serve_stats_get": ([_P, C.POINTER(rr_serve_stats), C.c_int], C.c_int),
    "rr_scan_debug": ([_P, C.POINTER(rr_pose), C.POINTER(rr_sensor_params), _P, _P, _P, C.c_uint64,
                       C.POINTER(C.c_uint64), _P], C.c_int),
    "rr_accumulate_returns": ([_P, _P, _P, C.c_uint64, C.c_uint32, C.c_uint32, _P], C.c_int),
    "rr_polar_to_db_u8": ([_P, C.c_uint64, C.c_float, _P], C.c_int),
    "rr_scene_stats": ([_P, C.POINTER(rr_stats), C.c_int], C.c_int),
    "rr_profile_enable": ([_P, C.c_int], C.c_int),
    "rr_profile_read": ([_P, C.POINTER(rr_profile), C.c_int], C.c_int),
}

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load librr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing: run paper_2310_03505_gb300.build first")
            lib = C.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(rc):
    if rc != RR_OK:
        raise RRError(rc, load().rr_last_error().decode())


def _ptr(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "buffers must be contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "buffers must be contiguous"
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _use_torch_stream():
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            load().rr_set_stream(C.c_void_p(torch.cuda.current_stream().cuda_stream))
    except ImportError:
        pass


# ------------------------------------------------------------------- structs
def make_params(s: dict) -> rr_sensor_params:
    flags = ((RR_MULTIPATH if s.get("multipath") else 0) | (RR_REFRACTION if s.get("refraction") else 0) |
             (RR_SPECKLE if s.get("speckle") else 0) | (RR_NOISE if s.get("noise") else 0) |
             (RR_COUNT_TRAVERSAL if s.get("count_traversal") else 0) | (RR_NOISE_PERLIN if s.get("perlin") else 0))
    return rr_sensor_params(s["n_azimuth"], s["rays_per_beam"], s["max_bounces"], s["n_bins"], s["beam_width"],
                            s["beam_prob"], s["elevation"], s["bin_size"], s["t_min"], s["min_energy"], s["freq_hz"],
                            s["blur_sigma_bins"], s["az_pattern_sigma"], s["noise_sys"], s["noise_amb"], flags,
                            int(s["seed"]), int(s["scan_id"]), s.get("beam_aspect", 0.0),
                            s.get("noise_cell_az", 0.0), s.get("noise_cell_bins", 0.0),
                            s.get("range_falloff", 0.0))


def make_pose(pz: dict) -> rr_pose:
    P = rr_pose()
    for i in range(3):
        P.p[i] = float(pz["p"][i])
    for i in range(4):
        P.q[i] = float(pz["q"][i])
    return P


def make_materials(mats) -> C.Array:
    arr = (rr_material * len(mats))()
    for i, m in enumerate(mats):
        lobe = m.get("lobe", "eq5")
        flags = ((RR_MAT_PERFECT_CONDUCTOR if m.get("pec") else 0) |
                 (RR_MAT_COOK_TORRANCE if lobe == "cook_torrance" else 0) |
                 (RR_MAT_TABULATED_LOBE if lobe == "table" else 0))
        arr[i] = rr_material(m["eps_r"], m["loss_tangent"], m["A"], m["B"], m["C"], flags)
    return arr


# ------------------------------------------------------------------- C ABI
def rr_version() -> int:
    return load().rr_version()


def rr_last_error() -> str:
    return load().rr_last_error().decode()


def rr_set_stream(stream_handle) -> None:
    _check(load().rr_set_stream(C.c_void_p(stream_handle)))


def rr_fault_inject_alloc(fail_at: int) -> int:
    """Arms (fail_at >= 0: that many more allocations pass, the next fails)
    or disarms (fail_at < 0) the library's allocation fault injection;
    returns the allocations that passed the gate since the previous call."""
    seen = C.c_uint64(0)
    _check(load().rr_fault_inject_alloc(C.c_int64(int(fail_at)), C.byref(seen)))
    return int(seen.value)


def rr_selftest_wait(which: int):
    """Run one of the library's bounded device waits on a flag that nothing
    sets.  Returns (status, wall ms); RR_ERR_TIMEOUT is the expected status
    (the wait gave up and raised its error bit).  Never raises on a status."""
    _use_torch_stream()
    ms = C.c_double(0.0)
    rc = load().rr_selftest_wait(C.c_uint32(which), C.byref(ms))
    return rc, ms.value


def rr_scene_create(vertices, triangles, material_ids, materials):
    """vertices [V,3] float32, triangles [T,3] uint32, material_ids [T] uint16,
    materials: list of dicts (eps_r, loss_tangent, A, B, C, pec).  Returns the handle."""
    _use_torch_stream()
    L = load()
    mats = make_materials(materials)
    h = C.c_void_p()
    nv = int(vertices.shape[0])
    nt = int(triangles.shape[0])
    _check(L.rr_scene_create(_ptr(vertices), nv, _ptr(triangles), nt, _ptr(material_ids), C.cast(mats, C.c_void_p),
                             len(materials), C.byref(h)))
    return h


def rr_scene_destroy(scene) -> None:
    _check(load().rr_scene_destroy(scene))


def rr_scene_update_vertices(scene, vertices) -> None:
    _use_torch_stream()
    _check(load().rr_scene_update_vertices(scene, _ptr(vertices)))


def rr_scene_save(scene) -> bytes:
    """The scene's mesh, materials, tabulated lobes and launch configuration
    as a blob (see rr_scene_load)."""
    _use_torch_stream()
    size = C.c_uint64(0)
    _check(load().rr_scene_save(scene, None, 0, C.byref(size)))
    buf = np.zeros(size.value, np.uint8)
    _check(load().rr_scene_save(scene, _ptr(buf), size.value, C.byref(size)))
    return buf.tobytes()


def rr_scene_load(blob: bytes):
    """A new scene from a blob written by rr_scene_save; returns the handle."""
    _use_torch_stream()
    b = np.frombuffer(blob, np.uint8)
    h = _P()
    _check(load().rr_scene_load(_ptr(b), b.size, C.byref(h)))
    return h


def rr_scene_set_lobe(scene, material: int, density) -> None:
    """density: RR_LOBE_SAMPLES floats over [0, pi/2] (host or device)."""
    _use_torch_stream()
    d = density
    if isinstance(d, (list, tuple)) or (isinstance(d, np.ndarray) and d.dtype != np.float32):
        d = np.ascontiguousarray(np.asarray(d, np.float32))
    if int(np.prod(d.shape)) != RR_LOBE_SAMPLES:
        raise ValueError(f"a lobe has {RR_LOBE_SAMPLES} samples")
    _check(load().rr_scene_set_lobe(scene, int(material), _ptr(d)))


def rr_scene_info_get(scene) -> dict:
    info = rr_scene_info()
    _check(load().rr_scene_info_get(scene, C.byref(info)))
    return {k: getattr(info, k) for k, _ in rr_scene_info._fields_ if not k.startswith("reserved")}


def rr_scene_export_bvh(scene, n_triangles: int) -> dict:
    T = int(n_triangles)
    out = dict(morton=np.zeros(T, np.uint32), perm=np.zeros(T, np.uint32),
               children=np.zeros((max(T - 1, 0), 2), np.uint32), parents=np.zeros(max(2 * T - 1, 0), np.uint32),
               boxes=np.zeros((max(T - 1, 0), 2, 6), np.float32))
    _use_torch_stream()
    _check(load().rr_scene_export_bvh(scene, _ptr(out["morton"]), _ptr(out["perm"]), _ptr(out["children"]),
                                      _ptr(out["parents"]), _ptr(out["boxes"])))
    return out


def rr_scene_export_wide(scene, n_triangles: int) -> dict:
    """nodes: [n, 80] uint8 raw node records, tris: [T, 3, 4] float32 in wide-leaf order."""
    _use_torch_stream()
    L = load()
    n = C.c_uint32()
    _check(L.rr_scene_export_wide(scene, None, 0, C.byref(n), None))
    nodes = np.zeros((n.value, WIDE_NODE_BYTES), np.uint8)
    tris = np.zeros((int(n_triangles), 3, 4), np.float32)
    _check(L.rr_scene_export_wide(scene, _ptr(nodes), n.value, C.byref(n), _ptr(tris)))
    return {"nodes": nodes, "tris": tris}


def rr_scan(scene, pose: dict, params: dict, out_polar) -> None:
    _use_torch_stream()
    P, S = make_pose(pose), make_params(params)
    _check(load().rr_scan(scene, C.byref(P), C.byref(S), _ptr(out_polar)))


def rr_scan_async(scene, pose: dict, params: dict, out_polar) -> None:
    _use_torch_stream()
    P, S = make_pose(pose), make_params(params)
    _check(load().rr_scan_async(scene, C.byref(P), C.byref(S), _ptr(out_polar)))


def rr_scan_static(scene, pose: dict, params: dict, out_polar) -> None:
    """rr_scan without allocation: scratch in the library's fixed 64 MiB device
    array, out_polar must be device memory (see include/rr.h)."""
    _use_torch_stream()
    P, S = make_pose(pose), make_params(params)
    _check(load().rr_scan_static(scene, C.byref(P), C.byref(S), _ptr(out_polar)))


def rr_scene_sync(scene) -> None:
    _use_torch_stream()
    _check(load().rr_scene_sync(scene))


def _batch_arrays(poses, params, outs=None):
    n = len(poses)
    if len(params) != n or (outs is not None and len(outs) != n):
        raise ValueError("poses, params and outputs must have the same length")
    P = (rr_pose * n)(*[make_pose(p) for p in poses])
    S = (rr_sensor_params * n)(*[make_params(s) for s in params])
    O = (C.c_void_p * n)(*[_ptr(o) for o in outs]) if outs is not None else None
    return n, P, S, O


def rr_scan_batch(scene, poses, params, outs) -> None:
    _use_torch_stream()
    n, P, S, O = _batch_arrays(poses, params, outs)
    _check(load().rr_scan_batch(scene, n, C.cast(P, C.c_void_p), C.cast(S, C.c_void_p), C.cast(O, C.c_void_p)))


def rr_scan_batch_async(scene, poses, params, outs) -> None:
    """outs: device buffers; errors surface at rr_scene_sync."""
    _use_torch_stream()
    n, P, S, O = _batch_arrays(poses, params, outs)
    _check(load().rr_scan_batch_async(scene, n, C.cast(P, C.c_void_p), C.cast(S, C.c_void_p),
                                      C.cast(O, C.c_void_p)))


def rr_batch_config_get(scene) -> dict:
    c = rr_batch_config()
    _check(load().rr_batch_config_get(scene, C.byref(c)))
    return {k: getattr(c, k) for k, _ in rr_batch_config._fields_ if k != "reserved"}


def rr_batch_config_set(scene, **cfg) -> None:
    """Keyword arguments override the scene's current configuration."""
    cur = rr_batch_config_get(scene)
    unknown = set(cfg) - set(cur)
    if unknown:
        raise ValueError(f"unknown batch config keys {sorted(unknown)}")
    cur.update(cfg)
    c = rr_batch_config(*[int(cur.get(k, 0)) for k, _ in rr_batch_config._fields_])
    _check(load().rr_batch_config_set(scene, C.byref(c)))


def rr_batch_plan(params, config: dict | None = None):
    """Host-only: (first scan of every launch sequence, largest workspace bytes)."""
    n = len(params)
    S = (rr_sensor_params * n)(*[make_params(s) for s in params])
    cfg = None
    if config is not None:
        full = dict(wavefront_rays=0, trace_block=128, trace_blocks_per_sm=0, use_graph=1, node_format=1,
                    refill_threshold=16, workspace_limit=0, split_streams=3, bvh_build=1, query_order=0, reserved=0)
        full.update(config)
        cfg = C.byref(rr_batch_config(*[int(full[k]) for k, _ in rr_batch_config._fields_]))
    cap = max(n, 1)
    first = np.zeros(cap, np.uint32)
    ng, mx = C.c_uint32(), C.c_uint64()
    _check(load().rr_batch_plan(n, C.cast(S, C.c_void_p), cfg, _ptr(first), cap, C.byref(ng), C.byref(mx)))
    return first[: ng.value].copy(), mx.value


def rr_autotune(scene, poses, params, reps: int = 2) -> dict:
    """Returns the chosen configuration with 'best_ms' and 'start_ms'."""
    _use_torch_stream()
    n, P, S, _ = _batch_arrays(poses, params)
    c = rr_batch_config()
    best, start = C.c_float(), C.c_float()
    _check(load().rr_autotune(scene, n, C.cast(P, C.c_void_p), C.cast(S, C.c_void_p), int(reps), C.byref(c),
                              C.byref(best), C.byref(start)))
    out = {k: getattr(c, k) for k, _ in rr_batch_config._fields_}
    out.update(best_ms=best.value, start_ms=start.value)
    return out


def rr_serve_create(**config):
    """Keyword arguments: the rr_serve_config fields (missing ones: library defaults)."""
    unknown = set(config) - {k for k, _ in rr_serve_config._fields_}
    if unknown:
        raise ValueError(f"unknown server config keys {sorted(unknown)}")
    _use_torch_stream()
    c = rr_serve_config(**{k: (float(v) if k == "estimate_factor" else int(v)) for k, v in config.items()})
    h = C.c_void_p()
    _check(load().rr_serve_create(C.byref(c), C.byref(h)))
    return h


def rr_serve_destroy(server) -> None:
    _check(load().rr_serve_destroy(server))


def rr_serve_submit(server, scene, pose: dict, params: dict, out_polar) -> int:
    """Returns the ticket; out_polar must stay alive until the request finishes."""
    P, S = make_pose(pose), make_params(params)
    t = C.c_uint64()
    _check(load().rr_serve_submit(server, scene, C.byref(P), C.byref(S), _ptr(out_polar), C.byref(t)))
    return t.value


def rr_serve_cancel(server, ticket: int) -> bool:
    """True if the request was still queued and is now cancelled (it never
    runs); False if it was already launched or finished (left as it is)."""
    c = C.c_int(0)
    _check(load().rr_serve_cancel(server, int(ticket), C.byref(c)))
    return bool(c.value)


def rr_serve_poll(server, ticket: int) -> bool:
    d = C.c_int()
    _check(load().rr_serve_poll(server, int(ticket), C.byref(d)))
    return bool(d.value)


def rr_serve_wait(server, ticket: int, timeout_ms: int = 60_000) -> None:
    _check(load().rr_serve_wait(server, int(ticket), int(timeout_ms)))


def rr_serve_result(server, ticket: int) -> dict:
    r = rr_serve_record()
    _check(load().rr_serve_result(server, int(ticket), C.byref(r)))
    return {k: getattr(r, k) for k, _ in rr_serve_record._fields_ if k != "reserved"}


def rr_serve_stats_get(server, reset: bool = False) -> dict:
    st = rr_serve_stats()
    _check(load().rr_serve_stats_get(server, C.byref(st), 1 if reset else 0))
    return {k: getattr(st, k) for k, _ in rr_serve_stats._fields_}


def rr_scan_debug(scene, pose: dict, params: dict, out_polar, ray_mask=None, seg_capacity: int = 0,
                  tallies: bool = False):
    """Returns (segments structured array, per-ray tallies [n_az*Ns, 4] or None)."""
    _use_torch_stream()
    P, S = make_pose(pose), make_params(params)
    segs = np.zeros(int(seg_capacity), SEGMENT_DTYPE) if seg_capacity else None
    n0 = params["n_azimuth"] * params["rays_per_beam"]
    tal = np.zeros((n0, 4), np.float32) if tallies else None
    mask = None if ray_mask is None else np.ascontiguousarray(np.asarray(ray_mask, np.uint8).reshape(-1))
    n = C.c_uint64()
    _check(load().rr_scan_debug(scene, C.byref(P), C.byref(S), _ptr(mask), _ptr(out_polar), _ptr(segs),
                                int(seg_capacity), C.byref(n), _ptr(tal)))
    return (segs[: n.value] if segs is not None else None), tal


def rr_accumulate_returns(column, bin_, energy, n_columns: int, n_bins: int, out) -> None:
    """column, bin_ [n] uint32 (column non-decreasing), energy [n] float32;
    out [n_columns, n_bins] float32 (host or device)."""
    _use_torch_stream()
    n = int(column.shape[0])
    _check(load().rr_accumulate_returns(_ptr(column), _ptr(bin_), _ptr(energy), n, int(n_columns), int(n_bins),
                                        _ptr(out)))


def rr_polar_to_db_u8(polar, cutoff_db: float, out) -> None:
    _use_torch_stream()
    _check(load().rr_polar_to_db_u8(_ptr(polar), int(polar.numel()), float(cutoff_db), _ptr(out)))


def rr_scene_stats(scene, reset: bool = False) -> dict:
    st = rr_stats()
    _use_torch_stream()
    _check(load().rr_scene_stats(scene, C.byref(st), 1 if reset else 0))
    return {k: getattr(st, k) for k, _ in rr_stats._fields_}


def rr_profile_enable(scene, on: bool) -> None:
    _use_torch_stream()
    _check(load().rr_profile_enable(scene, 1 if on else 0))


def rr_profile_read(scene, reset: bool = False) -> dict:
    """Per kernel kind: (summed launch ms, launches, busy ms = union of the launch intervals)."""
    pr = rr_profile()
    _check(load().rr_profile_read(scene, C.byref(pr), 1 if reset else 0))
    return {KERNEL_NAMES[k]: (pr.ms[k], pr.launches[k], pr.busy_ms[k]) for k in range(RR_K_COUNT)}

"""Python wrapper of the FP64 brute-force oracle (``rr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path
(the CUDA library and its binding) never imports this module, and this module
imports nothing from the product package.

Inputs are plain numpy arrays and dicts (the shapes produced by the seeded
generators); every float parameter is taken as given (the generators round
them to float32 so that both implementations read identical numbers).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MULTIPATH, REFRACTION, SPECKLE, NOISE, NOISE_PERLIN = 1, 2, 4, 8, 32
NONE = 0xFFFFFFFF


LOBE_EQ5, LOBE_COOK_TORRANCE, LOBE_TABLE = 0, 1, 2
LOBE_CELLS = 2048
LOBE_SAMPLES = 2 * LOBE_CELLS + 1
_LOBE_KINDS = {"eq5": LOBE_EQ5, "cook_torrance": LOBE_COOK_TORRANCE, "table": LOBE_TABLE}


class Material(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("loss_tangent", C.c_double), ("A", C.c_double), ("B", C.c_double),
                ("C", C.c_double), ("pec", C.c_int32), ("lobe", C.c_int32), ("table", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("n_azimuth", C.c_uint32), ("rays_per_beam", C.c_uint32), ("max_bounces", C.c_uint32),
                ("n_bins", C.c_uint32),
                ("beam_width", C.c_double), ("beam_prob", C.c_double), ("elevation", C.c_double),
                ("bin_size", C.c_double), ("t_min", C.c_double), ("min_energy", C.c_double), ("freq_hz", C.c_double),
                ("blur_sigma_bins", C.c_double), ("az_pattern_sigma", C.c_double), ("noise_sys", C.c_double),
                ("noise_amb", C.c_double),
                ("flags", C.c_uint32), ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32), ("scan_id", C.c_uint32),
                ("beam_aspect", C.c_double), ("noise_cell_az", C.c_double), ("noise_cell_bins", C.c_double),
                ("ray_stride", C.c_uint32), ("range_falloff", C.c_double)]


class Pose(C.Structure):
    _fields_ = [("p", C.c_double * 3), ("q", C.c_double * 4)]


SEGMENT_DTYPE = np.dtype([("az", "<u4"), ("k", "<u4"), ("path", "<u4"), ("bounce", "<u4"), ("tri", "<u4"),
                          ("flags", "<u4"), ("t", "<f8"), ("E", "<f8"), ("cos_i", "<f8"), ("ret_t", "<f8"),
                          ("ret_a", "<f8"), ("e_org", "<f8"), ("e_dir", "<f8"), ("alpha2", "<f8")])


def build(force: bool = False) -> str:
    """Compile rr_oracle.c into liboracle.so (OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load(path):
    L = C.CDLL(path)
    if True:
        if True:
            d, u32, p = C.c_double, C.c_uint32, C.c_void_p
            L.orc_philox.argtypes = [p, p, p]
            L.orc_u24.argtypes = [u32]
            L.orc_u24.restype = d
            L.orc_erfinv.argtypes = [d]
            L.orc_erfinv.restype = d
            L.orc_d3_sigma.argtypes = [d, d]
            L.orc_d3_sigma.restype = d
            L.orc_angle.argtypes = [p, p]
            L.orc_angle.restype = d
            L.orc_beam_axis.argtypes = [p, p, u32, p]
            L.orc_d3_ray.argtypes = [p, p, u32, u32, p, p, p, p]
            L.orc_fresnel.argtypes = [d, d, d, p, p, p]
            L.orc_fresnel.restype = C.c_int
            L.orc_reflect.argtypes = [p, p, p]
            L.orc_refract.argtypes = [p, p, d, d, d, p]
            L.orc_int_cospow.argtypes = [d, d, d]
            L.orc_int_cospow.restype = d
            L.orc_brdf_norm.argtypes = [p]
            L.orc_brdf_norm.restype = d
            L.orc_brdf_density.argtypes = [p, d]
            L.orc_brdf_density.restype = d
            L.orc_brdf_window.argtypes = [p, d, d]
            L.orc_brdf_window.restype = d
            L.orc_tri_plane.argtypes = [p, p, p, p, p, p, p, p]
            L.orc_tri_plane.restype = C.c_int
            L.orc_closest.argtypes = [p, u32, p, u32, p, p, d, u32, p, p, p]
            L.orc_closest.restype = C.c_int
            L.orc_scan.argtypes = [p, u32, p, u32, p, p, u32, p, p, p, u32, p, p, p, p, p, p, C.c_uint64, p,
                                   p, C.c_int]
            L.orc_scan.restype = C.c_int
            L.orc_scan_accel.argtypes = L.orc_scan.argtypes + [p, C.c_int]
            L.orc_scan_accel.restype = C.c_int
            L.orc_bvh_build.argtypes = [p, u32, p, u32, p, u32, p, C.c_int]
            L.orc_bvh_build.restype = p
            L.orc_bvh_free.argtypes = [p]
            L.orc_post.argtypes = [p, p, p, u32]
            L.orc_post.restype = C.c_int
            L.orc_db_u8.argtypes = [p, C.c_uint64, d, p]
            L.orc_beckmann.argtypes = [d, d]
            L.orc_beckmann.restype = d
            L.orc_beckmann_norm.argtypes = [d]
            L.orc_beckmann_norm.restype = d
            L.orc_perlin.argtypes = [p, u32, u32, u32]
            L.orc_perlin.restype = d
            L.orc_receive_weight.argtypes = [p, p, u32, p]
            L.orc_receive_weight.restype = d
            L.orc_max_threads.restype = C.c_int
            L.orc_speckle_factor.argtypes = [p, u32, u32, u32, u32, C.c_int]
            L.orc_speckle_factor.restype = d
            L.orc_range_weight.argtypes = [p, d]
            L.orc_range_weight.restype = d
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _vec(x):
    return np.ascontiguousarray(np.asarray(x, np.float64).reshape(3))


# ---------------------------------------------------------------- conversions
def make_material(m: dict) -> Material:
    """Material dict: eps_r, loss_tangent, A, B, C, pec, lobe ("eq5",
    "cook_torrance" or "table") and, for "table", lobe_table (LOBE_SAMPLES
    densities over [0, pi/2])."""
    kind = _LOBE_KINDS[m.get("lobe", "eq5")]
    table = None
    if kind == LOBE_TABLE:
        table = np.ascontiguousarray(np.asarray(m["lobe_table"], np.float64))
        assert table.shape == (LOBE_SAMPLES,)
    out = Material(float(m["eps_r"]), float(m["loss_tangent"]), float(m["A"]), float(m["B"]), float(m["C"]),
                   1 if m.get("pec") else 0, kind, table.ctypes.data if table is not None else None)
    out._table = table   # keeps the samples alive as long as the struct
    return out


def make_params(s: dict) -> Params:
    flags = ((MULTIPATH if s.get("multipath") else 0) | (REFRACTION if s.get("refraction") else 0) |
             (SPECKLE if s.get("speckle") else 0) | (NOISE if s.get("noise") else 0) |
             (NOISE_PERLIN if s.get("perlin") else 0))
    seed = int(s["seed"])
    # 0 selects the defaults: a circular cone, Perlin cells of 8 beams x 32 bins
    return Params(s["n_azimuth"], s["rays_per_beam"], s["max_bounces"], s["n_bins"],
                  s["beam_width"], s["beam_prob"], s["elevation"], s["bin_size"], s["t_min"], s["min_energy"],
                  s["freq_hz"], s["blur_sigma_bins"], s["az_pattern_sigma"], s["noise_sys"], s["noise_amb"],
                  flags, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, int(s["scan_id"]),
                  s.get("beam_aspect") or 1.0, s.get("noise_cell_az") or 8.0, s.get("noise_cell_bins") or 32.0,
                  int(s.get("ray_stride") or 1), float(s.get("range_falloff") or 0.0))


def make_pose(pz: dict) -> Pose:
    P = Pose()
    for i in range(3):
        P.p[i] = float(pz["p"][i])
    for i in range(4):
        P.q[i] = float(pz["q"][i])
    return P


# ---------------------------------------------------------------- primitives
def philox(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, np.uint32))
    k = np.ascontiguousarray(np.asarray(key, np.uint32))
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def u24(x: int) -> float:
    return lib().orc_u24(int(x) & 0xFFFFFFFF)


def erfinv(y: float) -> float:
    return lib().orc_erfinv(float(y))


def d3_sigma(b: float, P: float) -> float:
    return lib().orc_d3_sigma(float(b), float(P))


def angle(a, b) -> float:
    return lib().orc_angle(_ptr(_vec(a)), _ptr(_vec(b)))


def beam_axis(params: dict, pz: dict, a: int):
    pr, po = make_params(params), make_pose(pz)
    out = np.zeros(3)
    lib().orc_beam_axis(C.byref(pr), C.byref(po), a, _ptr(out))
    return out


def d3_ray(params: dict, pz: dict, a: int, k: int):
    pr, po = make_params(params), make_pose(pz)
    o, d = np.zeros(3), np.zeros(3)
    r, w = C.c_double(), C.c_double()
    lib().orc_d3_ray(C.byref(pr), C.byref(po), a, k, _ptr(o), _ptr(d), C.byref(r), C.byref(w))
    return o, d, r.value, w.value


def fresnel(n1, n2, cos_i):
    R, ct, s2 = C.c_double(), C.c_double(), C.c_double()
    tir = lib().orc_fresnel(float(n1), float(n2), float(cos_i), C.byref(R), C.byref(ct), C.byref(s2))
    return R.value, ct.value, bool(tir)


def reflect(d, n):
    out = np.zeros(3)
    lib().orc_reflect(_ptr(_vec(d)), _ptr(_vec(n)), _ptr(out))
    return out


def refract(d, n, eta, cos_i, cos_t):
    out = np.zeros(3)
    lib().orc_refract(_ptr(_vec(d)), _ptr(_vec(n)), float(eta), float(cos_i), float(cos_t), _ptr(out))
    return out


def int_cospow(c, lo, hi):
    return lib().orc_int_cospow(float(c), float(lo), float(hi))


def brdf_norm(m: dict):
    mm = make_material(m)
    return lib().orc_brdf_norm(C.byref(mm))


def brdf_density(m: dict, w: float):
    mm = make_material(m)
    return lib().orc_brdf_density(C.byref(mm), float(w))


def brdf_window(m: dict, w: float, b: float):
    mm = make_material(m)
    return lib().orc_brdf_window(C.byref(mm), float(w), float(b))


def tri_plane(o, d, v0, v1, v2):
    t, b1, b2 = C.c_double(), C.c_double(), C.c_double()
    ok = lib().orc_tri_plane(_ptr(_vec(o)), _ptr(_vec(d)), _ptr(_vec(v0)), _ptr(_vec(v1)), _ptr(_vec(v2)),
                             C.byref(t), C.byref(b1), C.byref(b2))
    return (t.value, b1.value, b2.value) if ok else None


def closest(vertices, triangles, o, d, t_min=1e-4, skip=NONE):
    """Brute-force closest hit of one ray: (tri or None, t, flag bits)."""
    v = np.ascontiguousarray(vertices, np.float32)
    t = np.ascontiguousarray(triangles, np.uint32)
    tri, tt, fl = C.c_uint32(), C.c_double(), C.c_uint32()
    lib().orc_closest(_ptr(v), v.shape[0], _ptr(t), t.shape[0], _ptr(_vec(o)), _ptr(_vec(d)), float(t_min),
                      int(skip), C.byref(tri), C.byref(tt), C.byref(fl))
    return (None if tri.value == NONE else tri.value), tt.value, fl.value


def use_library(path):
    """Switch to another build of the oracle (the mutation tests load planted
    mistakes this way) and return the handle in use before; None restores
    the default build."""
    global _lib
    with _lock:
        prev = _lib
        _lib = _load(path) if path is not None else None
    return prev


def restore_library(handle):
    global _lib
    with _lock:
        _lib = handle


# ---------------------------------------------------------------- CPU BVH
class Bvh:
    """CPU BVH of a scene for ``scan(..., bvh=...)`` (the timed CPU baseline):
    binned-SAH binary tree over grown triangle boxes, plus the window tables
    of the materials for the fast mode.  Built with all host cores.  With
    ``flags`` (default) the boxes are grown so that the scan reproduces the
    brute-force parity flags; without, only the fast mode may use it."""

    def __init__(self, vertices, triangles, materials, flags: bool = True):
        self._lib = lib()
        v = np.ascontiguousarray(vertices, np.float32)
        t = np.ascontiguousarray(triangles, np.uint32)
        made = [make_material(x) for x in materials]
        mats = (Material * len(materials))(*made)
        depth = C.c_uint32()
        self.handle = self._lib.orc_bvh_build(_ptr(v), v.shape[0], _ptr(t), t.shape[0], mats, len(materials),
                                              C.byref(depth), 1 if flags else 0)
        del made
        if not self.handle:
            raise RuntimeError("orc_bvh_build failed (bad indices, no triangles or a tree deeper than its stack)")
        self.depth = depth.value

    def close(self):
        if self.handle:
            self._lib.orc_bvh_free(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


# ---------------------------------------------------------------- full scan
def scan(vertices, triangles, material_ids, materials, pz: dict, params: dict, az_list=None, post: bool = True,
         threads: int = 0, want_segments: bool = True, bvh: Bvh | None = None, fast: bool = False):
    """Run the brute-force scan on the azimuth columns az_list (all if None).

    Returns a dict with ``image`` [n_cols, n_bins] (every return, post pass
    applied when ``post``), ``image_masked`` (returns of flagged initial rays
    left out, post pass applied), ``raw`` / ``raw_masked`` (both before the
    post pass), ``slack`` (energy of unflagged returns next to a bin edge,
    before the post pass), ``flags`` [n_cols, Ns] (1 = initial ray flagged
    for parity), ``tallies`` [n_cols, Ns, 4] (returned, absorbed, escaped,
    terminated), ``segments`` (structured array, SEGMENT_DTYPE) and
    ``counts`` (closest-hit queries, shadow queries, returns).

    With ``bvh`` the queries go through that CPU BVH instead of brute force
    (the same results); ``fast`` then selects the timing mode (tabulated
    beam windows, strict pruning; ``flags``, ``image_masked`` and ``slack``
    are not meaningful)."""
    L = lib()
    v = np.ascontiguousarray(vertices, np.float32)
    t = np.ascontiguousarray(triangles, np.uint32)
    m = np.ascontiguousarray(material_ids, np.uint16)
    made = [make_material(x) for x in materials]   # holds the lobe tables during the call
    mats = (Material * len(materials))(*made)
    pr, po = make_params(params), make_pose(pz)
    if az_list is None:
        cols = None
        n_cols = params["n_azimuth"]
    else:
        cols = np.ascontiguousarray(np.asarray(list(az_list), np.uint32))
        n_cols = int(cols.size)
    ns, nb, nbnc = params["rays_per_beam"], params["n_bins"], params["max_bounces"]
    image = np.zeros((n_cols, nb))
    image_m = np.zeros((n_cols, nb))
    slack = np.zeros((n_cols, nb))
    flags = np.zeros((n_cols, ns), np.uint8)
    tallies = np.zeros((n_cols, ns, 4))
    cap = n_cols * ns * ((1 << nbnc) - 1) if want_segments else 0
    segs = np.zeros(cap, SEGMENT_DTYPE) if want_segments else None
    n_segs = C.c_uint64()
    counts = np.zeros(3, np.uint64)
    rc = L.orc_scan_accel(_ptr(v), v.shape[0], _ptr(t), t.shape[0], _ptr(m), mats, len(materials), C.byref(po),
                          C.byref(pr), _ptr(cols), n_cols, _ptr(image), _ptr(image_m), _ptr(slack), _ptr(flags),
                          _ptr(tallies), _ptr(segs), cap, C.byref(n_segs), _ptr(counts), int(threads),
                          bvh.handle if bvh is not None else None, 1 if fast else 0)
    del made
    if rc != 0:
        raise RuntimeError(f"orc_scan failed with code {rc}")
    raw, raw_m = image.copy(), image_m.copy()
    if post:
        for img in (image, image_m):
            if L.orc_post(_ptr(img), C.byref(pr), _ptr(cols), n_cols) != 0:
                raise RuntimeError("orc_post: the azimuth pattern needs every column")
    # bit 0: a decision float32 can take the other way (paths, energies,
    # images); bit 1: only the per-ray tallies can move past their tolerance
    return dict(image=image, image_masked=image_m, raw=raw, raw_masked=raw_m, slack=slack,
                flags=(flags & 1).astype(np.uint8), tally_flags=(flags != 0).astype(np.uint8),
                tallies=tallies, segments=segs[: n_segs.value] if want_segments else None, counts=counts)


def post(image, params: dict, az_list=None):
    img = np.ascontiguousarray(np.array(image, np.float64))
    pr = make_params(params)
    cols = None if az_list is None else np.ascontiguousarray(np.asarray(az_list, np.uint32))
    n_cols = img.shape[0]
    if lib().orc_post(_ptr(img), C.byref(pr), _ptr(cols), n_cols) != 0:
        raise RuntimeError("orc_post: the azimuth pattern needs every column")
    return img


def bin_returns(column, bin_, energy, n_columns: int, n_bins: int):
    """Sec. III-B: every return adds its energy to the pixel (column, bin) of
    an image that starts at zero; returns past the last bin are dropped.  Each
    pixel is the correctly rounded (double) value of the exact sum of its
    returns (math.fsum, Shewchuk's exact partial sums)."""
    import math
    groups = {}
    for c, b, e in zip(np.asarray(column).tolist(), np.asarray(bin_).tolist(), np.asarray(energy).tolist()):
        if b < n_bins:
            groups.setdefault((c, b), []).append(e)
    out = np.zeros((n_columns, n_bins), np.float64)
    for (c, b), es in groups.items():
        out[c, b] = math.fsum(es)
    return out


def beckmann(t: float, m: float) -> float:
    return lib().orc_beckmann(float(t), float(m))


def beckmann_norm(m: float) -> float:
    return lib().orc_beckmann_norm(float(m))


def receive_weight(params: dict, pz: dict, a: int, pt) -> float:
    """Sec. III-A receive weight of beam a for a return from point pt."""
    return lib().orc_receive_weight(C.byref(make_params(params)), C.byref(make_pose(pz)), a,
                                    _ptr(np.asarray(pt, np.float64)))


def perlin(params: dict, a: int, b: int, purpose: int) -> float:
    """Sec. III-C Perlin noise value in [0, 1] of pixel (a, b); purpose 4 system, 5 ambient."""
    return lib().orc_perlin(C.byref(make_params(params)), a, b, purpose)


def db_u8(image, cutoff_db: float):
    img = np.ascontiguousarray(np.asarray(image, np.float64))
    out = np.zeros(img.shape, np.uint8)
    lib().orc_db_u8(_ptr(img), img.size, float(cutoff_db), _ptr(out))
    return out


def speckle_factor(params: dict, a: int, k: int, path: int, bounce: int, which: int) -> float:
    """Sec. III-C speckle factor of the return `which` (0 traveled path, 1 air
    path) of segment (a, k, path, bounce)."""
    return lib().orc_speckle_factor(C.byref(make_params(params)), a, k, path, bounce, which)


def range_weight(params: dict, r: float) -> float:
    """Optional range weight (1 m / r)^range_falloff of a return at range r."""
    return lib().orc_range_weight(C.byref(make_params(params)), float(r))


def max_threads() -> int:
    return int(lib().orc_max_threads())

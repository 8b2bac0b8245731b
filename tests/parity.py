"""Helpers of the GPU-vs-oracle parity tests.

Tolerances (the parity contract):
  * every initial ray the oracle does not flag has the same segments
    (path, bounce) with the same triangle ids on both sides;
  * every single hit distance t agrees within 1e-5 of itself plus K_SIG
    standard deviations of the float32 hit point over the cosine of the
    incidence (a point moved by dx moves the distance to the plane by up to
    dx / cos theta0).  The standard deviation is the oracle's float32 error
    estimate of the segment (its origin's e_org and direction's e_dir, which
    it carries along the path: the rounding of every hit point, reflection
    and refraction), combined with half an ulp of the scene's largest
    coordinate and an ulp of t, and, for a segment that starts on an
    earlier hit, that hit point's error moved within its plane (its error
    across the ray over the cosine of its incidence).  K_SIG = 4 is the
    oracle's edge-flag threshold (FLAG_SIGMAS); over the full campus scan
    and 4,000 city rays (1.4M segments) the largest GPU deviation measured
    1.7 of these standard deviations, the 99.99th percentile 1.1;
  * the distance along the path from the sensor to every hit (the sum of
    the segment lengths, what the radar's range measures) agrees within
    1e-5 relative plus the sum of those per-segment terms along the path;
  * per-segment energies, cos theta0 and return energies as described in
    compare_segment_energies; per-ray energy tallies within TALLY_REL of the
    initial ray's energy;
  * image bins agree within 1e-3 of the oracle image's maximum plus the
    oracle's per-bin slack (returns next to a bin edge), after masking the
    flagged rays on both sides.

The oracle side is the FP64 brute-force oracle, or, for the full-size scans,
the same oracle with its queries answered through its CPU BVH, which gives
exactly the brute-force results (pinned on the CPU in test_cpu_bvh.py).
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as orc
from paper_2310_03505_gb300 import rr

T_REL = 1e-5
IMG_REL = 1e-3
K_SIG = 4.0
TALLY_REL = 1.6e-5
FLAG_BITS = {"EDGE": 1, "TMIN": 2, "TIE": 4, "TLIM": 8, "TIR": 16, "GRAZE": 32, "RMAX": 64, "VIS": 128,
             "EMIN": 256, "SNELL": 512, "TALLY": 1024, "ERR": 2048}


def gpu_scene(sc):
    import torch
    v = torch.from_numpy(sc.vertices).cuda()
    t = torch.from_numpy(sc.triangles.astype(np.int32)).cuda()
    m = torch.from_numpy(sc.material_ids.astype(np.int16)).cuda()
    h = rr.rr_scene_create(v, t, m, sc.materials)
    for i, mat in enumerate(sc.materials):
        if mat.get("lobe") == "table":
            rr.rr_scene_set_lobe(h, i, np.asarray(mat["lobe_table"], np.float32))
    torch.cuda.synchronize()
    return h


_BVH = {}


def oracle_scan(sc, pz, params, az_list=None, post=True, accel=False):
    """The oracle's scan; accel: through its CPU BVH (flag-exact mode, the
    brute-force results), built once per scene."""
    bvh = None
    if accel:
        key = (sc.name, sc.n_triangles, id(sc.vertices))
        if key not in _BVH:
            _BVH.clear()
            _BVH[key] = orc.Bvh(sc.vertices, sc.triangles, sc.materials)
        bvh = _BVH[key]
    return orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, params, az_list=az_list, post=post,
                    bvh=bvh)


def coord_max(sc, pz):
    """Largest absolute coordinate of the scene and the sensor (metres)."""
    return float(max(np.abs(sc.vertices).max(), np.abs(np.asarray(pz["p"], np.float64)).max(), 1.0))


def flag_census(ora, keep=None):
    """Initial rays removed from the comparisons, by flag kind (a ray counts
    under every kind its tree holds)."""
    segs, fl, tf = ora["segments"], ora["flags"].astype(bool), ora["tally_flags"].astype(bool)
    if keep is not None:
        fl, tf = fl[:, keep], tf[:, keep]
    out = {"rays": int(fl.size), "flagged": int(fl.sum()), "tally_only": int((tf & ~fl).sum())}
    for name, b in FLAG_BITS.items():
        sel = (segs["flags"] & b) != 0
        out[name] = len(set(zip(segs["az"][sel].tolist(), segs["k"][sel].tolist())))
    return out


def compare_tallies(tal_gpu, ora, az_list, rays_per_beam):
    """Per-ray energy tallies (returned, absorbed, escaped, terminated) of the
    rays the oracle does not flag for them, within TALLY_REL of the initial
    ray's energy.  Returns (worst excess over the tolerance, its (column
    index, k))."""
    ok = ora["tally_flags"] == 0
    diff = np.abs(tal_gpu[list(az_list)] - ora["tallies"]).max(-1) * ok
    worst = np.unravel_index(np.argmax(diff), diff.shape)
    return float(diff[worst]) / (TALLY_REL / rays_per_beam), worst


def compare_segment_distances(gpu_segs, ora_segs, ora_flags, az_list, coord_max):
    """Every single hit distance of every unflagged ray (see the module
    notes).  Returns (segments compared, mismatches, largest error over its
    tolerance)."""
    az_list = list(az_list)
    ns = ora_flags.shape[1]
    o, g = _Segs(ora_segs, az_list, ora_flags, coord_max), _Segs(gpu_segs, az_list, ora_flags)
    gi = np.searchsorted(g.key, o.key)
    gi = np.minimum(gi, max(len(g.key) - 1, 0))
    ok = ((g.key[gi] == o.key) if len(g.key) else np.zeros(len(o.key), bool)) & (o.tri != orc.NONE)
    ok &= g.tri[gi] == o.tri if len(g.key) else ok
    t_o = o.s["t"].astype(np.float64)[ok]
    t_g = g.s["t"].astype(np.float64)[gi][ok]
    tol = T_REL * t_o + o.allow[ok]
    r = np.abs(t_g - t_o) / tol
    idx = np.nonzero(ok)[0]
    bad = []
    for j in np.nonzero(r > 1.0)[0][:20]:
        i = idx[j]
        bad.append(f"ray {(az_list[int(o.ray[i]) // ns], int(o.ray[i]) % ns)} seg {(int(o.path[i]), int(o.bounce[i]))}: "
                   f"t {t_g[j]:.9g} vs {t_o[j]:.9g} (tol {tol[j]:.3g}, cos {float(o.s['cos_i'][i]):.4f})")
    return int(ok.sum()), bad, float(r.max()) if r.size else 0.0


def gpu_debug(h, pz, params, mask=None, seg_capacity=None):
    import torch
    out = torch.zeros(params["n_azimuth"], params["n_bins"], device="cuda")
    n0 = params["n_azimuth"] * params["rays_per_beam"]
    cap = seg_capacity or n0 * ((1 << params["max_bounces"]) - 1)
    segs, tal = rr.rr_scan_debug(h, pz, params, out, ray_mask=mask, seg_capacity=cap, tallies=True)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), segs, tal.reshape(params["n_azimuth"], params["rays_per_beam"], 4)


def seg_table(segs, az_set=None):
    """{(az, k): {(path, bounce): (tri, t)}}"""
    tab = {}
    for s in segs:
        az = int(s["az"])
        if az_set is not None and az not in az_set:
            continue
        tab.setdefault((az, int(s["k"])), {})[(int(s["path"]), int(s["bounce"]))] = (int(s["tri"]), float(s["t"]))
    return tab


# energies below this are float32 underflow (a few e-38 and less), not physics:
# rays absorbed by a strongly lossy medium
E_FLOOR = 1e-30


def _ulp32(x):
    """One float32 ulp of |x| (elementwise)."""
    x = np.maximum(np.abs(np.asarray(x, np.float64)), 2.0 ** -126)
    return 2.0 ** (np.floor(np.log2(x)) - 23)


class _Segs:
    """Segments of the rays of az_list that the oracle does not flag, sorted by
    a key (initial ray, path, bounce), with the index of each segment's parent
    and, per segment, the distance along the path from the sensor to its hit
    and the sum of the energies from the initial ray down to it."""

    def __init__(self, segs, az_list, ora_flags, coord_max=None):
        az_list = np.asarray(list(az_list), np.int64)
        col = np.full(int(max(az_list.max(), int(segs["az"].max()) if len(segs) else 0)) + 1, -1, np.int64)
        col[az_list] = np.arange(len(az_list))
        ci = col[segs["az"].astype(np.int64)] if len(segs) else np.zeros(0, np.int64)
        keep = ci >= 0
        k = segs["k"].astype(np.int64)
        keep[keep] &= ora_flags[ci[keep], k[keep]] == 0
        s = segs[keep]
        self.ray = ci[keep] * ora_flags.shape[1] + k[keep]
        self.path = s["path"].astype(np.int64)
        self.bounce = s["bounce"].astype(np.int64)
        self.key = (self.ray << 22) | (self.path << 5) | self.bounce
        order = np.argsort(self.key, kind="stable")
        self.key, self.ray, self.path, self.bounce = self.key[order], self.ray[order], self.path[order], self.bounce[order]
        self.s = s[order]
        self.tri = self.s["tri"].astype(np.int64)
        t = self.s["t"].astype(np.float64)
        E = self.s["E"].astype(np.float64)
        pkey = (self.ray << 22) | ((self.path >> 1) << 5) | (self.bounce - 1)
        pi = np.searchsorted(self.key, pkey)
        pi = np.minimum(pi, len(self.key) - 1) if len(self.key) else pi
        has_parent = (self.bounce > 0) & (len(self.key) > 0)
        if len(self.key):
            has_parent &= self.key[pi] == pkey
        self.parent = np.where(has_parent, pi, -1)
        self.length = np.where(self.tri != orc.NONE, t, 0.0)
        self.along = E.copy()
        # float32 allowance of each hit distance (oracle segments only: they carry the error estimate)
        self.allow = np.zeros(len(self.key))
        if "e_org" in (s.dtype.names or ()) and coord_max is not None:
            hit = self.tri != orc.NONE
            th = np.where(hit, t, 0.0)
            r = 0.5 * _ulp32(coord_max)
            sig = np.sqrt(self.s["e_org"] ** 2 + (th * self.s["e_dir"]) ** 2 + r * r + _ulp32(th) ** 2)
            cos = np.maximum(self.s["cos_i"].astype(np.float64), 1e-3)
            self.allow = np.where(hit, K_SIG * sig / cos, 0.0)
        self.allow_path = self.allow.copy()
        # relative energy allowance from attenuation: a segment inside a lossy
        # medium whose length may move by its distance allowance changes the
        # energy it delivers by 2 alpha times that; the children inherit it
        self.att_own = self.s["alpha2"] * self.allow if "alpha2" in (s.dtype.names or ()) else np.zeros(len(self.key))
        self.att_path = np.zeros(len(self.key))   # over the strict ancestors
        for b in range(1, int(self.bounce.max()) + 1 if len(self.bounce) else 0):
            sel = np.nonzero((self.bounce == b) & (self.parent >= 0))[0]
            self.length[sel] += self.length[self.parent[sel]]
            self.along[sel] += self.along[self.parent[sel]]
            self.allow_path[sel] += self.allow_path[self.parent[sel]]
            self.att_path[sel] = self.att_path[self.parent[sel]] + self.att_own[self.parent[sel]]


def compare_segment_energies(gpu_segs, ora_segs, ora_flags, az_list, rel=1e-3, abs_rel_E=1e-6, coord_max=1.0):
    """Per segment of every unflagged ray: energy entering, cos theta0 and the
    two return energies, within rel of the oracle plus abs_rel_E of the
    energies along the path down to the segment (its own and every
    ancestor's) plus E_FLOOR, plus the attenuation allowance: inside a lossy
    medium the energy a segment delivers is E exp(-2 alpha t), so a length
    that may move by its distance allowance dt (module notes) moves the
    energy by 2 alpha dt of itself, for the segment's returns and for every
    descendant.  The path term: a child's energy is E R minus the returns
    (reading 8), a difference whose FP32 rounding is relative to the
    energies it is taken from -- when the returns take nearly all of E R the
    child is a residue far below them -- and that error then moves down the
    tree scaled by factors <= 1.  Returns a list of mismatch descriptions."""
    az_list = list(az_list)
    o, g = _Segs(ora_segs, az_list, ora_flags, coord_max), _Segs(gpu_segs, az_list, ora_flags)
    gi = np.searchsorted(g.key, o.key)
    gi = np.minimum(gi, max(len(g.key) - 1, 0))
    present = (g.key[gi] == o.key) if len(g.key) else np.zeros(len(o.key), bool)
    bad = []
    for f in ("E", "cos_i", "ret_t", "ret_a"):
        a = g.s[f][gi].astype(np.float64)
        b = o.s[f].astype(np.float64)
        scale = o.s["E"].astype(np.float64) if f == "cos_i" else o.along
        att = 0.0 if f == "cos_i" else (o.att_path if f == "E" else o.att_path + o.att_own)
        off = present & (np.abs(a - b) > (rel + att) * np.abs(b) + abs_rel_E * scale + E_FLOOR)
        for i in np.nonzero(off)[0][:20]:
            az, k = az_list[int(o.ray[i]) // ora_flags.shape[1]], int(o.ray[i]) % ora_flags.shape[1]
            bad.append(f"ray {(az, k)} seg {(int(o.path[i]), int(o.bounce[i]))} {f}: gpu {a[i]:.9g} oracle "
                       f"{b[i]:.9g} (cos_i {float(o.s['cos_i'][i]):.7f})")
        if off.sum() > 20:
            bad.append(f"... {int(off.sum()) - 20} more {f} mismatches")
    return bad


def compare_paths(gpu_segs, ora_segs, ora_flags, az_list, coord_max=1.0):
    """Same segments and triangle ids for every unflagged ray; distance along
    the path to every hit within T_REL relative plus the float32 allowances
    of its segments (module notes).  Returns (n_rays_compared,
    mismatches[list of str], largest path-length error over its tolerance)."""
    az_list = list(az_list)
    ns = ora_flags.shape[1]
    o, g = _Segs(ora_segs, az_list, ora_flags, coord_max), _Segs(gpu_segs, az_list, ora_flags)
    n = int((ora_flags == 0).sum())
    name = lambda r: (az_list[int(r) // ns], int(r) % ns)
    bad = []
    if len(o.key) != len(g.key) or not np.array_equal(o.key, g.key):
        diff = np.setxor1d(o.key, g.key)
        for r in np.unique(diff >> 22)[:20]:
            bad.append(f"ray {name(r)}: segments differ")
        return n, bad, 0.0
    tri_off = np.nonzero(o.tri != g.tri)[0]
    for i in tri_off[:20]:
        bad.append(f"ray {name(o.ray[i])} seg {(int(o.path[i]), int(o.bounce[i]))}: tri {int(g.tri[i])} vs "
                   f"{int(o.tri[i])}")
    hit = (o.tri == g.tri) & (o.tri != orc.NONE)
    rel = np.abs(g.length[hit] - o.length[hit]) / (T_REL * o.length[hit] + o.allow_path[hit])
    max_rel = float(rel.max()) if rel.size else 0.0
    for i in np.nonzero(hit)[0][rel > 1.0][:20]:
        bad.append(f"ray {name(o.ray[i])} seg {(int(o.path[i]), int(o.bounce[i]))}: path length {g.length[i]} vs "
                   f"{o.length[i]} (allowance {T_REL * o.length[i] + o.allow_path[i]:.3g})")
    return n, bad, max_rel


def slack_after_post(ora, params, az_list=None):
    p = dict(params)
    p["noise"] = False
    full = az_list is None
    if not full and p.get("az_pattern_sigma", 0.0) > 0:
        raise ValueError("the beam pattern needs all columns")
    return orc.post(ora["slack"], p, az_list)


def image_excess(img_gpu, img_ora, slack):
    """Largest |gpu - oracle| - slack, relative to the oracle maximum."""
    mx = float(np.max(np.abs(img_ora))) if img_ora.size else 0.0
    excess = np.abs(img_gpu - img_ora) - slack
    return float(np.max(excess)) / max(mx, 1e-300), mx

"""Helpers of the GPU-vs-oracle parity tests.

Tolerances (the parity contract):
  * every initial ray the oracle does not flag has the same segments
    (path, bounce) with the same triangle ids on both sides;
  * the distance along the path from the sensor to every hit (the sum of
    the segment lengths, what the radar's range measures) agrees within
    1e-5 relative -- single segments deep in a path cannot: their end
    points carry the float32 resolution of coordinates ~100 m from the
    origin (7.6e-6 m);
  * image bins agree within 1e-3 of the oracle image's maximum plus the
    oracle's per-bin slack (returns next to a bin edge), after masking the
    flagged rays on both sides.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as orc
from paper_2310_03505_gb300 import rr

T_REL = 1e-5
IMG_REL = 1e-3


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


def oracle_scan(sc, pz, params, az_list=None, post=True):
    return orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, params, az_list=az_list, post=post)


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


def compare_segment_energies(gpu_segs, ora_segs, ora_flags, az_list, rel=1e-3, abs_rel_E=1e-6):
    """Per segment of every unflagged ray: energy entering, cos theta0 and the
    two return energies, within rel of the oracle plus abs_rel_E of the
    energies along the path down to the segment (its own and every
    ancestor's) plus E_FLOOR.  The path term: a child's energy is E R minus
    the returns (reading 8), a difference whose FP32 rounding is relative to
    the energies it is taken from -- when the returns take nearly all of E R
    the child is a residue far below them -- and that error then moves down
    the tree scaled by factors <= 1.  Returns a list of mismatch descriptions."""
    az_index = {az: i for i, az in enumerate(az_list)}
    def table(segs):
        out = {}
        for s in segs:
            az = int(s["az"])
            if az in az_index:
                out[(az, int(s["k"]), int(s["path"]), int(s["bounce"]))] = s
        return out
    g, o = table(gpu_segs), table(ora_segs)
    along = {}   # sum of the oracle energies from the initial ray down to the segment
    for key in sorted(o, key=lambda x: x[3]):
        az, k, path, b = key
        along[key] = float(o[key]["E"]) + (along.get((az, k, path >> 1, b - 1), 0.0) if b > 0 else 0.0)
    bad = []
    for key, os_ in o.items():
        az, k = key[0], key[1]
        if ora_flags[az_index[az], k] or key not in g:
            continue
        gs = g[key]
        for f in ("E", "cos_i", "ret_t", "ret_a"):
            a, b = float(gs[f]), float(os_[f])
            scale = float(os_["E"]) if f == "cos_i" else along[key]
            if abs(a - b) > rel * abs(b) + abs_rel_E * scale + E_FLOOR:
                bad.append(f"ray {key[:2]} seg {key[2:]} {f}: gpu {a:.9g} oracle {b:.9g} (cos_i {float(os_['cos_i']):.7f})")
    return bad


def path_lengths(table):
    """Distance along the path from the sensor to every hit: the sum of the
    segment lengths from the initial ray down to this segment."""
    out = {}
    for ray, segs in table.items():
        for (path, bounce) in sorted(segs, key=lambda x: x[1]):
            tri, t = segs[(path, bounce)]
            prev = out.get((ray, path >> 1, bounce - 1), 0.0) if bounce else 0.0
            out[(ray, path, bounce)] = prev + t
    return out


def compare_paths(gpu_segs, ora_segs, ora_flags, az_list):
    """Same segments and triangle ids for every unflagged ray; distance along
    the path to every hit within T_REL relative.  Returns (n_rays_compared,
    mismatches[list of str], max relative path-length error)."""
    az_list = list(az_list)
    g = seg_table(gpu_segs, set(az_list))
    o = seg_table(ora_segs, set(az_list))
    gl, ol = path_lengths(g), path_lengths(o)
    bad = []
    max_rel = 0.0
    n = 0
    for ci, az in enumerate(az_list):
        for k in range(ora_flags.shape[1]):
            if ora_flags[ci, k]:
                continue
            n += 1
            gs, os_ = g.get((az, k), {}), o.get((az, k), {})
            if set(gs) != set(os_):
                bad.append(f"ray {(az, k)}: segments differ {sorted(set(gs) ^ set(os_))[:4]}")
                continue
            for key, (otri, ot) in os_.items():
                gtri, gt = gs[key]
                if gtri != otri:
                    bad.append(f"ray {(az, k)} seg {key}: tri {gtri} vs {otri}")
                elif otri != orc.NONE:
                    od, gd = ol[((az, k),) + key], gl[((az, k),) + key]
                    rel = abs(gd - od) / od
                    max_rel = max(max_rel, rel)
                    if rel > T_REL:
                        bad.append(f"ray {(az, k)} seg {key}: path length {gd} vs {od}")
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

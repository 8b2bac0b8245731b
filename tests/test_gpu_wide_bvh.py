"""The 8-wide BVH with 8-bit quantised child boxes.

Structure (exported, checked in numpy): every triangle sits in exactly one
leaf slot (a leaf slot holds one triangle or a group of two consecutive
ones; the format has room for three), every decoded bound is an exact float,
every slot's decoded box contains the true box of what it holds and is at
most one quantum looser per side.  Behaviour: a scan traced through the wide
BVH and through the binary
LBVH (float boxes) gives the same segments -- same triangle, same distance,
bit for bit -- for every ray.  Needs a GPU."""
import numpy as np
import pytest

from paper_2310_03505_gb300 import rr, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu


def decode(nodes):
    """Per node: origin P [n,3], scale s [n,3] (float64), imask, first child,
    first triangle, valid mask, q bytes lo/hi [n,3,8]."""
    n = nodes.shape[0]
    w = nodes.view(np.uint32).reshape(n, 20)
    Pn = w[:, 0:3].view(np.float32).astype(np.float64)
    eb = w[:, 3]
    e = np.stack([eb & 0xFF, (eb >> 8) & 0xFF, (eb >> 16) & 0xFF], 1).astype(np.int64) - 127
    s = np.ldexp(1.0, e)
    q = nodes[:, 32:80].reshape(n, 6, 8).astype(np.int64)
    return dict(P=Pn, s=s, imask=(eb >> 24).astype(np.int64), cb=w[:, 4].astype(np.int64),
                tb=w[:, 5].astype(np.int64), valid=w[:, 6].astype(np.int64), counts=w[:, 7].astype(np.int64),
                qlo=q[:, 0:3], qhi=q[:, 3:6])


def check_wide(sc, h):
    ex = rr.rr_scene_export_wide(h, sc.n_triangles)
    nodes, tris = ex["nodes"], ex["tris"]
    info = rr.rr_scene_info_get(h)
    n = nodes.shape[0]
    assert n == info["n_wide_nodes"] and 1 <= n <= max(1, sc.n_triangles - 1)
    # triangles: a permutation of the scene's, with ids and materials
    ids = tris[:, 0, 3].view(np.uint32)
    assert np.array_equal(np.sort(ids), np.arange(sc.n_triangles, dtype=np.uint32))
    src = sc.vertices[sc.triangles[ids]]
    assert np.array_equal(tris[:, :, :3], src)
    assert np.array_equal(tris[:, 1, 3].view(np.uint32), sc.material_ids[ids].astype(np.uint32))
    tri_lo = tris[:, :, :3].min(1).astype(np.float64)
    tri_hi = tris[:, :, :3].max(1).astype(np.float64)
    d = decode(nodes)
    # decoded bounds: P + (2^23 + q) s, exact in float
    lo = d["P"][:, :, None] + (2.0 ** 23 + d["qlo"]) * d["s"][:, :, None]
    hi = d["P"][:, :, None] + (2.0 ** 23 + d["qhi"]) * d["s"][:, :, None]
    for b in (lo, hi):
        assert np.array_equal(b.astype(np.float32).astype(np.float64), b), "a decoded bound is not a float"
    # true boxes bottom up: children are numbered after their parents
    box_lo = np.full((n, 3), np.inf)
    box_hi = np.full((n, 3), -np.inf)
    seen_nodes = np.zeros(n, np.int64)
    seen_tris = np.zeros(sc.n_triangles, np.int64)
    groups = 0
    seen_nodes[0] = 1
    for i in range(n - 1, -1, -1):
        v, im = int(d["valid"][i]), int(d["imask"][i])
        assert im & ~v == 0
        # inner and empty slots hold no triangle count
        for k in range(8):
            if not ((v >> k) & 1) or ((im >> k) & 1):
                assert (int(d["counts"][i]) >> (2 * k)) & 3 == 0
        ri = rl = 0
        for k in range(8):
            if not (v >> k) & 1:
                continue
            if (im >> k) & 1:
                c = int(d["cb"][i]) + ri
                ri += 1
                assert i < c < n
                seen_nodes[c] += 1
                clo, chi = box_lo[c], box_hi[c]
            else:
                # a leaf slot: 1..3 consecutive triangles
                c = (int(d["counts"][i]) >> (2 * k)) & 3
                assert 1 <= c <= 2, f"node {i} slot {k}: {c} triangles"
                groups += c > 1
                j0 = int(d["tb"][i]) + rl
                rl += c
                assert 0 <= j0 and j0 + c <= sc.n_triangles
                seen_tris[j0:j0 + c] += 1
                clo, chi = tri_lo[j0:j0 + c].min(0), tri_hi[j0:j0 + c].max(0)
            qlo, qhi = lo[i, :, k], hi[i, :, k]
            assert np.all(qlo <= clo) and np.all(qhi >= chi), f"node {i} slot {k}: box not contained"
            s = d["s"][i]
            assert np.all(qlo > clo - s) and np.all(qhi < chi + s), f"node {i} slot {k}: looser than a quantum"
            box_lo[i] = np.minimum(box_lo[i], clo)
            box_hi[i] = np.maximum(box_hi[i], chi)
    assert np.all(seen_nodes == 1), "a node is not referenced exactly once"
    assert np.all(seen_tris == 1), "a triangle is not in exactly one leaf slot"
    # depth (stack bound)
    depth = np.zeros(n, np.int64)
    for i in range(n):
        ri = 0
        for k in range(8):
            if (int(d["imask"][i]) >> k) & 1:
                depth[int(d["cb"][i]) + ri] = depth[i] + 1
                ri += 1
    assert depth.max() <= 64
    return n, groups


def test_wide_bvh_structure_tiny(rrlib):
    sc, _, _ = scenes.config_tiny()
    h = P.gpu_scene(sc)
    try:
        n, groups = check_wide(sc, h)
        assert n < sc.n_triangles / 2 and groups > 0
    finally:
        rr.rr_scene_destroy(h)


def test_wide_bvh_structure_campus_after_rebuild(rrlib):
    import torch
    sc, _, _ = scenes.config_medium()
    h = P.gpu_scene(sc)
    try:
        n, groups = check_wide(sc, h)
        # two-triangle groups take the place of many wide nodes
        assert groups > sc.n_triangles / 8 and n < sc.n_triangles / 4
        # a rebuild with moved vertices collapses the new hierarchy
        moved = sc.vertices + np.float32(0.37)
        rr.rr_scene_update_vertices(h, torch.from_numpy(moved).cuda())
        rr.rr_scene_sync(h)
        sc2 = scenes.Scene(sc.name, moved, sc.triangles, sc.material_ids, sc.materials)
        check_wide(sc2, h)
    finally:
        rr.rr_scene_destroy(h)


def test_wide_bvh_single_triangle(rrlib):
    one = scenes.Scene("one", np.array([[5, -1, -1], [5, 1, -1], [5, 0, 1]], np.float32),
                       np.array([[0, 2, 1]], np.uint32), np.zeros(1, np.uint16), [scenes.MATERIALS["metal"]])
    h = P.gpu_scene(one)
    try:
        assert check_wide(one, h) == (1, 0)
    finally:
        rr.rr_scene_destroy(h)


def sorted_segments(segs):
    order = np.lexsort((segs["path"], segs["bounce"], segs["k"], segs["az"]))
    return segs[order]


def segments_with(h, pz, params, fmt, mask=None):
    saved = rr.rr_batch_config_get(h)
    try:
        rr.rr_batch_config_set(h, node_format=fmt)
        img, segs, tal = P.gpu_debug(h, pz, params, mask=mask)
    finally:
        rr.rr_batch_config_set(h, **saved)
    return img, sorted_segments(segs), tal


def assert_same_hits(a, b):
    assert len(a) == len(b)
    for f in ("az", "k", "path", "bounce", "tri", "t", "E", "flags", "cos_i", "ret_t", "ret_a"):
        assert np.array_equal(a[f], b[f]), f"field {f} differs"


@pytest.mark.parametrize("variant", ["plain", "no_multipath"])
def test_wide_and_binary_give_the_same_hits_tiny(rrlib, variant):
    sc, pz, params = scenes.config_tiny()
    if variant == "no_multipath":
        params = scenes.sensor(**{**params, "multipath": False})
    h = P.gpu_scene(sc)
    try:
        iw, sw, tw = segments_with(h, pz, params, rr.RR_NODES_WIDE8)
        ib, sb, tb = segments_with(h, pz, params, rr.RR_NODES_BINARY)
        assert_same_hits(sw, sb)
        assert np.max(np.abs(iw - ib)) <= 1e-6 * ib.max()
        # the wide BVH visits fewer nodes per query
        assert sw["visits"].mean() < 0.5 * sb["visits"].mean()
    finally:
        rr.rr_scene_destroy(h)


def test_wide_and_binary_give_the_same_hits_campus(rrlib):
    """Every segment of the full campus scan (80k initial rays, 5 bounces,
    refraction and multipath on)."""
    sc, pz, params = scenes.config_medium()
    h = P.gpu_scene(sc)
    try:
        _, sw, _ = segments_with(h, pz, params, rr.RR_NODES_WIDE8)
        _, sb, _ = segments_with(h, pz, params, rr.RR_NODES_BINARY)
        assert_same_hits(sw, sb)
        assert sw["visits"].mean() < 0.5 * sb["visits"].mean()
    finally:
        rr.rr_scene_destroy(h)


@pytest.mark.parametrize("fmt", [rr.RR_NODES_BINARY, rr.RR_NODES_WIDE8])
def test_refill_threshold_does_not_change_hits(rrlib, fmt):
    """The query kernels hand new queries to idle lanes at a threshold; the
    results of every query are the same whatever the threshold."""
    sc, pz, params = scenes.config_tiny()
    h = P.gpu_scene(sc)
    saved = rr.rr_batch_config_get(h)
    try:
        ref = None
        for refill in (1, 8, 32):
            rr.rr_batch_config_set(h, node_format=fmt, refill_threshold=refill)
            _, segs, _ = P.gpu_debug(h, pz, params)
            segs = sorted_segments(segs)
            if ref is None:
                ref = segs
            else:
                assert_same_hits(segs, ref)
                assert np.array_equal(segs["visits"], ref["visits"])
    finally:
        rr.rr_batch_config_set(h, **saved)
        rr.rr_scene_destroy(h)


@pytest.mark.parametrize("config", ["tiny", "campus"])
def test_query_order_does_not_change_hits(rrlib, config):
    """The closest-hit queries of bounces >= 1 handed out in bucket order
    (direction octant and origin cell) instead of queue order: every segment
    (triangle, distance, energies, visits) is the same, the image the same
    up to the rounding of the bin sums."""
    sc, pz, params = scenes.config_tiny() if config == "tiny" else scenes.config_medium()
    h = P.gpu_scene(sc)
    saved = rr.rr_batch_config_get(h)
    try:
        out = []
        for order in (rr.RR_ORDER_QUEUE, rr.RR_ORDER_CELL_OCTANT):
            rr.rr_batch_config_set(h, query_order=order)
            img, segs, _ = P.gpu_debug(h, pz, params)
            out.append((img, sorted_segments(segs)))
        assert_same_hits(out[1][1], out[0][1])
        assert np.array_equal(out[1][1]["visits"], out[0][1]["visits"])
        assert np.max(np.abs(out[1][0] - out[0][0])) <= 1e-6 * out[0][0].max()
    finally:
        rr.rr_batch_config_set(h, **saved)
        rr.rr_scene_destroy(h)

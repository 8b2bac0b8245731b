"""LBVH rows on the GPU (ingest, Morton, radix sort, Karras hierarchy,
refit) and the SAH top over the LBVH's subtrees against the CPU reference,
bit for bit, from 2 to 600,000 triangles (the largest with more sort
counters than one block scans in one round trip).  Needs a GPU."""
import numpy as np
import pytest

from oracle import lbvh_ref as L
from paper_2310_03505_gb300 import rr, scenes

pytestmark = pytest.mark.gpu


def soup(n, seed, dup=False):
    rng = np.random.default_rng(seed)
    if dup:
        # few distinct centroids: many equal Morton codes (index tie-break)
        base = rng.uniform(-3, 3, size=(17, 3, 3)).astype(np.float32)
        tri = base[rng.integers(0, 17, size=n)]
    else:
        c = rng.uniform(-50, 50, size=(n, 1, 3))
        tri = (c + rng.normal(scale=0.5, size=(n, 3, 3))).astype(np.float32)
    v = tri.reshape(-1, 3)
    t = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
    m = np.zeros(n, np.uint16)
    return scenes.Scene("soup", v, t, m, [scenes.MATERIALS["metal"]])


CASES = {
    "tiny_room": lambda: scenes.tiny_room(),
    "soup_20k": lambda: soup(20000, 1),
    "soup_dup": lambda: soup(5000, 2, dup=True),
    "soup_ragged": lambda: soup(2049, 3),
    "two": lambda: soup(2, 4),
    # 293 sort tiles: 75,008 counters per pass, scanned by the multi-block counter scan
    "soup_600k": lambda: soup(600000, 9),
}


def check_tree(got, n, leaf_box):
    """A full binary tree over all n leaves with consistent parents and child
    boxes that are the exact unions of their leaves; returns its preorder."""
    ch, par = got["children"], got["parents"]
    enc = L.preorder(ch, n)
    assert sorted(x for x in enc if x >= 0) == list(range(n))
    assert sum(1 for x in enc if x < 0) == n - 1
    if n > 1:
        assert par[0] == 0xFFFFFFFF
        for i in range(n - 1):
            for c in ch[i]:
                c = int(c)
                assert par[(n - 1 + (c & ~L.LEAF)) if c & L.LEAF else c] == i
        assert np.array_equal(got["boxes"], L.refit(ch, leaf_box))
    return enc


@pytest.mark.parametrize("name", sorted(CASES))
def test_lbvh_matches_reference(rrlib, name):
    sc = CASES[name]()
    h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
    try:
        rr.rr_batch_config_set(h, bvh_build=rr.RR_BVH_LBVH)   # rebuilds without the SAH top
        got = rr.rr_scene_export_bvh(h, sc.n_triangles)
        info = rr.rr_scene_info_get(h)
    finally:
        rr.rr_scene_destroy(h)
    codes = L.morton(sc.vertices, sc.triangles)
    skeys, perm = L.sort_codes(codes)
    assert np.array_equal(got["morton"], skeys)
    assert np.array_equal(got["perm"], perm)
    ch, par = L.radix_tree(skeys)
    assert np.array_equal(got["children"], ch)
    assert np.array_equal(got["parents"], par)
    boxes = L.refit(ch, L.leaf_boxes(sc.vertices, sc.triangles, perm))
    assert np.array_equal(got["boxes"], boxes)
    assert info["bvh_depth"] <= 64


def soup_flat(n, seed):
    """A wide flat sheet with tall thin boxes on it: the shape where Morton
    order groups ground with facades."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(-100, 100, size=(n, 1, 3)) * np.array([1.0, 1.0, 0.0])
    tri = g + rng.normal(scale=0.8, size=(n, 3, 3)) * np.array([1.0, 1.0, 0.02])
    k = n // 10
    tri[:k, :, 2] += rng.uniform(0, 25, size=(k, 1))
    tri = tri.astype(np.float32)
    return scenes.Scene("flat", tri.reshape(-1, 3), np.arange(3 * n, dtype=np.uint32).reshape(n, 3),
                        np.zeros(n, np.uint16), [scenes.MATERIALS["metal"]])


SAH_CASES = dict({k: f for k, f in CASES.items() if k != "soup_600k"}, soup_40=lambda: soup(40, 8), soup_flat=lambda: soup_flat(30000, 7),
                 campus=lambda: scenes.campus())


@pytest.mark.parametrize("name", sorted(SAH_CASES))
def test_sah_top_matches_reference(rrlib, name):
    """The default build: the LBVH, then the part above its subtrees of at
    most 32 leaves rebuilt by binned SAH -- the same tree as the host
    restatement of the rules, node for node."""
    sc = SAH_CASES[name]()
    n = sc.n_triangles
    h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
    try:
        assert rr.rr_batch_config_get(h)["bvh_build"] == rr.RR_BVH_SAH_TOP
        got = rr.rr_scene_export_bvh(h, n)
        info = rr.rr_scene_info_get(h)
    finally:
        rr.rr_scene_destroy(h)
    skeys, perm = L.sort_codes(L.morton(sc.vertices, sc.triangles))
    assert np.array_equal(got["morton"], skeys) and np.array_equal(got["perm"], perm)
    ch, _ = L.radix_tree(skeys)
    lb = L.leaf_boxes(sc.vertices, sc.triangles, perm)
    assert check_tree(got, n, lb) == L.sah_top(ch, lb)
    assert info["bvh_depth"] <= 64


def test_update_vertices_matches_fresh_build(rrlib):
    import torch
    sc = soup(3000, 5)
    h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
    try:
        moved = (sc.vertices + np.float32(0.25) * np.sin(sc.vertices)).astype(np.float32)
        rr.rr_scene_update_vertices(h, torch.from_numpy(moved).cuda())
        rr.rr_scene_sync(h)
        got = rr.rr_scene_export_bvh(h, sc.n_triangles)
        rr.rr_batch_config_set(h, bvh_build=rr.RR_BVH_LBVH)
        got_lbvh = rr.rr_scene_export_bvh(h, sc.n_triangles)
    finally:
        rr.rr_scene_destroy(h)
    skeys, perm = L.sort_codes(L.morton(moved, sc.triangles))
    ch, _ = L.radix_tree(skeys)
    lb = L.leaf_boxes(moved, sc.triangles, perm)
    assert np.array_equal(got["morton"], skeys)
    assert check_tree(got, sc.n_triangles, lb) == L.sah_top(ch, lb)
    assert np.array_equal(got_lbvh["children"], ch)
    assert np.array_equal(got_lbvh["boxes"], L.refit(ch, lb))


@pytest.mark.parametrize("config", ["tiny", "campus"])
def test_sah_top_traces_the_same_paths(rrlib, config):
    """Closest hits are unique ((t, triangle id) order) and visibility is a
    yes / no per segment, so both trees give the same ray tree: every
    segment's triangle, distance and energies, bit for bit."""
    if config == "tiny":
        sc, pz, p = scenes.config_tiny()
    else:
        sc, pz, p = scenes.config_medium()
        p = dict(p, n_azimuth=48, rays_per_beam=40)
    h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
    try:
        runs = []
        for build in (rr.RR_BVH_SAH_TOP, rr.RR_BVH_LBVH):
            rr.rr_batch_config_set(h, bvh_build=build)
            out = np.zeros((p["n_azimuth"], p["n_bins"]), np.float32)
            segs, _ = rr.rr_scan_debug(h, pz, p, out, seg_capacity=2_000_000)
            runs.append((segs, out))
    finally:
        rr.rr_scene_destroy(h)
    (sa, ia), (sb, ib) = runs
    assert len(sa) == len(sb) > 0
    sa = sa[np.lexsort((sa["path"], sa["bounce"], sa["k"], sa["az"]))]
    sb = sb[np.lexsort((sb["path"], sb["bounce"], sb["k"], sb["az"]))]
    for f in sa.dtype.names:
        if f != "visits":
            assert np.array_equal(sa[f], sb[f]), f
    assert np.abs(ia - ib).max() <= 1e-5 * np.abs(ib).max()
    if config == "campus":   # the SAH top needs fewer node visits
        assert sa["visits"].mean() < 0.85 * sb["visits"].mean()


def test_invalid_scene_inputs(rrlib):
    sc = soup(10, 6)
    bad = sc.triangles.copy()
    bad[3, 1] = 10 ** 6
    with pytest.raises(rr.RRError) as e:
        rr.rr_scene_create(sc.vertices, bad, sc.material_ids, sc.materials)
    assert e.value.code == rr.RR_ERR_INVALID_ARG
    badm = sc.material_ids.copy()
    badm[0] = 7
    with pytest.raises(rr.RRError) as e:
        rr.rr_scene_create(sc.vertices, sc.triangles, badm, sc.materials)
    assert e.value.code == rr.RR_ERR_INVALID_ARG
    nanv = sc.vertices.copy()
    nanv[4, 2] = np.nan
    with pytest.raises(rr.RRError) as e:
        rr.rr_scene_create(nanv, sc.triangles, sc.material_ids, sc.materials)
    assert e.value.code == rr.RR_ERR_INVALID_ARG
    badmat = [dict(sc.materials[0], A=0.8, B=0.5)]
    with pytest.raises(rr.RRError) as e:
        rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, badmat)
    assert e.value.code == rr.RR_ERR_INVALID_ARG

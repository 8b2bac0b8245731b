"""LBVH rows on the GPU (ingest, Morton, radix sort, Karras hierarchy,
refit) against the CPU reference, bit for bit.  Needs a GPU."""
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
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_lbvh_matches_reference(rrlib, name):
    sc = CASES[name]()
    h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
    try:
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


def test_update_vertices_matches_fresh_build(rrlib):
    import torch
    sc = soup(3000, 5)
    h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
    try:
        moved = (sc.vertices + np.float32(0.25) * np.sin(sc.vertices)).astype(np.float32)
        rr.rr_scene_update_vertices(h, torch.from_numpy(moved).cuda())
        rr.rr_scene_sync(h)
        got = rr.rr_scene_export_bvh(h, sc.n_triangles)
    finally:
        rr.rr_scene_destroy(h)
    skeys, perm = L.sort_codes(L.morton(moved, sc.triangles))
    ch, _ = L.radix_tree(skeys)
    assert np.array_equal(got["morton"], skeys)
    assert np.array_equal(got["children"], ch)
    assert np.array_equal(got["boxes"], L.refit(ch, L.leaf_boxes(moved, sc.triangles, perm)))


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

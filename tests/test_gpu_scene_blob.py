"""Scene serialisation (rr_scene_save / rr_scene_load), needs a GPU.

A scene saved after its vertices moved, with a tabulated lobe and a launch
configuration of its own, loads into a scene with the same configuration,
the same hierarchy node for node and the same scan segments bit for bit
(the build and the scan are deterministic).  Truncated, corrupted or foreign
blobs are refused.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2310_03505_gb300 import rr, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu


def _segments(h, pz, params):
    img = np.zeros((params["n_azimuth"], params["n_bins"]), np.float32)
    n0 = params["n_azimuth"] * params["rays_per_beam"]
    segs, tal = rr.rr_scan_debug(h, pz, params, img, seg_capacity=n0 * (1 << params["max_bounces"]), tallies=True)
    return segs, tal, img


@pytest.fixture(scope="module")
def saved(rrlib):
    sc, pz, params = scenes.config_tiny()
    mats = [sc.materials[0], scenes.tabulated(4.0, 0.01, lambda x: np.cos(x) ** 8 + 0.05, name="tab")]
    h = P.gpu_scene(scenes.Scene(sc.name, sc.vertices, sc.triangles, sc.material_ids, mats))
    moved = sc.vertices + np.float32(0.01) * np.sin(sc.vertices[:, ::-1])
    rr.rr_scene_update_vertices(h, np.ascontiguousarray(moved, np.float32))
    rr.rr_batch_config_set(h, bvh_build=rr.RR_BVH_LBVH, trace_block=128, refill_threshold=8)
    blob = rr.rr_scene_save(h)
    yield h, blob, sc, pz, scenes.sensor(**{**params, "n_azimuth": 64})
    rr.rr_scene_destroy(h)


def test_loaded_scene_equals_the_saved_one(saved):
    h, blob, sc, pz, params = saved
    g = rr.rr_scene_load(blob)
    try:
        assert rr.rr_batch_config_get(g) == rr.rr_batch_config_get(h)
        a, b = rr.rr_scene_export_bvh(h, sc.n_triangles), rr.rr_scene_export_bvh(g, sc.n_triangles)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
        sa, ta, ia = _segments(h, pz, params)
        sb, tb, ib = _segments(g, pz, params)
        assert len(sa) == len(sb) > 0
        for f in sa.dtype.names:
            assert np.array_equal(sa[f], sb[f]), f
        assert np.max(np.abs(ta - tb)) <= 1e-6 * np.abs(ta).max()
        assert np.max(np.abs(ia - ib)) <= 1e-6 * ia.max()
        assert rr.rr_scene_save(g) == blob   # saving the loaded scene gives the same blob
    finally:
        rr.rr_scene_destroy(g)


@pytest.mark.parametrize("damage", ["checksum", "truncated", "magic", "version"])
def test_damaged_blobs_are_refused(saved, damage):
    _, blob, _, _, _ = saved
    b = bytearray(blob)
    if damage == "checksum":
        b[100] ^= 0x40
    elif damage == "truncated":
        b = b[: len(b) - 7]
    elif damage == "magic":
        b[0] ^= 0x01
    else:
        b[8] = 99
    with pytest.raises(rr.RRError) as e:
        rr.rr_scene_load(bytes(b))
    assert e.value.code == rr.RR_ERR_INVALID_ARG


def test_save_reports_the_size_it_needs(saved, rrlib):
    h, blob, _, _, _ = saved
    small = np.zeros(16, np.uint8)
    size = C.c_uint64(0)
    rc = rrlib.rr_scene_save(h, small.ctypes.data, small.size, C.byref(size))
    assert rc == rr.RR_ERR_INVALID_ARG and size.value == len(blob)

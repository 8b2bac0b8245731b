"""The timed CPU baseline: the oracle's physics with its closest-hit and
any-hit queries answered through a CPU BVH (``orc_scan_accel``) instead of
brute force.  Pinned here to give exactly the brute-force oracle's results:
every segment (triangle, distance, energies, flags), every per-ray tally and
parity flag, and every pixel, on the whole tiny scan and on random triangle
soups; the fast timing mode gives the same ray paths and images within
1e-9 of the maximum.  CPU only."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2310_03505_gb300 import scenes

KEYS = ("image", "image_masked", "raw", "raw_masked", "slack", "flags", "tally_flags", "tallies", "counts")


def _both(sc, pz, p, **kw):
    ref = orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, p, **kw)
    bvh = orc.Bvh(sc.vertices, sc.triangles, sc.materials)
    got = orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, p, bvh=bvh, **kw)
    fast = orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, p, bvh=bvh, fast=True, **kw)
    bvh.close()
    return ref, got, fast


def _assert_equal(ref, got):
    for k in KEYS:
        assert np.array_equal(ref[k], got[k]), k
    assert np.array_equal(ref["segments"], got["segments"])


def _assert_fast_close(ref, fast):
    key = lambda s: np.lexsort((s["path"], s["bounce"], s["k"], s["az"]))
    a, b = ref["segments"][key(ref["segments"])], fast["segments"][key(fast["segments"])]
    assert len(a) == len(b)
    for f in ("az", "k", "path", "bounce", "tri", "t", "cos_i"):
        assert np.array_equal(a[f], b[f]), f
    # the beam windows come from tables (cubic Hermite, ~1e-11): energies agree closely, not exactly
    for f in ("E", "ret_t", "ret_a"):
        assert np.allclose(a[f], b[f], rtol=1e-8, atol=1e-14), f
    assert ref["counts"][0] == fast["counts"][0]
    mx = ref["image"].max()
    assert np.abs(fast["image"] - ref["image"]).max() <= 1e-9 * mx
    assert np.abs(fast["tallies"] - ref["tallies"]).max() <= 1e-12


@pytest.mark.parametrize("variant", [{}, dict(speckle=True, seed=0xBEEF), dict(multipath=False, refraction=False),
                                     dict(beam_aspect=2.5, noise=True, noise_sys=1e-4, blur_sigma_bins=1.5)])
def test_whole_tiny_scan_equals_brute_force(variant):
    sc, pz, p = scenes.config_tiny()
    p = scenes.sensor(**{**p, **variant})
    ref, got, fast = _both(sc, pz, p)
    assert ref["image"].max() > 0 and len(ref["segments"]) >= 9600
    _assert_equal(ref, got)
    _assert_fast_close(ref, fast)


def _soup(seed, n_tris, extent, dup=0, axis_aligned=0):
    """Random triangles around a sensor at the origin: arbitrary sizes and
    orientations, some duplicated, some axis aligned (flat boxes)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-extent, extent, (n_tris, 3))
    c[:, 2] = rng.uniform(-2.0, 3.0, n_tris)
    size = 10 ** rng.uniform(-1.0, 0.7, (n_tris, 1, 1))
    v = c[:, None, :] + size * rng.normal(size=(n_tris, 3, 3))
    if axis_aligned:
        v[:axis_aligned, :, 2] = np.round(v[:axis_aligned, :1, 2], 1)
    if dup:
        v[-dup:] = v[:dup]
    verts = v.reshape(-1, 3).astype(np.float32)
    tris = np.arange(3 * n_tris, dtype=np.uint32).reshape(-1, 3)
    mats = [scenes.MATERIALS["metal"], scenes.MATERIALS["dielectric"], scenes.MATERIALS["wood"]]
    mid = rng.integers(0, len(mats), n_tris).astype(np.uint16)
    return scenes.Scene(f"soup{seed}", verts, tris, mid, mats)


@pytest.mark.parametrize("seed,n_tris,dup,flat", [(1, 300, 0, 0), (2, 1500, 40, 200), (3, 4000, 0, 1000)])
def test_random_soups_equal_brute_force(seed, n_tris, dup, flat):
    sc = _soup(seed, n_tris, 12.0, dup, flat)
    pz = scenes.pose(0.0, 0.0, 0.3, 0.4)
    p = scenes.sensor(n_azimuth=48, rays_per_beam=16, max_bounces=4, n_bins=800, bin_size=0.05,
                      multipath=True, refraction=True, seed=0x5EED0 + seed)
    ref, got, fast = _both(sc, pz, p)
    assert ref["counts"][0] > 1000
    _assert_equal(ref, got)
    _assert_fast_close(ref, fast)


@pytest.mark.slow
def test_campus_columns_equal_brute_force():
    """The 200k-triangle campus: four azimuth columns, every 8th initial ray
    with all its bounces, identical through the BVH and by brute force."""
    sc, pz, p = scenes.config_medium()
    p = {**p, "ray_stride": 8}
    ref, got, fast = _both(sc, pz, p, az_list=[3, 137, 250, 333])
    assert ref["counts"][0] > 500
    _assert_equal(ref, got)
    _assert_fast_close(ref, fast)

"""Batched scans (rr_scan_batch and friends) against the same scans run
alone.  Scans of a batch share every launch, so each image may differ from
the scan alone only by the order in which the returns of a bin are added
(shared-memory atomics): the bar is 1e-5 of the image maximum.  The single
scans themselves are held to the oracle by the parity tests.  Needs a GPU."""
import math

import numpy as np
import pytest

from paper_2310_03505_gb300 import rr, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu

BATCH_REL = 1e-5


@pytest.fixture(scope="module")
def tiny_scene(rrlib):
    sc, pz, params = scenes.config_tiny()
    h = P.gpu_scene(sc)
    yield sc, pz, params, h
    rr.rr_scene_destroy(h)


def mixed_tiny_batch(base):
    """Uneven scans of the tiny room: ray counts, bounce limits, bins, flags,
    post passes and poses all differ."""
    variants = [
        dict(rays_per_beam=8),
        dict(rays_per_beam=3, max_bounces=1, n_bins=500, scan_id=1),
        dict(rays_per_beam=17, max_bounces=2, az_pattern_sigma=1.0, blur_sigma_bins=1.0, scan_id=2),
        dict(rays_per_beam=1, n_azimuth=64, multipath=False, scan_id=3),
        dict(rays_per_beam=12, refraction=False, speckle=True, n_bins=1500, bin_size=0.03, scan_id=4),
        dict(rays_per_beam=5, noise=True, noise_sys=1e-4, noise_amb=5e-5, seed=0xABCDEF12345, scan_id=5),
        dict(rays_per_beam=9, n_azimuth=257, az_pattern_sigma=2.0, max_bounces=3, scan_id=6),
        dict(rays_per_beam=30, n_azimuth=100, max_bounces=3, min_energy=1e-4, elevation=math.radians(2.0),
             scan_id=7),
    ]
    params = [scenes.sensor(**{**base, **v}) for v in variants]
    poses = [scenes.pose(0.4 * math.cos(i), 0.4 * math.sin(i), 0.5 + 0.05 * i, yaw=0.3 * i)
             for i in range(len(variants))]
    return poses, params


def alone(h, pz, p):
    import torch
    out = torch.zeros(p["n_azimuth"], p["n_bins"], device="cuda")
    rr.rr_scan(h, pz, p, out)
    return out.cpu().numpy()


def assert_close(img, ref, what):
    mx = float(np.abs(ref).max())
    assert mx > 0, f"{what}: empty image"
    err = float(np.abs(img - ref).max())
    assert err <= BATCH_REL * mx, f"{what}: max |batch - alone| {err:.3g} of image max {mx:.3g}"


def device_outputs(params):
    import torch
    return [torch.zeros(p["n_azimuth"], p["n_bins"], device="cuda") for p in params]


def test_batch_equals_alone(tiny_scene):
    _, _, base, h = tiny_scene
    poses, params = mixed_tiny_batch(base)
    refs = [alone(h, pz, p) for pz, p in zip(poses, params)]
    outs = device_outputs(params)
    rr.rr_scan_batch(h, poses, params, outs)
    for i, (o, r) in enumerate(zip(outs, refs)):
        assert_close(o.cpu().numpy(), r, f"scan {i}")


def test_batch_host_outputs_and_async(tiny_scene):
    import torch
    _, _, base, h = tiny_scene
    poses, params = mixed_tiny_batch(base)
    refs = [alone(h, pz, p) for pz, p in zip(poses, params)]
    # every other output in host memory
    outs = [np.zeros((p["n_azimuth"], p["n_bins"]), np.float32) if i % 2 else
            torch.zeros(p["n_azimuth"], p["n_bins"], device="cuda") for i, p in enumerate(params)]
    rr.rr_scan_batch(h, poses, params, outs)
    for i, (o, r) in enumerate(zip(outs, refs)):
        assert_close(o if isinstance(o, np.ndarray) else o.cpu().numpy(), r, f"scan {i}")
    outs = device_outputs(params)
    rr.rr_scan_batch_async(h, poses, params, outs)
    rr.rr_scene_sync(h)
    for i, (o, r) in enumerate(zip(outs, refs)):
        assert_close(o.cpu().numpy(), r, f"async scan {i}")
    with pytest.raises(rr.RRError):
        rr.rr_scan_batch_async(h, poses[:1], params[:1], [np.zeros((400, 1142), np.float32)])


def test_batch_split_into_sequences_equals_one_sequence(tiny_scene):
    _, _, base, h = tiny_scene
    poses, params = mixed_tiny_batch(base)
    refs = [alone(h, pz, p) for pz, p in zip(poses, params)]
    first, _ = rr.rr_batch_plan(params, dict(wavefront_rays=4000))
    assert len(first) > 3
    saved = rr.rr_batch_config_get(h)
    try:
        rr.rr_batch_config_set(h, wavefront_rays=4000)
        outs = device_outputs(params)
        rr.rr_scan_batch(h, poses, params, outs)
        for i, (o, r) in enumerate(zip(outs, refs)):
            assert_close(o.cpu().numpy(), r, f"scan {i}")
    finally:
        rr.rr_batch_config_set(h, **saved)


def test_graph_replay_reads_new_descriptors(tiny_scene):
    """Two batches of the same shape (so the captured graph is replayed) but
    other poses and seeds: the replay must use the new scans."""
    _, _, base, h = tiny_scene
    poses, params = mixed_tiny_batch(base)
    poses2 = [scenes.pose(-0.3, 0.2 * i - 0.5, 0.6, yaw=-0.2 * i) for i in range(len(poses))]
    params2 = [scenes.sensor(**{**p, "seed": p["seed"] + 99, "scan_id": p["scan_id"] + 100}) for p in params]
    rr.rr_batch_config_set(h, use_graph=1)
    outs = device_outputs(params)
    rr.rr_scan_batch(h, poses, params, outs)
    outs2 = device_outputs(params2)
    rr.rr_scan_batch(h, poses2, params2, outs2)
    for i, (pz, p, o) in enumerate(zip(poses2, params2, outs2)):
        assert_close(o.cpu().numpy(), alone(h, pz, p), f"replayed scan {i}")
    # graph replay off gives the same images
    rr.rr_batch_config_set(h, use_graph=0)
    try:
        outs3 = device_outputs(params2)
        rr.rr_scan_batch(h, poses2, params2, outs3)
        for i, (a, b) in enumerate(zip(outs2, outs3)):
            assert_close(a.cpu().numpy(), b.cpu().numpy(), f"graph off scan {i}")
    finally:
        rr.rr_batch_config_set(h, use_graph=1)


def test_trace_block_sizes_agree(tiny_scene):
    _, _, base, h = tiny_scene
    poses, params = mixed_tiny_batch(base)
    ref = device_outputs(params)
    rr.rr_scan_batch(h, poses, params, ref)
    saved = rr.rr_batch_config_get(h)
    try:
        for block, per_sm in ((64, 0), (256, 0), (128, 2)):
            rr.rr_batch_config_set(h, trace_block=block, trace_blocks_per_sm=per_sm)
            outs = device_outputs(params)
            rr.rr_scan_batch(h, poses, params, outs)
            for i, (a, b) in enumerate(zip(outs, ref)):
                assert_close(a.cpu().numpy(), b.cpu().numpy(), f"block {block}/{per_sm} scan {i}")
    finally:
        rr.rr_batch_config_set(h, **saved)


def test_batch_counters(tiny_scene):
    _, _, base, h = tiny_scene
    poses, params = mixed_tiny_batch(base)
    rr.rr_scene_stats(h, reset=True)
    rr.rr_scan_batch(h, poses, params, device_outputs(params))
    st = rr.rr_scene_stats(h)
    assert st["scans"] == len(params)
    # one launch sequence: raygen, closest-hit query + shade per bounce,
    # visibility preparation + any-hit query from bounce 1 on, bin columns, pattern
    mb = max(p["max_bounces"] for p in params)
    assert st["kernel_launches"] == 2 + 2 * mb + 2 * (mb - 1) + 1
    n0 = sum(p["n_azimuth"] * p["rays_per_beam"] for p in params)
    assert st["closest_queries"] >= n0


def test_autotune(tiny_scene):
    _, _, base, h = tiny_scene
    poses, params = mixed_tiny_batch(base)
    saved = rr.rr_batch_config_get(h)
    try:
        best = rr.rr_autotune(h, poses, params, reps=2)
        assert best["trace_block"] in (64, 128, 256)
        assert 0 < best["best_ms"] <= best["start_ms"] * 1.0001
        assert rr.rr_batch_config_get(h)["trace_block"] == best["trace_block"]
        outs = device_outputs(params)
        rr.rr_scan_batch(h, poses, params, outs)
        for i, (pz, p, o) in enumerate(zip(poses, params, outs)):
            assert_close(o.cpu().numpy(), alone(h, pz, p), f"tuned scan {i}")
    finally:
        rr.rr_batch_config_set(h, **saved)


def test_batch_invalid_arguments(tiny_scene):
    _, pz, base, h = tiny_scene
    good = scenes.sensor(**base)
    bad = scenes.sensor(**{**base, "n_bins": 0})
    with pytest.raises(rr.RRError, match="scan 1"):
        rr.rr_scan_batch(h, [pz, pz], [good, bad], device_outputs([good, good]))
    with pytest.raises(rr.RRError):
        rr.rr_batch_config_set(h, trace_block=100)
    rr.rr_scan_batch(h, [], [], [])   # an empty batch is a no-op


@pytest.fixture(scope="module")
def medium_scene(rrlib):
    sc, pz, params = scenes.config_medium()
    h = P.gpu_scene(sc)
    yield sc, pz, params, h
    rr.rr_scene_destroy(h)


def test_medium_uneven_batch_equals_alone(medium_scene):
    """Campus scans of uneven ray counts (32..512 per beam) and bounce limits."""
    _, pz, base, h = medium_scene
    rng = np.random.default_rng(3)
    params, poses = [], []
    for i in range(6):
        params.append(scenes.sensor(**{**base, "rays_per_beam": int(rng.integers(32, 513)),
                                       "max_bounces": int(rng.integers(3, 6)), "scan_id": i}))
        poses.append(scenes.pose(float(rng.uniform(-4, 4)), float(rng.uniform(-4, 4)), 1.8,
                                 yaw=float(rng.uniform(-math.pi, math.pi))))
    outs = device_outputs(params)
    rr.rr_scan_batch(h, poses, params, outs)
    for i, (p, q, o) in enumerate(zip(poses, params, outs)):
        assert_close(o.cpu().numpy(), alone(h, p, q), f"campus scan {i}")


@pytest.mark.parametrize("variant", ["plain", "noise_blur", "pattern"])
def test_split_scan_equals_whole(tiny_scene, variant):
    """rr_scan / rr_scan_async with split_streams = 2..4 trace the azimuth
    ranges on separate streams: the same image up to the bin sums' rounding
    and exactly the same queries (a beam-pattern scan runs whole)."""
    import torch
    _, pz, base, h = tiny_scene
    extra = {"plain": {}, "noise_blur": dict(noise=True, noise_sys=1e-4, noise_amb=5e-5, blur_sigma_bins=1.5),
             "pattern": dict(az_pattern_sigma=1.0)}[variant]
    p = scenes.sensor(**{**base, **extra, "n_azimuth": 397, "rays_per_beam": 5})
    saved = rr.rr_batch_config_get(h)
    try:
        rr.rr_scene_stats(h, reset=True)
        ref = alone(h, pz, p)
        q_ref = rr.rr_scene_stats(h, reset=True)["closest_queries"]
        for k in (2, 3, 4):
            rr.rr_batch_config_set(h, split_streams=k)
            img = alone(h, pz, p)
            assert rr.rr_scene_stats(h, reset=True)["closest_queries"] == q_ref
            assert_close(img, ref, f"split {k}")
            out = torch.zeros(p["n_azimuth"], p["n_bins"], device="cuda")
            rr.rr_scan_async(h, pz, p, out)
            rr.rr_scene_sync(h)
            assert_close(out.cpu().numpy(), ref, f"async split {k}")
            rr.rr_scene_stats(h, reset=True)
    finally:
        rr.rr_batch_config_set(h, **saved)


def test_profile_busy_time(tiny_scene):
    """rr_profile_read's busy_ms is the union of a kind's launch intervals: on
    one stream the launches of a kind never overlap, so it equals the summed
    durations; split scans overlap their ranges' launches, so it is at most
    that sum."""
    _, pz, base, h = tiny_scene
    p = scenes.sensor(**{**base, "rays_per_beam": 16})
    saved = rr.rr_batch_config_get(h)
    try:
        for k in (1, 3):
            rr.rr_batch_config_set(h, split_streams=k)
            alone(h, pz, p)
            rr.rr_profile_read(h, reset=True)
            rr.rr_profile_enable(h, True)
            for i in range(3):
                alone(h, pz, {**p, "scan_id": i})
            rr.rr_profile_enable(h, False)
            prof = rr.rr_profile_read(h, reset=True)
            ms, launches, busy = prof["trace"]
            assert launches == 3 * k * p["max_bounces"]
            tol = 2e-3 * launches + 1e-3   # event times are kept to about a microsecond
            assert 0.0 < busy <= ms + tol, (k, ms, busy)
            if k == 1:
                for name, (m, n, b) in prof.items():
                    assert abs(b - m) <= 2e-3 * n + 1e-3, (name, m, b)
            assert rr.rr_profile_read(h)["trace"] == (0.0, 0, 0.0)   # the reset cleared it
    finally:
        rr.rr_batch_config_set(h, **saved)

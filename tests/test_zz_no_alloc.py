"""rr_scan_static, the scan entry point that allocates nothing, for callers
that cannot allocate device memory while they run (real-time loops that
must not block on the allocator, programs whose device memory belongs to
another allocator).  Its image must equal rr_scan's on the same scene and
pose, on two calls in a row (the fixed scratch array keeps the previous
call's contents, which must not leak into the next scan).  This file is
named so that pytest collects it last.  Needs a GPU."""
import numpy as np
import pytest

from paper_2310_03505_gb300 import rr, scenes

pytestmark = pytest.mark.gpu


def _scene():
    import torch
    sc, pz, params = scenes.config_tiny()
    v = torch.from_numpy(sc.vertices).cuda()
    return rr.rr_scene_create(v, sc.triangles, sc.material_ids, sc.materials), pz, params


def _pair(h, pz, p, static_first=False):
    """(rr_scan image, rr_scan_static image) of one scan, as numpy arrays."""
    import torch
    shape = (p["n_azimuth"], p["n_bins"])
    ref = torch.zeros(shape, device="cuda")
    got = torch.full(shape, -1.0, device="cuda")
    if static_first:
        rr.rr_scan_static(h, pz, p, got)
        rr.rr_scan(h, pz, p, ref)
    else:
        rr.rr_scan(h, pz, p, ref)
        rr.rr_scan_static(h, pz, p, got)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy()


def test_static_scan_on_a_fresh_scene_allocates_no_workspace(rrlib):
    """The first scan of a new scene through the static entry point leaves the
    scene without a workspace (rr_scan would have grown one), and its image
    equals rr_scan's."""
    import torch
    h, pz, params = _scene()
    try:
        assert rr.rr_scene_info_get(h)["workspace_bytes"] == 0
        p = scenes.sensor(**params)
        got = torch.full((p["n_azimuth"], p["n_bins"]), -1.0, device="cuda")
        rr.rr_scan_static(h, pz, p, got)
        torch.cuda.synchronize()
        assert rr.rr_scene_info_get(h)["workspace_bytes"] == 0
        ref = torch.zeros_like(got)
        rr.rr_scan(h, pz, p, ref)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert r.max() > 0
        assert np.max(np.abs(g - r)) <= 1e-6 * r.max()
    finally:
        rr.rr_scene_destroy(h)


def test_static_scan_matches_rr_scan(rrlib):
    """Two calls in a row, the first the larger one (more rays, bounces and
    bins, multipath on), so that the second, smaller scan would see any
    leftover queue, record or tile flag of the first."""
    import torch
    h, pz, params = _scene()
    try:
        big = dict(rays_per_beam=24, max_bounces=5, n_bins=2000, multipath=True, scan_id=11)
        small = dict(rays_per_beam=8, max_bounces=2, n_bins=600, multipath=False, scan_id=3, noise=True,
                     noise_sys=1e-4, blur_sigma_bins=1.0)
        for call, extra in enumerate((big, small)):
            p = scenes.sensor(**{**params, **extra})
            r, g = _pair(h, pz, p)
            assert r.max() > 0, call
            # the same kernels on the same rays: equal up to the order of float additions
            assert np.max(np.abs(g - r)) <= 1e-6 * r.max(), call
        # a scan whose scratch does not fit the fixed array is refused, with the size in the message
        huge = scenes.sensor(**{**params, "rays_per_beam": 2000, "max_bounces": 8})
        out = torch.zeros(huge["n_azimuth"], huge["n_bins"], device="cuda")
        with pytest.raises(rr.RRError) as e:
            rr.rr_scan_static(h, pz, huge, out)
        assert e.value.code == rr.RR_ERR_INVALID_ARG and "bytes of scratch" in str(e.value)
    finally:
        rr.rr_scene_destroy(h)


def test_static_scan_with_the_wide_node_format_set(rrlib):
    """A scene set to the 8-wide quantised nodes: rr_scan traverses them,
    rr_scan_static the binary nodes (the same closest hits); the images
    agree, with the static call first (before any collapse) and after."""
    h, pz, params = _scene()
    try:
        rr.rr_batch_config_set(h, node_format=rr.RR_NODES_WIDE8)
        p = scenes.sensor(**{**params, "scan_id": 21})
        for static_first in (True, False):
            r, g = _pair(h, pz, p, static_first=static_first)
            assert r.max() > 0
            assert np.max(np.abs(g - r)) <= 1e-6 * r.max(), static_first
    finally:
        rr.rr_scene_destroy(h)

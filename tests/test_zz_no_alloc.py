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


def test_static_scan_matches_rr_scan(rrlib):
    import torch
    sc, pz, params = scenes.config_tiny()
    v = torch.from_numpy(sc.vertices).cuda()
    h = rr.rr_scene_create(v, sc.triangles, sc.material_ids, sc.materials)
    try:
        shape = (params["n_azimuth"], params["n_bins"])
        for call, extra in enumerate(({}, {"scan_id": 3, "noise": True, "noise_sys": 1e-4, "blur_sigma_bins": 1.0})):
            p = scenes.sensor(**{**params, **extra})
            ref = torch.zeros(shape, device="cuda")
            rr.rr_scan(h, pz, p, ref)
            got = torch.full(shape, -1.0, device="cuda")
            rr.rr_scan_static(h, pz, p, got)
            torch.cuda.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            assert r.max() > 0, call
            # the same kernels on the same rays: equal up to the order of float additions
            assert np.max(np.abs(g - r)) <= 1e-6 * r.max(), call
        # a scan whose scratch does not fit the fixed array is refused, with the size in the message
        big = scenes.sensor(**{**params, "rays_per_beam": 2000, "max_bounces": 8})
        out = torch.zeros(big["n_azimuth"], big["n_bins"], device="cuda")
        with pytest.raises(rr.RRError) as e:
            rr.rr_scan_static(h, pz, big, out)
        assert e.value.code == rr.RR_ERR_INVALID_ARG and "bytes of scratch" in str(e.value)
    finally:
        rr.rr_scene_destroy(h)

"""Failure detection without a GPU fault: each bounded device wait of the
library, run by its own kernel on a flag that nothing sets, gives up within
seconds, raises its error bit (RR_ERR_TIMEOUT to the caller), and leaves the
CUDA context usable -- a scan right after it matches the oracle-checked one
from before.  Needs a GPU."""
import numpy as np
import pytest

from paper_2310_03505_gb300 import rr, scenes

pytestmark = pytest.mark.gpu

WAITS = {"top_task": rr.RR_WAIT_TOP_TASK, "wide_node": rr.RR_WAIT_WIDE_NODE,
         "shade_prefix": rr.RR_WAIT_SHADE_PREFIX}


def _scan(h, pz, params):
    img = np.zeros((params["n_azimuth"], params["n_bins"]), np.float32)
    rr.rr_scan(h, pz, params, img)
    return img


def test_bounded_waits_give_up_and_context_survives(rrlib):
    sc, pz, params = scenes.config_tiny()
    params = scenes.sensor(**{**params, "n_azimuth": 32})
    h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
    try:
        before = _scan(h, pz, params)
        assert before.max() > 0
        for name, which in WAITS.items():
            rc, ms = rr.rr_selftest_wait(which)
            assert rc == rr.RR_ERR_TIMEOUT, (name, rc, rrlib.rr_last_error().decode())
            assert 1.0 < ms < 30000.0, (name, ms)
            # the context is still usable: the same scan gives the same image
            # (up to the order of the additions into a bin)
            after = _scan(h, pz, params)
            assert np.max(np.abs(after - before)) <= 1e-5 * before.max(), name
    finally:
        rr.rr_scene_destroy(h)


def test_unknown_wait_is_refused(rrlib):
    rc, _ = rr.rr_selftest_wait(7)
    assert rc == rr.RR_ERR_INVALID_ARG


def test_scene_used_from_another_device_is_refused(rrlib):
    """A scene's buffers live on the device that was current at creation;
    every call that would launch its kernels with another device current is
    refused before anything is queued (nothing runs on the wrong device).
    Needs two GPUs."""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    sc, pz, params = scenes.config_tiny()
    params = scenes.sensor(**{**params, "n_azimuth": 16})
    torch.cuda.set_device(0)
    h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
    try:
        torch.cuda.set_device(1)
        img = np.zeros((params["n_azimuth"], params["n_bins"]), np.float32)
        with pytest.raises(rr.RRError) as e:
            rr.rr_scan(h, pz, params, img)
        assert e.value.code == rr.RR_ERR_INVALID_ARG and "device" in str(e.value)
        out = torch.zeros(params["n_azimuth"], params["n_bins"], device="cuda:1")
        with pytest.raises(rr.RRError) as e:
            rr.rr_scan_static(h, pz, params, out)
        assert e.value.code == rr.RR_ERR_INVALID_ARG
    finally:
        torch.cuda.set_device(0)
        rr.rr_scene_destroy(h)

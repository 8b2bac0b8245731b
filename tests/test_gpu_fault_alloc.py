"""Failure detection by host-side fault injection (needs a GPU).

Every device and pinned host allocation of the library passes one gate, and
rr_fault_inject_alloc can make a chosen one fail as an out-of-memory error
without calling CUDA (no GPU fault is involved).  For each allocation that
creating a scene and scanning it makes, in turn: the failing call reports
RR_ERR_OOM, nothing else breaks, and a scene created afterwards scans to the
same image as before.
"""
import numpy as np
import pytest

from paper_2310_03505_gb300 import rr, scenes

pytestmark = pytest.mark.gpu


def _create_and_scan(sc, pz, params):
    """Scene from host arrays, one scan into a host image, destroyed again."""
    h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
    try:
        img = np.zeros((params["n_azimuth"], params["n_bins"]), np.float32)
        rr.rr_scan(h, pz, params, img)
        return img
    finally:
        rr.rr_scene_destroy(h)


def test_each_allocation_failure_is_reported_and_the_library_recovers(rrlib):
    sc, pz, params = scenes.config_tiny()
    params = scenes.sensor(**{**params, "n_azimuth": 32})
    rr.rr_fault_inject_alloc(-1)
    ref = _create_and_scan(sc, pz, params)   # first use: one-time state made here
    assert ref.max() > 0
    rr.rr_fault_inject_alloc(-1)                     # reset the count
    again = _create_and_scan(sc, pz, params)
    n = rr.rr_fault_inject_alloc(-1)                 # allocations of one create + scan
    assert np.max(np.abs(again - ref)) <= 1e-5 * ref.max()
    assert n >= 10, n
    try:
        for k in range(n):
            rr.rr_fault_inject_alloc(k)
            with pytest.raises(rr.RRError) as err:
                _create_and_scan(sc, pz, params)
            assert err.value.code == rr.RR_ERR_OOM, (k, str(err.value))
            rr.rr_fault_inject_alloc(-1)
            img = _create_and_scan(sc, pz, params)
            assert np.max(np.abs(img - ref)) <= 1e-5 * ref.max(), k
    finally:
        rr.rr_fault_inject_alloc(-1)


def test_injection_past_the_last_allocation_changes_nothing(rrlib):
    sc, pz, params = scenes.config_tiny()
    params = scenes.sensor(**{**params, "n_azimuth": 16})
    rr.rr_fault_inject_alloc(-1)
    ref = _create_and_scan(sc, pz, params)
    rr.rr_fault_inject_alloc(-1)
    _create_and_scan(sc, pz, params)
    n = rr.rr_fault_inject_alloc(1 << 40)            # armed far beyond what one scan allocates
    try:
        img = _create_and_scan(sc, pz, params)
        assert np.max(np.abs(img - ref)) <= 1e-5 * ref.max()
        assert rr.rr_fault_inject_alloc(-1) == n     # the same allocations passed the gate
    finally:
        rr.rr_fault_inject_alloc(-1)

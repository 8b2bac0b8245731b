"""Deferred visibility against the in-order sequence (needs a GPU).

By default the shading pass of a bounce finds the air-path candidates and the
visibility query settles the visible ones afterwards (Sec. III-A: the
children's geometry does not depend on the air-path return, only their
energy).  A min_energy cut makes a child's existence depend on that return,
so launch sequences with a cut keep the in-order sequence (candidates,
visibility, shading).  A cut of the smallest positive float removes only
children of zero energy, so the two sequences must agree on every other
segment: the same triangle and visibility flags, and distances, energies,
returns and image equal up to float rounding.  (The window of a candidate is
computed by the shading kernel instead of the preparation kernel; their
compiled arithmetic may round differently, and a steep lobe turns a one-ulp
angle into a relative change of about 1e-6 of the return.)
"""
import numpy as np
import pytest
import torch

from paper_2310_03505_gb300 import rr, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu

TINY_CUT = float(np.nextafter(np.float32(0), np.float32(1)))   # 1.4e-45


def _run(h, pz, params):
    out = torch.zeros(params["n_azimuth"], params["n_bins"], device="cuda")
    n0 = params["n_azimuth"] * params["rays_per_beam"]
    segs, tal = rr.rr_scan_debug(h, pz, params, out, seg_capacity=n0 * (1 << params["max_bounces"]), tallies=True)
    torch.cuda.synchronize()
    return segs, tal, out.cpu().numpy()


def _by_key(segs):
    key = (segs["az"].astype(np.int64) << 40) | (segs["k"].astype(np.int64) << 24) | \
          (segs["path"].astype(np.int64) << 5) | segs["bounce"].astype(np.int64)
    order = np.argsort(key, kind="stable")
    return key[order], segs[order]


def _compare(h, pz, params):
    assert params.get("multipath", True)
    sa, ta, ia = _run(h, pz, {**params, "min_energy": 0.0})
    sb, tb, ib = _run(h, pz, {**params, "min_energy": TINY_CUT})
    ka, sa = _by_key(sa)
    kb, sb = _by_key(sb)
    assert len(np.unique(ka)) == len(ka) and len(np.unique(kb)) == len(kb)
    # every segment of the cut sequence exists in the deferred one; what only
    # the deferred one traced starts from a child of zero energy
    ia_in = np.isin(ka, kb)
    assert np.isin(kb, ka).all()
    assert np.all(sa["E"][~ia_in] == 0.0)
    a = sa[ia_in]
    assert (a["tri"] == sb["tri"]).all()
    assert ((a["flags"] & 3) == (sb["flags"] & 3)).all()
    assert (a["flags"] & 2).any(), "no visible air-path candidate: the case is not exercised"
    for f in ("t", "E", "cos_i", "ret_t", "ret_a"):
        np.testing.assert_allclose(a[f], sb[f], rtol=1e-4, atol=1e-30, err_msg=f)
    np.testing.assert_allclose(ta, tb, rtol=0, atol=1e-5 * max(float(np.abs(tb).max()), 1e-30))
    np.testing.assert_allclose(ia, ib, rtol=0, atol=1e-5 * float(ib.max()))
    assert ib.max() > 0


def test_deferred_equals_in_order_tiny(rrlib):
    sc, pz, params = scenes.config_tiny()
    h = P.gpu_scene(sc)
    try:
        _compare(h, pz, params)
    finally:
        rr.rr_scene_destroy(h)


def test_deferred_equals_in_order_campus(rrlib):
    sc, pz, params = scenes.config_medium()
    h = P.gpu_scene(sc)
    try:
        _compare(h, pz, scenes.sensor(**{**params, "rays_per_beam": 8}))
    finally:
        rr.rr_scene_destroy(h)

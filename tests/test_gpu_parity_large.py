"""Parity at the full size of the large city workload (about 5M triangles,
400 beams x 1000 rays, at most 8 bounces, 4000 bins): the GPU traces the
whole scan; the FP64 brute-force oracle recomputes a sample of initial rays
-- every 100th ray of 16 azimuth columns, 160 rays with all their bounces,
each ray's tree being independent of the others -- and the two are compared
ray by ray, segment by segment and, through the GPU's ray mask, bin by bin
on the image of exactly those rays.  Properties that hold at any size are
checked on the whole image.  Needs a GPU."""
import numpy as np
import pytest

from paper_2310_03505_gb300 import rr, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu

COLS = list(range(0, 400, 25))
STRIDE = 100


@pytest.fixture(scope="module")
def large(rrlib):
    sc, pz, params = scenes.config_large()
    h = P.gpu_scene(sc)
    yield sc, pz, params, h
    rr.rr_scene_destroy(h)


def test_large_sampled_rays(large):
    sc, pz, params, h = large
    ns = params["rays_per_beam"]
    ora = P.oracle_scan(sc, pz, {**params, "ray_stride": STRIDE}, az_list=COLS)
    keep = np.arange(ns) % STRIDE == 0
    flags = ora["flags"].astype(bool)
    assert flags[:, keep].mean() < 0.05, f"{flags.sum()} of {keep.sum() * len(COLS)} sampled rays flagged"
    skip = flags | ~keep[None, :]   # flagged, or not in the sample
    # every segment is one closest-hit query: size the dump from a plain scan's count
    out = np.zeros((params["n_azimuth"], params["n_bins"]), np.float32)
    rr.rr_scene_stats(h, reset=True)
    rr.rr_scan(h, pz, params, out)
    cap = int(rr.rr_scene_stats(h, reset=True)["closest_queries"]) + 1024
    img_all, segs, tal = P.gpu_debug(h, pz, params, seg_capacity=cap)
    assert np.allclose(img_all, out, rtol=0, atol=1e-5 * float(out.max()))   # the debug scan is the scan
    segs = segs[np.isin(segs["az"], COLS) & (segs["k"] % STRIDE == 0)]
    n, bad, max_rel = P.compare_paths(segs, ora["segments"], skip.astype(np.uint8), COLS)
    assert n == int((~skip).sum()) > 120
    assert not bad, f"{len(bad)} mismatches of {n} rays, first: {bad[:5]}"
    ebad = P.compare_segment_energies(segs, ora["segments"], skip.astype(np.uint8), COLS)
    assert not ebad, f"{len(ebad)} energy mismatches, first: {ebad[:3]}"
    # the image of the sampled, unflagged rays alone: every other ray masked
    mask = np.ones((params["n_azimuth"], ns), np.uint8)
    mask[COLS] = skip
    img, _, _ = P.gpu_debug(h, pz, params, mask=mask, seg_capacity=cap)
    slack = P.slack_after_post(ora, params, COLS)
    excess, mx = P.image_excess(img[COLS], ora["image_masked"], slack)
    assert mx > 0
    assert excess <= P.IMG_REL, f"image excess {excess:.3g} of max {mx:.3g}"
    # at full size: a finite, non-negative image within the returned energy,
    # and energy conserved for every one of the 400,000 initial rays
    assert np.all(np.isfinite(img_all)) and np.all(img_all >= 0)
    assert 0 < img_all.sum() <= tal[..., 0].sum() * (1 + 1e-4)
    assert np.max(np.abs(tal.sum(-1) - 1.0 / ns)) < 1e-4 / ns

"""Parity at the full size of the medium campus workload (about 200k
triangles, 400 beams x 200 rays, 5 bounces, 2000 bins) in the launch
configuration the benchmark times: the GPU traces the whole scan and the FP64
oracle traces every one of its 80,000 initial rays with all their bounces
(its queries answered through its CPU BVH, which gives exactly the
brute-force results).  Compared ray by ray, segment by segment (triangle,
hit distance, energies), per-ray energy tallies, and bin by bin.  Needs a
GPU."""
import numpy as np
import pytest

from paper_2310_03505_gb300 import rr, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def medium(rrlib):
    sc, pz, params = scenes.config_medium()
    h = P.gpu_scene(sc)
    yield sc, pz, params, h
    rr.rr_scene_destroy(h)


@pytest.mark.parametrize("variant", ["bench", "noise_blur"])
def test_medium_full_scan_every_ray(medium, variant):
    sc, pz, params, h = medium
    if variant == "noise_blur":
        params = scenes.sensor(**{**params, "noise": True, "noise_sys": 1e-5, "noise_amb": 1e-5,
                                  "blur_sigma_bins": 1.0, "scan_id": 9})
    cols = range(params["n_azimuth"])
    ns = params["rays_per_beam"]
    ora = P.oracle_scan(sc, pz, params, accel=True)
    flags = ora["flags"]
    census = P.flag_census(ora)
    assert flags.mean() < 0.05, census
    img_all, segs, tal = P.gpu_debug(h, pz, params)
    cmax = P.coord_max(sc, pz)
    n, bad, _ = P.compare_paths(segs, ora["segments"], flags, cols, cmax)
    assert n == int((flags == 0).sum())
    assert not bad, f"{len(bad)} mismatches of {n} rays, first: {bad[:5]}"
    ebad = P.compare_segment_energies(segs, ora["segments"], flags, cols, coord_max=cmax)
    assert not ebad, f"{len(ebad)} segment energy mismatches, first: {ebad[:5]}"
    nd, dbad, worst = P.compare_segment_distances(segs, ora["segments"], flags, cols, cmax)
    assert nd > 500_000 and not dbad, f"{len(dbad)} of {nd} hit distances off (worst {worst:.3g}), first: {dbad[:5]}"
    excess, w = P.compare_tallies(tal, ora, cols, ns)
    assert excess <= 1.0, f"tallies of ray {w}: gpu {tal[w]} oracle {ora['tallies'][w]}"
    # energy bookkeeping holds for every ray of the full scan
    assert np.max(np.abs(tal.sum(-1) - 1.0 / ns)) < 1e-4 / ns
    # the image with the flagged rays masked on both sides
    img, _, _ = P.gpu_debug(h, pz, params, mask=flags)
    slack = P.slack_after_post(ora, params)
    excess, mx = P.image_excess(img, ora["image_masked"], slack)
    assert mx > 0
    assert excess <= P.IMG_REL, f"image excess {excess:.3g} of max {mx:.3g}"


def test_medium_full_scan_properties(medium):
    """Properties that hold at any size, on the whole image: non-negative,
    zero beyond every column's last possible return, total returned energy
    equal to the per-ray tallies."""
    sc, pz, params, h = medium
    img, segs, tal = P.gpu_debug(h, pz, params)
    assert np.all(img >= 0) and np.all(np.isfinite(img))
    # the image holds the returned energy that lands inside the range window
    assert img.sum() <= tal[..., 0].sum() * (1 + 1e-4)
    assert img.sum() > 0.5 * tal[..., 0].sum()
    st = rr.rr_scene_stats(h)
    assert st["closest_queries"] > 0

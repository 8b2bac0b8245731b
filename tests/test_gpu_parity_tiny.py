"""Full-scan parity on the tiny room (400 beams x 8 rays, 3 bounces): the
CUDA path through the C ABI against the FP64 oracle, ray by ray, segment by
segment and bin by bin.  Needs a GPU."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2310_03505_gb300 import rr, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_scene(rrlib):
    sc, pz, params = scenes.config_tiny()
    h = P.gpu_scene(sc)
    yield sc, pz, params, h
    rr.rr_scene_destroy(h)


VARIANTS = {
    "plain": {},
    "noise_blur": dict(noise=True, noise_sys=1e-4, noise_amb=5e-5, blur_sigma_bins=1.5),
    "az_pattern": dict(az_pattern_sigma=1.0, blur_sigma_bins=1.0),
    "no_multipath": dict(multipath=False),
    "no_refraction": dict(refraction=False),
    "speckle": dict(speckle=True),
    "other_seed": dict(seed=0xABCDEF12345, scan_id=7),
    "min_energy": dict(min_energy=1e-4),
    "elliptic": dict(beam_aspect=2.5),
    "range_falloff": dict(range_falloff=2.0),
    "perlin_noise": dict(noise=True, perlin=True, noise_sys=1e-4, noise_amb=5e-5, noise_cell_az=8.0,
                         noise_cell_bins=16.0, blur_sigma_bins=1.0),
}


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_tiny_parity(tiny_scene, variant):
    sc, pz, params, h = tiny_scene
    params = scenes.sensor(**{**params, **VARIANTS[variant]})
    check_parity(sc, pz, params, h)


# lobes other than Eq. 5 (Sec. III-A user BRDFs): the room's dielectric
# with the paper's Cook-Torrance lobe (diffuse 0.2, roughness 0.5) or a
# sharper one, or with a tabulated lobe
LOBE_VARIANTS = {
    "cook_torrance": lambda mats: [mats[0], scenes.cook_torrance(4.0, 0.01, 0.2, 0.5, name="ct")],
    "cook_torrance_sharp": lambda mats: [mats[0], scenes.cook_torrance(4.0, 0.01, 0.1, 0.08, name="ct")],
    "tabulated": lambda mats: [mats[0], scenes.tabulated(
        4.0, 0.01, lambda x: 0.3 + np.exp(-0.5 * (x / 0.12) ** 2) + 0.2 * np.cos(x) ** 4, name="tab")],
}


@pytest.mark.parametrize("variant", sorted(LOBE_VARIANTS))
def test_tiny_parity_lobes(rrlib, variant):
    sc, pz, params = scenes.config_tiny()
    sc = scenes.Scene(sc.name, sc.vertices, sc.triangles, sc.material_ids, LOBE_VARIANTS[variant](sc.materials))
    h = P.gpu_scene(sc)
    try:
        check_parity(sc, pz, params, h)
    finally:
        rr.rr_scene_destroy(h)


def check_parity(sc, pz, params, h, max_flagged=0.02, seg_capacity=None):
    ora = P.oracle_scan(sc, pz, params)
    flags = ora["flags"]
    assert flags.mean() < max_flagged, f"{flags.sum()} of {flags.size} rays flagged"
    # ray paths and hit distances (no mask: every ray traced)
    img_all, segs, tal = P.gpu_debug(h, pz, params, seg_capacity=seg_capacity)
    cmax = P.coord_max(sc, pz)
    n, bad, max_rel = P.compare_paths(segs, ora["segments"], flags, range(params["n_azimuth"]), cmax)
    assert n >= (~flags.astype(bool)).sum()
    assert not bad, f"{len(bad)} mismatches, first: {bad[:5]}"
    assert len(segs) == len(ora["segments"]) or flags.any()
    ebad = P.compare_segment_energies(segs, ora["segments"], flags, range(params["n_azimuth"]), coord_max=cmax)
    assert not ebad, f"{len(ebad)} segment energy mismatches, first: {ebad[:6]}"
    # every single hit distance
    nd, dbad, _ = P.compare_segment_distances(segs, ora["segments"], flags, range(params["n_azimuth"]), cmax)
    assert nd > 0 and not dbad, f"{len(dbad)} of {nd} hit distances off, first: {dbad[:5]}"
    # energy bookkeeping per initial ray
    assert np.max(np.abs(tal.sum(-1) - 1.0 / params["rays_per_beam"])) < 1e-5 / params["rays_per_beam"] * 10
    excess, worst = P.compare_tallies(tal, ora, range(params["n_azimuth"]), params["rays_per_beam"])
    if excess > 1.0:
        az, k = int(worst[0]), int(worst[1])
        g = segs[(segs["az"] == az) & (segs["k"] == k)]
        o = ora["segments"][(ora["segments"]["az"] == az) & (ora["segments"]["k"] == k)]
        raise AssertionError(f"tallies of ray {(az, k)}: gpu {tal[worst]} oracle {ora['tallies'][worst]}\n"
                             f"gpu segments {g}\noracle segments {o}")
    # image with the flagged rays masked on both sides
    img, _, _ = P.gpu_debug(h, pz, params, mask=flags, seg_capacity=seg_capacity)
    slack = P.slack_after_post(ora, params)
    excess, mx = P.image_excess(img, ora["image_masked"], slack)
    assert mx > 0
    assert excess <= P.IMG_REL, f"image excess {excess:.3g} of max {mx:.3g}"


def test_tiny_parity_at_the_bounce_and_bin_limits(tiny_scene):
    """The largest path depth and image the ABI accepts: RR_MAX_BOUNCES
    reflections per path (refraction off, so each hit spawns one child and
    the tree stays one path per ray) into RR_MAX_BINS range bins (717 m of
    range: no path is cut by the range limit), every ray of 64 columns."""
    sc, pz, params, h = tiny_scene
    params = scenes.sensor(**{**params, "n_azimuth": 64, "max_bounces": 16, "n_bins": 16384,
                              "refraction": False})
    # one path per ray: at most 16 segments each
    check_parity(sc, pz, params, h, max_flagged=0.1, seg_capacity=2 * 64 * 8 * 16)


def test_tiny_parity_at_the_ray_limit(tiny_scene):
    """RR_MAX_RAYS_PER_BEAM (65,535) rays in each of 2 beams: the GPU traces
    all 131,070 initial rays; the oracle traces every 257th ray of both
    columns (255 rays with all their bounces), compared ray by ray, segment
    by segment and, with every other ray masked on the GPU, bin by bin;
    energy is conserved for every initial ray."""
    sc, pz, params, h = tiny_scene
    stride = 257
    params = scenes.sensor(**{**params, "n_azimuth": 2, "rays_per_beam": 65535})
    cols = [0, 1]
    ns = params["rays_per_beam"]
    ora = P.oracle_scan(sc, pz, {**params, "ray_stride": stride}, az_list=cols)
    keep = np.arange(ns) % stride == 0
    flags = ora["flags"].astype(bool)
    skip = flags | ~keep[None, :]
    assert flags[:, keep].mean() < 0.05
    img_all, segs, tal = P.gpu_debug(h, pz, params, seg_capacity=4 << 20)
    segs = segs[segs["k"] % stride == 0]
    n, bad, _ = P.compare_paths(segs, ora["segments"], skip.astype(np.uint8), cols, P.coord_max(sc, pz))
    assert n == int((~skip).sum()) > 400
    assert not bad, f"{len(bad)} mismatches of {n} rays, first: {bad[:5]}"
    ebad = P.compare_segment_energies(segs, ora["segments"], skip.astype(np.uint8), cols,
                                      coord_max=P.coord_max(sc, pz))
    assert not ebad, f"{len(ebad)} energy mismatches, first: {ebad[:3]}"
    img, _, _ = P.gpu_debug(h, pz, params, mask=skip.astype(np.uint8), seg_capacity=4 << 20)
    slack = P.slack_after_post(ora, params, cols)
    excess, mx = P.image_excess(img, ora["image_masked"], slack)
    assert mx > 0
    assert excess <= P.IMG_REL, f"image excess {excess:.3g} of max {mx:.3g}"
    assert np.max(np.abs(tal.sum(-1) - 1.0 / ns)) < 1e-4 / ns


def test_tiny_scan_entry_points_agree(tiny_scene):
    """rr_scan (device out), rr_scan (host out), rr_scan_async + sync,
    rr_scan_batch and the debug path give the same image."""
    import torch
    sc, pz, params, h = tiny_scene
    shape = (params["n_azimuth"], params["n_bins"])
    dev = torch.zeros(shape, device="cuda")
    rr.rr_scan(h, pz, params, dev)
    host = np.zeros(shape, np.float32)
    rr.rr_scan(h, pz, params, host)
    asy = torch.zeros(shape, device="cuda")
    rr.rr_scan_async(h, pz, params, asy)
    rr.rr_scene_sync(h)
    b1, b2 = torch.zeros(shape, device="cuda"), np.zeros(shape, np.float32)
    rr.rr_scan_batch(h, [pz, pz], [params, params], [b1, b2])
    dbg, _, _ = P.gpu_debug(h, pz, params)
    ref = dev.cpu().numpy()
    scale = float(ref.max())
    for other in (host, asy.cpu().numpy(), b1.cpu().numpy(), b2, dbg):
        assert np.max(np.abs(other - ref)) <= 1e-6 * scale


def test_tiny_determinism(tiny_scene):
    sc, pz, params, h = tiny_scene
    a, sa, ta = P.gpu_debug(h, pz, params)
    b, sb, tb = P.gpu_debug(h, pz, params)
    # segments are appended in completion order: compare them sorted by ray, bounce and branch
    key = lambda x: np.lexsort((x["path"], x["bounce"], x["k"], x["az"]))
    sa, sb = sa[key(sa)], sb[key(sb)]
    # same rays, same hits, same energies; the node-visit count is a
    # diagnostic that depends on which rays share a warp
    for f in sa.dtype.names:
        if f != "visits":
            assert np.array_equal(sa[f], sb[f]), f
    assert np.max(np.abs(a - b)) <= 1e-6 * a.max()


def test_db_map(tiny_scene):
    import torch
    sc, pz, params, h = tiny_scene
    img = torch.zeros(params["n_azimuth"], params["n_bins"], device="cuda")
    rr.rr_scan(h, pz, params, img)
    out = torch.zeros(img.shape, dtype=torch.uint8, device="cuda")
    rr.rr_polar_to_db_u8(img, 60.0, out)
    g = out.cpu().numpy()
    x = img.cpu().numpy().astype(np.float64)
    o = orc.db_u8(x, 60.0)
    # integer outputs agree except where the float value sits at a rounding edge
    v = np.where(x > 0, 255.0 * (10 * np.log10(np.maximum(x, 1e-300)) + 60.0) / 60.0, 0.0)
    edge = np.abs(v - np.floor(v) - 0.5) < 1e-3
    assert np.array_equal(g[~edge], o[~edge])


def test_empty_and_single_triangle(rrlib):
    import torch
    params = scenes.sensor(n_azimuth=16, rays_per_beam=4, max_bounces=2, n_bins=128, bin_size=0.1,
                           noise=True, noise_sys=0.01, noise_amb=0.0)
    pz = scenes.pose(0, 0, 0)
    one = scenes.Scene("one", np.array([[5, -1, -1], [5, 1, -1], [5, 0, 1]], np.float32),
                       np.array([[0, 2, 1]], np.uint32), np.zeros(1, np.uint16), [scenes.MATERIALS["metal"]])
    empty = scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32), np.zeros(0, np.uint16),
                         [scenes.MATERIALS["metal"]])
    for sc in (empty, one):
        h = rr.rr_scene_create(sc.vertices, sc.triangles, sc.material_ids, sc.materials)
        try:
            img = np.zeros((16, 128), np.float32)
            rr.rr_scan(h, pz, params, img)
        finally:
            rr.rr_scene_destroy(h)
        ora = orc.scan(sc.vertices, sc.triangles, sc.material_ids, sc.materials, pz, params)
        assert np.max(np.abs(img - ora["image"])) <= 1e-3 * max(ora["image"].max(), 1e-30) + 1e-7


def test_invalid_params(tiny_scene):
    sc, pz, params, h = tiny_scene
    out = np.zeros((params["n_azimuth"], params["n_bins"]), np.float32)
    for bad in (dict(n_azimuth=0), dict(max_bounces=17), dict(n_bins=10 ** 6), dict(beam_prob=1.0),
                dict(bin_size=0.0), dict(rays_per_beam=70000), dict(blur_sigma_bins=-1.0)):
        with pytest.raises(rr.RRError) as e:
            rr.rr_scan(h, pz, {**params, **bad}, out)
        assert e.value.code == rr.RR_ERR_INVALID_ARG
    with pytest.raises(rr.RRError):
        rr.rr_scan(h, dict(p=(0, 0, 0), q=(0, 0, 0, 0)), params, out)


def test_capacity_error_reports_size(tiny_scene):
    """A workspace limit below the worst-case ray tree sizes the queues down;
    a scan whose tree then outgrows them fails with RR_ERR_CAPACITY and says
    how much it needed (the kernels drop what does not fit, nothing is
    written out of bounds).  A debug scan with too small a segment buffer
    fails the same way."""
    sc, pz, params, h = tiny_scene
    import torch
    out = torch.zeros(params["n_azimuth"], params["n_bins"], device="cuda")
    with pytest.raises(rr.RRError) as e:
        rr.rr_scan_debug(h, pz, params, out, seg_capacity=10)
    assert e.value.code == rr.RR_ERR_CAPACITY
    saved = rr.rr_batch_config_get(h)
    try:
        # 64 rays per beam: the queues shrink to the 25,600 initial rays,
        # while nearly every ray hits a dielectric wall of the closed room and
        # spawns two children
        rr.rr_batch_config_set(h, workspace_limit=1 << 20)
        with pytest.raises(rr.RRError) as e:
            rr.rr_scan(h, pz, {**params, "rays_per_beam": 64}, out)
        assert e.value.code == rr.RR_ERR_CAPACITY
        assert "were needed" in str(e.value)
    finally:
        rr.rr_batch_config_set(h, **saved)
    # the scene stays usable
    rr.rr_scan(h, pz, params, out)
    assert float(out.max()) > 0


def test_set_lobe_checks_its_arguments(rrlib):
    sc, _, _ = scenes.config_tiny()
    mats = [sc.materials[0], scenes.tabulated(4.0, 0.01, lambda x: np.cos(x), name="tab")]
    h = P.gpu_scene(scenes.Scene(sc.name, sc.vertices, sc.triangles, sc.material_ids, mats))
    try:
        good = np.cos(np.linspace(0, np.pi / 2, rr.RR_LOBE_SAMPLES)).astype(np.float32)
        with pytest.raises(rr.RRError):   # material 0 is not tabulated
            rr.rr_scene_set_lobe(h, 0, good)
        with pytest.raises(rr.RRError):
            rr.rr_scene_set_lobe(h, 2, good)
        with pytest.raises(rr.RRError):
            rr.rr_scene_set_lobe(h, 1, -good)
        with pytest.raises(rr.RRError):
            rr.rr_scene_set_lobe(h, 1, np.zeros(rr.RR_LOBE_SAMPLES, np.float32))
        rr.rr_scene_set_lobe(h, 1, good)
    finally:
        rr.rr_scene_destroy(h)

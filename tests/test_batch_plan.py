"""Host logic of the batched path: how a request of scans is cut into launch
sequences (rr_batch_plan runs on the host only, so these run without a GPU).

The limits come from the device record layout: a return record keys its
image column in 18 bits and its range bin in 14, a ray carries its scan in
16 bits, and queues are sized for the worst-case ray tree (every hit spawning
both children) of the scans traced together."""
import pytest

from paper_2310_03505_gb300 import rr, scenes


@pytest.fixture(scope="module")
def lib():
    from paper_2310_03505_gb300 import build
    build.build()
    return rr.load()


def params(n_az=400, ns=8, bounces=3, bins=1142, **kw):
    p = scenes.sensor(n_azimuth=n_az, rays_per_beam=ns, max_bounces=bounces, n_bins=bins)
    p.update(kw)
    return p


def worst_case_bytes(ps):
    """Workspace of scans traced together, from the queue and record bounds."""
    a256 = lambda x: (x + 255) // 256 * 256
    n0 = sum(p["n_azimuth"] * p["rays_per_beam"] for p in ps)
    q = max(n0, sum(p["n_azimuth"] * p["rays_per_beam"] << (p["max_bounces"] - 1) for p in ps))
    r = sum(2 * p["n_azimuth"] * p["rays_per_beam"] * ((1 << p["max_bounces"]) - 1) for p in ps)
    tmp = sum(p["n_azimuth"] * p["n_bins"] for p in ps if p["az_pattern_sigma"] > 0)
    tiles = (q + 255) // 256 + 1
    desc = len(ps) * 160 + 2 * (len(ps) + 1) * 4
    # ray queues (x2), hits, the list of air-path candidates, records, tile flags, images, descriptors
    return 2 * a256(q * 48) + a256(q * 16) + a256(q * 4) + a256(r * 8) + a256(tiles * 8) + a256(tmp * 4) + a256(desc)


def test_empty_request(lib):
    first, ws = rr.rr_batch_plan([])
    assert len(first) == 0 and ws == 0


def test_one_scan_one_sequence(lib):
    p = params(ns=200, bounces=5, bins=2000)
    first, ws = rr.rr_batch_plan([p])
    assert list(first) == [0]
    assert ws == worst_case_bytes([p])


def test_small_scans_share_one_sequence(lib):
    ps = [params(ns=ns, bounces=b) for ns, b in zip([1, 8, 33, 512, 7], [1, 3, 2, 4, 3])]
    first, ws = rr.rr_batch_plan(ps)
    assert list(first) == [0]
    assert ws == worst_case_bytes(ps)


def test_column_key_limit(lib):
    # 2^18 = 262144 columns: 655 scans of 400 azimuths fit, 656 do not
    ps = [params(ns=1, bounces=1, bins=16) for _ in range(700)]
    first, _ = rr.rr_batch_plan(ps)
    assert list(first) == [0, 655]


def test_scan_index_limit(lib):
    # a ray carries its scan in 16 bits: at most 65535 scans per sequence
    ps = [params(n_az=1, ns=1, bounces=1, bins=1) for _ in range(70000)]
    first, _ = rr.rr_batch_plan(ps)
    assert list(first) == [0, 65535]


def test_wavefront_cap(lib):
    ps = [params(ns=200, bounces=5, bins=2000) for _ in range(7)]   # 80k initial rays each
    first, _ = rr.rr_batch_plan(ps, dict(wavefront_rays=200_000))
    assert list(first) == [0, 2, 4, 6]
    first, _ = rr.rr_batch_plan(ps, dict(wavefront_rays=80_000))
    assert list(first) == list(range(7))


def test_workspace_limit(lib):
    p = params(ns=200, bounces=5, bins=2000)
    one = worst_case_bytes([p])
    three = worst_case_bytes([p] * 3)
    ps = [p] * 7
    first, ws = rr.rr_batch_plan(ps, dict(workspace_limit=three))
    assert list(first) == [0, 3, 6]
    assert ws == three
    first, ws = rr.rr_batch_plan(ps, dict(workspace_limit=one))
    assert list(first) == list(range(7)) and ws == one
    # a scan larger than the limit runs alone with its queues sized down
    first, ws = rr.rr_batch_plan(ps, dict(workspace_limit=one // 2))
    assert list(first) == list(range(7))
    assert ws <= one // 2 + 4096


def test_uneven_request_respects_every_limit(lib):
    import numpy as np
    rng = np.random.default_rng(7)
    ps = [params(ns=int(rng.integers(16, 513)), bounces=int(rng.integers(3, 9)), bins=int(rng.integers(500, 4001)),
                 az_pattern_sigma=float(rng.choice([0.0, 1.5]))) for _ in range(64)]
    limit = 8 << 30
    first, ws = rr.rr_batch_plan(ps, dict(workspace_limit=limit, wavefront_rays=1 << 21))
    bounds = list(first) + [len(ps)]
    assert bounds[0] == 0 and all(a < b for a, b in zip(bounds, bounds[1:]))
    for a, b in zip(bounds, bounds[1:]):
        g = ps[a:b]
        rays = sum(p["n_azimuth"] * p["rays_per_beam"] for p in g)
        if b - a > 1:
            assert rays <= 1 << 21
            assert worst_case_bytes(g) <= limit
        # greedy: the next scan would have broken a limit
        if b < len(ps):
            g2 = ps[a:b + 1]
            rays2 = rays + ps[b]["n_azimuth"] * ps[b]["rays_per_beam"]
            assert rays2 > 1 << 21 or worst_case_bytes(g2) > limit


def test_invalid_config_and_params(lib):
    with pytest.raises(rr.RRError):
        rr.rr_batch_plan([params()], dict(trace_block=96))
    with pytest.raises(rr.RRError):
        rr.rr_batch_plan([params()], dict(use_graph=2))
    with pytest.raises(rr.RRError):
        rr.rr_batch_plan([params()], dict(workspace_limit=1000))
    with pytest.raises(rr.RRError):
        rr.rr_batch_plan([params()], dict(bvh_build=2))
    with pytest.raises(rr.RRError):
        rr.rr_batch_plan([params(), params(bins=0)])

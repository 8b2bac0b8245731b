"""The scan server (rr_serve_*): requests from several client threads over
resident scenes, batched as they arrive and run on overlapping slots.  Each
result must equal the same scan run alone (rr_scan) up to the order of the
float sums in a bin: 1e-5 of the image maximum.  Needs a GPU."""
import math
import threading
import time

import numpy as np
import pytest

from paper_2310_03505_gb300 import rr, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def two_scenes(rrlib):
    room, _, base = scenes.config_tiny()
    yard = scenes.campus(target_tris=50_000, seed=0x5EED0004, n_buildings=60, n_cylinders=150, extent=80.0)
    hs = [P.gpu_scene(room), P.gpu_scene(yard)]
    yield hs, base
    for h in hs:
        rr.rr_scene_destroy(h)


def random_request(rng, base, scene_index):
    p = scenes.sensor(**{**base,
                         "rays_per_beam": int(rng.integers(1, 24)),
                         "max_bounces": int(rng.integers(1, 5)),
                         "n_bins": int(rng.integers(200, 1500)),
                         "n_azimuth": int(rng.choice([64, 200, 400])),
                         "multipath": bool(rng.integers(0, 2)),
                         "refraction": bool(rng.integers(0, 2)),
                         "noise": bool(rng.integers(0, 2)), "noise_sys": 1e-4, "noise_amb": 5e-5,
                         "blur_sigma_bins": float(rng.choice([0.0, 1.0])),
                         "az_pattern_sigma": float(rng.choice([0.0, 1.5])),
                         "seed": int(rng.integers(1, 2 ** 40)), "scan_id": int(rng.integers(0, 2 ** 20))})
    if scene_index == 0:
        pz = scenes.pose(float(rng.uniform(-2, 2)), float(rng.uniform(-2, 2)), 0.5, yaw=float(rng.uniform(-3, 3)))
    else:
        pz = scenes.pose(float(rng.uniform(-3, 3)), float(rng.uniform(-3, 3)), 1.8, yaw=float(rng.uniform(-3, 3)))
    return pz, p


def alone(h, pz, p):
    out = np.zeros((p["n_azimuth"], p["n_bins"]), np.float32)
    rr.rr_scan(h, pz, p, out)
    return out


def assert_close(img, ref, what):
    mx = float(np.abs(ref).max())
    assert mx > 0, what
    err = float(np.abs(img - ref).max())
    assert err <= REL * mx, f"{what}: max |served - alone| {err:.3g} of image max {mx:.3g}"


def test_served_results_equal_alone_in_the_mix(two_scenes):
    import torch
    hs, base = two_scenes
    sv = rr.rr_serve_create(memory_budget=4 << 30, slots=3, max_batch_scans=8)
    try:
        jobs = []
        lock = threading.Lock()

        def client(k):
            rng = np.random.default_rng(100 + k)
            for j in range(12):
                si = int(rng.integers(0, 2))
                pz, p = random_request(rng, base, si)
                shape = (p["n_azimuth"], p["n_bins"])
                out = np.zeros(shape, np.float32) if (j + k) % 2 else torch.zeros(shape, device="cuda")
                t = rr.rr_serve_submit(sv, hs[si], pz, p, out)
                with lock:
                    jobs.append((t, si, pz, p, out))
                time.sleep(float(rng.uniform(0, 0.004)))

        threads = [threading.Thread(target=client, args=(k,)) for k in range(3)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        sizes = []
        for t, si, pz, p, out in jobs:
            rr.rr_serve_wait(sv, t, 60_000)
            rec = rr.rr_serve_result(sv, t)
            assert rec["state"] == rr.RR_REQ_DONE and rec["status"] == rr.RR_OK
            assert rec["submit_ms"] <= rec["start_ms"] <= rec["done_ms"]
            sizes.append(rec["batch_size"])
        torch.cuda.synchronize()
        for t, si, pz, p, out in jobs:
            img = out if isinstance(out, np.ndarray) else out.cpu().numpy()
            assert_close(img, alone(hs[si], pz, p), f"ticket {t} (scene {si})")
        st = rr.rr_serve_stats_get(sv)
        assert st["completed"] == len(jobs) and st["failed"] == 0
        assert st["latency_p50_ms"] > 0 and st["latency_p99_ms"] >= st["latency_p50_ms"]
        assert st["closest_queries"] > 0
    finally:
        rr.rr_serve_destroy(sv)


def test_burst_is_batched(two_scenes):
    """A burst of requests on one scene runs in fewer launch sequences than
    requests (continuous batching), with every result complete."""
    hs, base = two_scenes
    sv = rr.rr_serve_create(memory_budget=2 << 30, slots=1, max_batch_scans=16)
    try:
        rng = np.random.default_rng(7)
        reqs = [random_request(rng, base, 0) for _ in range(40)]
        outs = [np.zeros((p["n_azimuth"], p["n_bins"]), np.float32) for _, p in reqs]
        tickets = [rr.rr_serve_submit(sv, hs[0], pz, p, o) for (pz, p), o in zip(reqs, outs)]
        for t in tickets:
            rr.rr_serve_wait(sv, t, 60_000)
        recs = [rr.rr_serve_result(sv, t) for t in tickets]
        st = rr.rr_serve_stats_get(sv, reset=True)
        assert st["completed"] == 40
        assert st["batches"] < 40
        assert max(r["batch_size"] for r in recs) > 1
        for (pz, p), o in zip(reqs[:6], outs[:6]):
            assert_close(o, alone(hs[0], pz, p), "burst")
        assert rr.rr_serve_stats_get(sv)["completed"] == 0   # the reset started a new window
    finally:
        rr.rr_serve_destroy(sv)


def test_ticket_lifecycle(two_scenes):
    hs, base = two_scenes
    sv = rr.rr_serve_create(memory_budget=1 << 30, slots=2)
    try:
        pz, p = scenes.pose(0.0, 0.0, 0.5), scenes.sensor(**base)
        out = np.zeros((p["n_azimuth"], p["n_bins"]), np.float32)
        t = rr.rr_serve_submit(sv, hs[0], pz, p, out)
        rr.rr_serve_wait(sv, t, 60_000)
        assert rr.rr_serve_poll(sv, t)
        rec = rr.rr_serve_result(sv, t)
        assert rec["state"] == rr.RR_REQ_DONE
        with pytest.raises(rr.RRError):   # a read record is forgotten
            rr.rr_serve_poll(sv, t)
        with pytest.raises(rr.RRError):
            rr.rr_serve_poll(sv, 10 ** 12)
        assert_close(out, alone(hs[0], pz, p), "single")
    finally:
        rr.rr_serve_destroy(sv)


def test_admission_by_memory(two_scenes):
    hs, base = two_scenes
    sv = rr.rr_serve_create(memory_budget=64 << 20, slots=2)
    try:
        big = scenes.sensor(**{**base, "rays_per_beam": 512, "max_bounces": 8})
        out = np.zeros((big["n_azimuth"], big["n_bins"]), np.float32)
        with pytest.raises(rr.RRError) as e:
            rr.rr_serve_submit(sv, hs[0], scenes.pose(0, 0, 0.5), big, out)
        assert e.value.code == rr.RR_ERR_INVALID_ARG and "worst-case" in str(e.value)
        bad = scenes.sensor(**{**base, "n_bins": 0})
        with pytest.raises(rr.RRError):
            rr.rr_serve_submit(sv, hs[0], scenes.pose(0, 0, 0.5), bad, out)
    finally:
        rr.rr_serve_destroy(sv)
    with pytest.raises(rr.RRError):
        rr.rr_serve_create(slots=17)


def test_full_queue_refuses(two_scenes):
    hs, base = two_scenes
    sv = rr.rr_serve_create(memory_budget=1 << 30, slots=1, max_batch_scans=1, max_queue=2)
    try:
        p = scenes.sensor(**{**base, "rays_per_beam": 16})
        pz = scenes.pose(0, 0, 0.5)
        outs, tickets, busy = [], [], 0
        for _ in range(60):
            o = np.zeros((p["n_azimuth"], p["n_bins"]), np.float32)
            try:
                tickets.append(rr.rr_serve_submit(sv, hs[0], pz, p, o))
                outs.append(o)
            except rr.RRError as e:
                assert e.code == rr.RR_ERR_BUSY
                busy += 1
        for t in tickets:
            rr.rr_serve_wait(sv, t, 60_000)
        st = rr.rr_serve_stats_get(sv)
        assert busy > 0 and st["rejected_busy"] == busy
        assert st["completed"] == len(tickets)
    finally:
        rr.rr_serve_destroy(sv)


def test_estimated_batch_that_overflows_is_rerun(two_scenes):
    """Admission by the scene's growth estimate: with an estimate factor far
    too small the second batch on a scene outgrows its workspace; the device
    reports the overflow, the server reruns those requests sized for the
    worst case, and each result still equals the scan alone."""
    import torch
    hs, base = two_scenes
    sv = rr.rr_serve_create(slots=1, memory_budget=2 << 30, estimate_factor=0.01)
    try:
        p = scenes.sensor(**{**base, "rays_per_beam": 8, "max_bounces": 4, "refraction": True, "scan_id": 1})
        pz = scenes.pose(0.3, -0.2, 0.5, yaw=0.4)
        outs = []
        for i in range(3):
            q = {**p, "scan_id": 10 + i}
            out = torch.zeros(q["n_azimuth"], q["n_bins"], device="cuda")
            t = rr.rr_serve_submit(sv, hs[0], pz, q, out)
            rr.rr_serve_wait(sv, t, 60_000)
            assert rr.rr_serve_result(sv, t)["state"] == rr.RR_REQ_DONE
            outs.append((q, out))
        st = rr.rr_serve_stats_get(sv)
        # the first batch seeded the estimate at worst-case size; the next ones overflowed and were rerun
        assert st["retried"] >= 2 and st["failed"] == 0
        for q, out in outs:
            assert_close(out.cpu().numpy(), alone(hs[0], pz, q), f"scan {q['scan_id']}")
    finally:
        rr.rr_serve_destroy(sv)


def test_estimated_admission_batches_more_requests(two_scenes):
    """Requests queued behind a busy slot: sized by the estimate, more of
    them share a launch sequence than under worst-case sizing with the same
    arena, and every result equals the scan alone."""
    import torch
    hs, base = two_scenes
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(24):
        p = scenes.sensor(**{**base, "rays_per_beam": 512, "max_bounces": 6, "refraction": True,
                             "multipath": True, "scan_id": 100 + i})
        pz = scenes.pose(float(rng.uniform(-2, 2)), float(rng.uniform(-2, 2)), 0.5, yaw=float(rng.uniform(-3, 3)))
        reqs.append((pz, p))
    sizes = {}
    for admission in (rr.RR_ADMIT_WORST_CASE, rr.RR_ADMIT_ESTIMATE):
        sv = rr.rr_serve_create(slots=1, memory_budget=6 << 30, admission=admission, max_batch_rays=64 << 20)
        try:
            # one request seeds the estimate
            seed = torch.zeros(base["n_azimuth"], base["n_bins"], device="cuda")
            t0 = rr.rr_serve_submit(sv, hs[0], reqs[0][0], reqs[0][1], seed)
            rr.rr_serve_wait(sv, t0, 60_000)
            rr.rr_serve_result(sv, t0)
            rr.rr_serve_stats_get(sv, reset=True)
            outs, tickets = [], []
            for pz, p in reqs:
                out = torch.zeros(p["n_azimuth"], p["n_bins"], device="cuda")
                tickets.append(rr.rr_serve_submit(sv, hs[0], pz, p, out))
                outs.append(out)
            for t in tickets:
                rr.rr_serve_wait(sv, t, 120_000)
            sizes[admission] = [rr.rr_serve_result(sv, t)["batch_size"] for t in tickets]
            st = rr.rr_serve_stats_get(sv)
            assert st["completed"] == len(reqs) and st["failed"] == 0
            if admission == rr.RR_ADMIT_ESTIMATE:
                for (pz, p), out in zip(reqs, outs):
                    assert_close(out.cpu().numpy(), alone(hs[0], pz, p), f"scan {p['scan_id']}")
        finally:
            rr.rr_serve_destroy(sv)
    assert max(sizes[rr.RR_ADMIT_ESTIMATE]) > max(sizes[rr.RR_ADMIT_WORST_CASE]), sizes


def test_cancel_queued_requests(two_scenes):
    """Requests cancelled while queued never run: their outputs stay as they
    were and they finish as cancelled; the others complete as if alone.  A
    request already launched or finished is not cancelled."""
    hs, base = two_scenes
    sv = rr.rr_serve_create(memory_budget=1 << 30, slots=1, max_batch_scans=1)
    try:
        p = scenes.sensor(**{**base, "rays_per_beam": 16})
        pz = scenes.pose(0, 0, 0.5)
        outs = [np.full((p["n_azimuth"], p["n_bins"]), -1.0, np.float32) for _ in range(24)]
        tickets = [rr.rr_serve_submit(sv, hs[0], pz, p, o) for o in outs]
        cancelled = {t for t in tickets[::2] if rr.rr_serve_cancel(sv, t)}
        assert cancelled, "every request had been launched before the cancel"
        for t in tickets:
            if t in cancelled:
                with pytest.raises(rr.RRError) as e:
                    rr.rr_serve_wait(sv, t, 60_000)
                assert e.value.code == rr.RR_ERR_CANCELLED
                assert rr.rr_serve_poll(sv, t)
            else:
                rr.rr_serve_wait(sv, t, 60_000)
        ref = alone(hs[0], pz, p)
        for t, o in zip(tickets, outs):
            rec = rr.rr_serve_result(sv, t)
            if t in cancelled:
                assert rec["state"] == rr.RR_REQ_CANCELLED and rec["status"] == rr.RR_ERR_CANCELLED
                assert (o == -1.0).all(), "a cancelled request wrote its output"
            else:
                assert rec["state"] == rr.RR_REQ_DONE
                assert_close(o, ref, "not cancelled")
        st = rr.rr_serve_stats_get(sv)
        assert st["cancelled"] == len(cancelled)
        assert st["completed"] == len(tickets) - len(cancelled)
        t = rr.rr_serve_submit(sv, hs[0], pz, p, outs[1])
        rr.rr_serve_wait(sv, t, 60_000)
        assert not rr.rr_serve_cancel(sv, t)   # finished: left as it is
        assert rr.rr_serve_result(sv, t)["state"] == rr.RR_REQ_DONE
        with pytest.raises(rr.RRError):
            rr.rr_serve_cancel(sv, 10 ** 12)
    finally:
        rr.rr_serve_destroy(sv)

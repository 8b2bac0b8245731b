"""Range-bin accumulation (Sec. III-B) through rr_accumulate_returns: the
image kernel of every scan run on given returns.  Its FP32 sums are
compensated, so every pixel stays within a few units in the last place of
the exactly rounded sum (the oracle's math.fsum) however many returns it
gets; a plain FP32 sum of the same returns drifts much further.  Needs a GPU."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2310_03505_gb300 import rr

pytestmark = pytest.mark.gpu

ULPS = 3


def ulp32(x):
    x = np.abs(np.asarray(x, np.float32))
    return np.spacing(np.maximum(x, np.float32(np.finfo(np.float32).tiny)))


def returns(rng, n, n_columns, n_bins, heavy=0):
    col = np.sort(rng.integers(0, n_columns, n)).astype(np.uint32)
    b = rng.integers(0, n_bins + 3, n).astype(np.uint32)   # a few past the last bin
    e = (10.0 ** rng.uniform(-9, 0, n)).astype(np.float32)
    if heavy:   # one pixel with many returns of mixed magnitude
        hc = np.full(heavy, n_columns // 2, np.uint32)
        hb = np.full(heavy, 7, np.uint32)
        he = (rng.uniform(0, 1, heavy) * 10.0 ** rng.uniform(-4, 0, heavy)).astype(np.float32)
        col, b, e = np.concatenate([col, hc]), np.concatenate([b, hb]), np.concatenate([e, he])
        order = np.argsort(col, kind="stable")
        col, b, e = col[order], b[order], e[order]
    return col, b, e


def run(col, b, e, n_columns, n_bins, device=True):
    import torch
    if device:
        out = torch.zeros(n_columns, n_bins, device="cuda")
        rr.rr_accumulate_returns(torch.from_numpy(col).cuda(), torch.from_numpy(b).cuda(),
                                 torch.from_numpy(e).cuda(), n_columns, n_bins, out)
        return out.cpu().numpy()
    out = np.zeros((n_columns, n_bins), np.float32)
    rr.rr_accumulate_returns(col, b, e, n_columns, n_bins, out)
    return out


def test_compensated_sums_match_the_exact_sum(rrlib):
    rng = np.random.default_rng(3)
    n_columns, n_bins = 64, 2000
    col, b, e = returns(rng, 300_000, n_columns, n_bins, heavy=200_000)
    ref = orc.bin_returns(col, b, e, n_columns, n_bins)
    got = run(col, b, e, n_columns, n_bins)
    err = np.abs(got.astype(np.float64) - ref)
    tol = ULPS * ulp32(ref)
    worst = np.unravel_index(np.argmax(err / tol), err.shape)
    assert np.all(err <= tol), f"pixel {worst}: {got[worst]!r} vs {ref[worst]!r}"
    # the heavy pixel: a plain float32 running sum of the same returns is off
    # by far more than the bound the compensated sum meets
    sel = (col == n_columns // 2) & (b == 7)
    naive = np.float32(0)
    for x in e[sel]:
        naive = np.float32(naive + x)
    h = (n_columns // 2, 7)
    assert abs(float(naive) - ref[h]) > 10 * tol[h]


def test_host_buffers_and_edge_cases(rrlib):
    rng = np.random.default_rng(4)
    col, b, e = returns(rng, 5000, 10, 16384)   # the largest bin count: bin 16383 is a pixel
    b[:5] = 16383
    got = run(col, b, e, 10, 16384, device=False)
    ref = orc.bin_returns(col, b, e, 10, 16384)
    assert np.all(np.abs(got - ref) <= ULPS * ulp32(ref))
    # no returns: a zero image
    z = np.zeros(0, np.uint32)
    assert not run(z, z, np.zeros(0, np.float32), 3, 5, device=False).any()
    # a decreasing or out-of-range column is refused
    with pytest.raises(rr.RRError):
        run(np.array([1, 0], np.uint32), np.array([0, 0], np.uint32), np.ones(2, np.float32), 2, 4, device=False)
    with pytest.raises(rr.RRError):
        run(np.array([0, 5], np.uint32), np.array([0, 0], np.uint32), np.ones(2, np.float32), 2, 4, device=False)

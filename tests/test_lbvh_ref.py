"""Pins of the CPU LBVH reference (oracle/lbvh_ref.py): Morton codes by hand,
the stable sort, and the radix-tree property on keys with many duplicates.
CPU only."""
import numpy as np

from oracle import lbvh_ref as L


def test_interleave_by_hand():
    # x = 1 -> bit 2, y = 1 -> bit 1, z = 1 -> bit 0; top bits land at 29, 28, 27
    assert L.interleave_bits(np.array([1]), np.array([0]), np.array([0]))[0] == 0b100
    assert L.interleave_bits(np.array([0]), np.array([1]), np.array([0]))[0] == 0b010
    assert L.interleave_bits(np.array([0]), np.array([0]), np.array([1]))[0] == 0b001
    assert L.interleave_bits(np.array([512]), np.array([0]), np.array([0]))[0] == 1 << 29
    assert L.interleave_bits(np.array([1023]), np.array([1023]), np.array([1023]))[0] == (1 << 30) - 1
    assert L.interleave_bits(np.array([3]), np.array([5]), np.array([6]))[0] == 0b011101110


def test_morton_extremes():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [9, 9, 9], [10, 9, 9], [9, 10, 9]], np.float32)
    t = np.array([[0, 1, 2], [3, 4, 5]], np.uint32)
    m = L.morton(v, t)
    assert m[0] == 0 and m[1] == (1 << 30) - 1


def test_stable_sort():
    codes = np.array([5, 3, 5, 1, 3, 5], np.uint32)
    s, p = L.sort_codes(codes)
    assert list(s) == [1, 3, 3, 5, 5, 5]
    assert list(p) == [3, 1, 4, 0, 2, 5]


def _check_tree(keys, children, parents):
    n = len(keys)
    # every leaf reached exactly once, ranges contiguous, radix property at each split
    ranges = {0: (0, n - 1)}
    leaves = []
    stack = [0]
    while stack:
        i = stack.pop()
        a, b = ranges[i]
        full = [(int(keys[j]) << 32) | j for j in range(a, b + 1)]
        common = 64 - (full[0] ^ full[-1]).bit_length()
        bit = 63 - common            # first bit that differs inside the range
        l, r = int(children[i][0]), int(children[i][1])
        lr = (l & ~L.LEAF, l & ~L.LEAF) if l & L.LEAF else None
        g = (l & ~L.LEAF) if l & L.LEAF else None
        # left child covers a..g where g is the last key with bit == 0
        zeros = [j for j, f in zip(range(a, b + 1), full) if not (f >> bit) & 1]
        ones = [j for j, f in zip(range(a, b + 1), full) if (f >> bit) & 1]
        assert zeros and ones and max(zeros) + 1 == min(ones)
        split = max(zeros)
        for ch, (ca, cb) in ((l, (a, split)), (r, (split + 1, b))):
            if ch & L.LEAF:
                assert ca == cb == (ch & ~L.LEAF)
                leaves.append(ca)
                assert parents[n - 1 + ca] == i
            else:
                assert ch in (split, split + 1)
                ranges[int(ch)] = (ca, cb)
                assert parents[ch] == i
                stack.append(int(ch))
        del lr, g
    assert sorted(leaves) == list(range(n))
    assert len(ranges) == n - 1


def test_radix_tree_property_with_duplicates():
    rng = np.random.default_rng(0)
    for n, hi in ((2, 4), (7, 3), (64, 8), (300, 16), (1000, 1 << 30)):
        keys = np.sort(rng.integers(0, hi, size=n).astype(np.uint32))
        children, parents = L.radix_tree(keys)
        _check_tree(keys, children, parents)


def test_refit_contains_children():
    rng = np.random.default_rng(1)
    v = rng.uniform(-5, 5, size=(300, 3)).astype(np.float32)
    t = rng.integers(0, 300, size=(100, 3)).astype(np.uint32)
    codes, perm = L.sort_codes(L.morton(v, t))
    ch, par = L.radix_tree(codes)
    lb = L.leaf_boxes(v, t, perm)
    boxes = L.refit(ch, lb)
    root = np.concatenate([np.minimum(boxes[0, 0, :3], boxes[0, 1, :3]), np.maximum(boxes[0, 0, 3:], boxes[0, 1, 3:])])
    assert np.array_equal(root[:3], lb[:, :3].min(0)) and np.array_equal(root[3:], lb[:, 3:].max(0))


# ---------------------------------------------------------------- SAH top
def _soup(centres, spread=0.3, seed=0):
    rng = np.random.default_rng(seed)
    c = np.asarray(centres, np.float64)[:, None, :]
    tri = (c + rng.normal(scale=spread, size=(len(centres), 3, 3))).astype(np.float32)
    return tri.reshape(-1, 3), np.arange(3 * len(centres), dtype=np.uint32).reshape(-1, 3)


def _build(v, t):
    sk, perm = L.sort_codes(L.morton(v, t))
    ch, _ = L.radix_tree(sk)
    return ch, L.leaf_boxes(v, t, perm), perm


def _is_tree(enc, n):
    assert sorted(x for x in enc if x >= 0) == list(range(n))
    assert sum(1 for x in enc if x < 0) == n - 1
    need = 1   # a preorder of a full binary tree: open slots reach zero exactly at the end
    for x in enc:
        assert need > 0
        need += 1 if x < 0 else -1
    assert need == 0


def _sah_top_by_masks(children, leaf_box, cluster_max=32, bins=32, median_depth=32):
    """The same rules, every split's sides taken as masks over the clusters
    and their boxes reduced directly (no bin accumulation)."""
    n = len(leaf_box)
    roots, size = L.cluster_roots(children, n, cluster_max)
    if n < 2 or len(roots) == 1:
        return L.preorder(children, n)
    boxes = L.refit(children, leaf_box)

    def ref_box(ref):
        if ref & L.LEAF:
            return np.asarray(leaf_box[ref & ~L.LEAF], np.float32)
        b0, b1 = boxes[ref]
        return np.concatenate([np.minimum(b0[:3], b1[:3]), np.maximum(b0[3:], b1[3:])]).astype(np.float32)

    cbox = np.stack([ref_box(r) for r in roots]).astype(np.float32)
    cen = (np.float32(0.5) * (cbox[:, :3] + cbox[:, 3:])).astype(np.float32)
    wgt = np.array([L._size(r, size) for r in roots], np.int64)
    out = []

    def task(m, depth):
        nm = len(m)
        c = cen[m]
        cmin, cmax = c.min(0), c.max(0)
        best = None
        for k in range(3) if depth < median_depth else ():
            ext = np.float32(cmax[k] - cmin[k])
            if not ext > 0:
                continue
            scale = np.float32(np.float32(bins) / ext)
            q = np.minimum(((c[:, k] - cmin[k]).astype(np.float32) * scale).astype(np.float32).astype(np.int64),
                           bins - 1)
            for split in range(1, bins):
                left = q < split
                if not 0 < left.sum() < nm:
                    continue
                bl, br = cbox[m[left]], cbox[m[~left]]
                al = L._area(bl[:, :3].min(0), bl[:, 3:].max(0))
                ar = L._area(br[:, :3].min(0), br[:, 3:].max(0))
                cost = np.float32(np.float32(al * np.float32(wgt[m[left]].sum()))
                                  + np.float32(ar * np.float32(wgt[m[~left]].sum())))
                if best is None or cost < best[0]:
                    best = (cost, left)
        left = np.arange(nm) < nm // 2 if best is None else best[1]
        out.append(-1)
        for side in (m[left], m[~left]):
            if len(side) == 1:
                out.extend(L.preorder_from(children, roots[int(side[0])]))
            else:
                task(side, depth + 1)

    task(np.arange(len(roots)), 0)
    return out


def test_sah_top_equals_the_rules_by_masks():
    """Prefix / suffix unions of the bins give the same tree as reducing each
    split's sides directly: random and duplicate-heavy soups, clusters of 1
    (a full binned SAH over triangles), 4 and 32 leaves."""
    for seed in range(4):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(40, 1500))
        if seed % 2:
            base = rng.uniform(-3, 3, size=(23, 3, 3)).astype(np.float32)
            tri = base[rng.integers(0, 23, size=n)]
        else:
            c = rng.uniform(-50, 50, size=(n, 1, 3)) * np.array([1, 1, 0.1])
            tri = (c + rng.normal(scale=0.5, size=(n, 3, 3))).astype(np.float32)
        v = tri.reshape(-1, 3)
        t = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
        ch, lb, _ = _build(v, t)
        for k in (1, 4, 32):
            enc = L.sah_top(ch, lb, cluster_max=k)
            assert enc == _sah_top_by_masks(ch, lb, cluster_max=k), (seed, k)
            _is_tree(enc, n)


def test_sah_top_keeps_a_small_tree():
    v, t = _soup(np.random.default_rng(1).uniform(-5, 5, size=(30, 3)))
    ch, lb, _ = _build(v, t)
    assert L.sah_top(ch, lb, cluster_max=32) == L.preorder(ch, 30)


def test_sah_top_separates_far_groups():
    """Two compact groups 100 m apart: the root's children hold one group
    each, whatever the Morton order interleaves below."""
    rng = np.random.default_rng(2)
    a = rng.uniform(0, 2, size=(60, 3))
    b = rng.uniform(0, 2, size=(60, 3)) + np.array([100.0, 0.0, 0.0])
    v, t = _soup(np.concatenate([a, b]))
    ch, lb, perm = _build(v, t)
    enc = L.sah_top(ch, lb, cluster_max=4)
    _is_tree(enc, 120)
    need, k = 1, 1   # the root's left subtree: up to where its preorder closes
    while need:
        need += 1 if enc[k] < 0 else -1
        k += 1
    left = {int(perm[x]) for x in enc[1:k] if x >= 0}
    assert left in (set(range(60)), set(range(60, 120)))


def test_sah_top_split_cost_by_hand():
    """Single-triangle clusters at x = 0, 1 and 10 (unit boxes, half-area 3):
    {0, 1} | {10} costs 2 * (2 + 1 + 2) + 1 * 3 = 13, {0} | {1, 10} costs
    1 * 3 + 2 * (10 + 1 + 10) = 45; the first wins, and {0, 1} is split below."""
    v = np.array([[[x, 0, 0], [x + 1, 0, 0], [x, 1, 1]] for x in (0.0, 1.0, 10.0)], np.float32).reshape(-1, 3)
    t = np.arange(9, dtype=np.uint32).reshape(3, 3)
    ch, lb, perm = _build(v, t)
    enc = L.sah_top(ch, lb, cluster_max=1)
    assert [int(perm[x]) if x >= 0 else -1 for x in enc] == [-1, -1, 0, 1, 2]
    assert L._area(np.float32([0, 0, 0]), np.float32([2, 1, 1])) == 5.0
    assert L._area(np.float32([1, 0, 0]), np.float32([11, 1, 1])) == 21.0


def test_sah_top_median_at_the_depth_limit():
    """At the depth limit every task halves its cluster list: with limit 0 the
    tree is the balanced split of the Morton-ordered leaves."""
    v, t = _soup(np.random.default_rng(3).uniform(-20, 20, size=(37, 3)))
    ch, lb, _ = _build(v, t)

    def balanced(lo, hi):
        if hi - lo == 1:
            return [lo]
        m = lo + (hi - lo) // 2
        return [-1] + balanced(lo, m) + balanced(m, hi)

    assert L.sah_top(ch, lb, cluster_max=1, median_depth=0) == balanced(0, 37)


def test_sah_top_keeps_the_clusters():
    rng = np.random.default_rng(4)
    for n, k in ((500, 8), (2000, 32), (777, 1)):
        c = rng.uniform(-50, 50, size=(n, 3)) * np.array([1.0, 1.0, 0.1])
        v, t = _soup(c, spread=0.5, seed=n)
        ch, lb, _ = _build(v, t)
        enc = L.sah_top(ch, lb, cluster_max=k)
        _is_tree(enc, n)
        s = "," + ",".join(map(str, enc)) + ","
        roots, _ = L.cluster_roots(ch, n, k)
        for r in roots[:50]:   # every cluster's subtree appears unchanged
            assert "," + ",".join(map(str, L.preorder_from(ch, r))) + "," in s

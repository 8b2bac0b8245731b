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

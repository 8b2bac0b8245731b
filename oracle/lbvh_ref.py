"""CPU reference of the LBVH build steps (test infrastructure only).

Plain numpy / Python restatements of the definitions the GPU build follows;
shares no code with the CUDA library:

* centroid  (v0 + v1 + v2) / 3 in float32, summed left to right
* Morton    centroid normalised to the centroid bounds in float32,
            q = min(floor(x * 1024), 1023) per axis, bits interleaved as
            x9 y9 z9 ... x0 y0 z0 (one bit at a time)
* sort      stable sort of the codes (numpy's stable argsort)
* topology  binary radix tree over the sorted codes, built top down from
            its definition: a node over [a, b] splits after the last index
            whose key shares more leading bits with key a than key b does;
            equal keys are told apart by their index bits (Karras, HPG 2012).
            Internal nodes are numbered like Karras's layout: the node over
            [a, b] with split g has children g (left) and g + 1 (right),
            leaves where a child range holds one key.
* refit     child boxes as float32 min / max of the triangle boxes
"""
from __future__ import annotations

import numpy as np

LEAF = 0x80000000


def centroids(vertices, triangles):
    v = np.asarray(vertices, np.float32)
    t = np.asarray(triangles, np.int64)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return ((a + b) + c) / np.float32(3.0)


def interleave_bits(qx, qy, qz):
    code = np.zeros(np.shape(qx), np.uint64)
    for bit in range(9, -1, -1):
        for q in (qx, qy, qz):
            code = (code << np.uint64(1)) | ((np.asarray(q, np.uint64) >> np.uint64(bit)) & np.uint64(1))
    return code.astype(np.uint32)


def morton(vertices, triangles):
    c = centroids(vertices, triangles)
    lo = c.min(axis=0)
    hi = c.max(axis=0)
    ext = (hi - lo).astype(np.float32)
    q = np.zeros(c.shape, np.uint32)
    for k in range(3):
        if ext[k] > 0:
            x = (c[:, k] - lo[k]) / ext[k]
        else:
            x = np.zeros(len(c), np.float32)
        q[:, k] = np.minimum(np.floor(x * np.float32(1024.0)), np.float32(1023.0)).astype(np.uint32)
    return interleave_bits(q[:, 0], q[:, 1], q[:, 2])


def sort_codes(codes):
    perm = np.argsort(codes, kind="stable").astype(np.uint32)
    return codes[perm], perm


def _prefix(keys, i, j):
    """Leading bits shared by (key_i, i) and (key_j, j) as 64-bit words."""
    a = (int(keys[i]) << 32) | i
    b = (int(keys[j]) << 32) | j
    x = a ^ b
    return 64 - x.bit_length()


def radix_tree(keys):
    """children [(n-1), 2] (leaf j as j | LEAF), parents [2n-1] (leaves at n-1+j)."""
    n = len(keys)
    children = np.zeros((max(n - 1, 0), 2), np.uint32)
    parents = np.full(max(2 * n - 1, 1), 0xFFFFFFFF, np.uint32)
    if n < 2:
        return children, parents
    stack = [(0, 0, n - 1)]
    seen = np.zeros(n - 1, bool)
    while stack:
        node, a, b = stack.pop()
        assert not seen[node]
        seen[node] = True
        common = _prefix(keys, a, b)
        # last index g in [a, b-1] whose key still shares more than `common` bits with key a
        g = a
        lo, hi = a, b - 1
        while lo <= hi:                      # binary search: prefix(a, m) > common is monotone in m
            m = (lo + hi) // 2
            if _prefix(keys, a, m) > common:
                g = m
                lo = m + 1
            else:
                hi = m - 1
        left = (g | LEAF) if g == a else g
        right = ((g + 1) | LEAF) if g + 1 == b else g + 1
        children[node] = (left, right)
        for ch, (ca, cb) in ((left, (a, g)), (right, (g + 1, b))):
            if ch & LEAF:
                parents[n - 1 + (ch & ~LEAF)] = node
            else:
                parents[ch] = node
                stack.append((ch, ca, cb))
    assert seen.all()
    return children, parents


def leaf_boxes(vertices, triangles, perm):
    v = np.asarray(vertices, np.float32)
    t = np.asarray(triangles, np.int64)[perm]
    p = np.stack([v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]], 1)
    return np.concatenate([p.min(1), p.max(1)], 1).astype(np.float32)


def refit(children, leaf_box):
    """Child boxes [(n-1), 2, 6] of every internal node (lo xyz, hi xyz)."""
    n = len(leaf_box)
    out = np.zeros((max(n - 1, 0), 2, 6), np.float32)
    own = {}

    def box(ref):
        if ref & LEAF:
            return leaf_box[ref & ~LEAF]
        return own[ref]

    # post-order without recursion
    order = []
    stack = [0] if n > 1 else []
    while stack:
        i = stack.pop()
        order.append(i)
        for ch in children[i]:
            if not ch & LEAF:
                stack.append(int(ch))
    for i in reversed(order):
        b0, b1 = box(int(children[i][0])), box(int(children[i][1]))
        out[i, 0], out[i, 1] = b0, b1
        own[i] = np.concatenate([np.minimum(b0[:3], b1[:3]), np.maximum(b0[3:], b1[3:])])
    return out

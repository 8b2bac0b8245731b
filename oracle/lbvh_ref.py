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
* SAH top   (optional) the part of the tree above its subtrees of at most
            `cluster_max` leaves rebuilt top down by binned SAH over those
            subtrees (HLBVH: Pantaleoni and Luebke, HPG 2010; Garanzha et al.,
            HPG 2011), the rules spelled out in `sah_top`
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


def subtree_sizes(children, n):
    """Leaves under every internal node (root 0)."""
    size = np.zeros(max(n - 1, 0), np.int64)
    order = []
    stack = [0] if n > 1 else []
    while stack:
        i = stack.pop()
        order.append(i)
        for ch in children[i]:
            if not ch & LEAF:
                stack.append(int(ch))
    for i in reversed(order):
        size[i] = sum(1 if ch & LEAF else size[int(ch)] for ch in children[i])
    return size


def _size(ref, size):
    return 1 if ref & LEAF else int(size[ref])


def cluster_roots(children, n, cluster_max):
    """Roots of the maximal subtrees with at most cluster_max leaves, in leaf order."""
    size = subtree_sizes(children, n)
    if n < 2 or n <= cluster_max:
        return [0 if n > 1 else LEAF], size
    out = []
    stack = [0]
    while stack:
        ref = stack.pop()
        if _size(ref, size) <= cluster_max:
            out.append(ref)
        else:
            c0, c1 = (int(c) for c in children[ref])
            stack.append(c1)   # left first
            stack.append(c0)
    return out, size


def _f32(x):
    return np.float32(x)


def _area(lo, hi):
    dx, dy, dz = (_f32(hi[k] - lo[k]) for k in range(3))
    return _f32(_f32(_f32(dx * dy) + _f32(dy * dz)) + _f32(dz * dx))


def sah_top(children, leaf_box, cluster_max=32, bins=32, median_depth=32):
    """Tree of the SAH-top build as a preorder encoding (see `preorder`).

    Clusters are the subtrees of `cluster_roots`, with the float32 union box
    of their leaves and weight = their leaf count.  A task over clusters
    [b, e) (n >= 2) at depth d:
      * centroid c = 0.5 * (lo + hi) per cluster; bounds cmin, cmax;
      * per axis with ext = cmax - cmin > 0: scale = bins / ext, bin
        q = min(bins - 1, trunc((c - cmin) * scale)), every step rounded to
        float32;
      * split after bin q (1 <= q < bins) with both sides non-empty costs
        area(L) * weight(L) + area(R) * weight(R) in float32, area =
        dx*dy + dy*dz + dz*dx; the lowest cost wins, ties to the lower axis,
        then the lower q;
      * without a split, or at depth >= median_depth: the first n // 2
        clusters go left;
      * the partition keeps the cluster order on each side; a side with one
        cluster is that cluster's subtree, otherwise a new task at d + 1.
    The bins of one axis are accumulated once (counts and weights are exact
    integer sums, boxes exact min / max), so the left and right sides of
    every split are prefix and suffix unions of the bins.
    """
    n = len(leaf_box)
    roots, size = cluster_roots(children, n, cluster_max)
    if n < 2 or len(roots) == 1:
        return preorder(children, n)
    boxes = refit(children, leaf_box)

    def ref_box(ref):
        if ref & LEAF:
            return np.asarray(leaf_box[ref & ~LEAF], np.float32)
        b0, b1 = boxes[ref]
        return np.concatenate([np.minimum(b0[:3], b1[:3]), np.maximum(b0[3:], b1[3:])]).astype(np.float32)

    cbox = np.stack([ref_box(r) for r in roots]).astype(np.float32)
    cen = (np.float32(0.5) * (cbox[:, :3] + cbox[:, 3:])).astype(np.float32)
    wgt = np.array([_size(r, size) for r in roots], np.int64)
    out = []

    def task(members, depth):
        m = np.asarray(members, np.int64)
        nm = len(m)
        c = cen[m]
        cmin, cmax = c.min(0), c.max(0)
        best = None   # (cost, axis, q, left mask)
        if depth < median_depth:
            for k in range(3):
                ext = _f32(cmax[k] - cmin[k])
                if not ext > 0:
                    continue
                scale = _f32(_f32(bins) / ext)
                q = np.minimum(((c[:, k] - cmin[k]).astype(np.float32) * scale).astype(np.float32).astype(np.int64),
                               bins - 1)
                cnt = np.bincount(q, minlength=bins)
                w = np.bincount(q, weights=wgt[m], minlength=bins).astype(np.int64)
                lo = np.full((bins, 3), np.inf, np.float32)
                hi = np.full((bins, 3), -np.inf, np.float32)
                np.minimum.at(lo, q, cbox[m, :3])
                np.maximum.at(hi, q, cbox[m, 3:])
                llo, lhi = np.minimum.accumulate(lo), np.maximum.accumulate(hi)
                rlo = np.minimum.accumulate(lo[::-1])[::-1]
                rhi = np.maximum.accumulate(hi[::-1])[::-1]
                ncum, wcum = np.cumsum(cnt), np.cumsum(w)
                for split in range(1, bins):
                    nl = int(ncum[split - 1])
                    if nl == 0 or nl == nm:
                        continue
                    al = _area(llo[split - 1], lhi[split - 1])
                    ar = _area(rlo[split], rhi[split])
                    wl = int(wcum[split - 1])
                    wr = int(wcum[-1]) - wl
                    cost = _f32(_f32(al * _f32(wl)) + _f32(ar * _f32(wr)))
                    if best is None or cost < best[0]:
                        best = (cost, k, split, q < split)
        if best is None:
            left = np.arange(nm) < nm // 2
        else:
            left = best[3]
        out.append(-1)
        for side in (m[left], m[~left]):
            if len(side) == 1:
                out.extend(preorder_from(children, roots[int(side[0])]))
            else:
                task(side, depth + 1)

    task(list(range(len(roots))), 0)
    return out


def preorder_from(children, ref):
    """Preorder of the subtree at `ref`: -1 for an internal node, j for leaf j."""
    out = []
    stack = [int(ref)]
    while stack:
        r = stack.pop()
        if r & LEAF:
            out.append(r & ~LEAF)
        else:
            out.append(-1)
            c0, c1 = (int(c) for c in children[r])
            stack.append(c1)
            stack.append(c0)
    return out


def preorder(children, n):
    """Topology of the tree rooted at internal node 0 (leaf 0 for one leaf)."""
    if n < 2:
        return [0] if n == 1 else []
    return preorder_from(children, 0)

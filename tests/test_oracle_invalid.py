"""Pins of the oracle's INVALID nodes and their pointers (Sec. 5.2: a node
whose information for a channel is not initialised stores a pointer to the
node in the next lower subdivision level that has valid information for the
channel, or UNKNOWN; Sec. 5.3: metadata arrives for volume regions, i.e. for
nodes of any depth).  CPU only.

Reading: a leaf's range is the one the data source gave; an inner node's is
the hull of its children's when all of them are valid, else the range given
for the node itself; without either the node is INVALID, and its word keeps
its residency mask with min8 = 255 and max8 = the depth of the nearest valid
ancestor (254 = UNKNOWN).  The walk reads an INVALID word with that
ancestor's range and its own mask.

The node words are checked against a brute force that takes another route
to the same definition: validity as "every path from the node down to a leaf
meets a node with a given range", the range as the hull over the first
such frontier node on each path, and the pointer by scanning the ancestors.
"""
import math

import numpy as np
import pytest

import oracle
import synth

UNKNOWN = 254


def tree(dims, leaf):
    nl = [-(-d // e) for d, e in zip(dims, leaf)]
    D = max(max(0, math.ceil(math.log2(n))) if n > 1 else 0 for n in nl)
    nn, off = [], [0]
    for d in range(D + 1):
        e = [x << (D - d) for x in leaf]
        nn.append([-(-dims[a] // e[a]) for a in range(3)])
        off.append(off[-1] + nn[-1][0] * nn[-1][1] * nn[-1][2])
    return D, nn, off


def node_id(nn, off, d, j):
    return off[d] + (j[2] * nn[d][1] + j[1]) * nn[d][0] + j[0]


def brute_ranges(dims, leaf, m, leaf_min, leaf_max, node_min, node_max, bpv):
    """Upper 16 bits of every node word, by path scans (see module doc)."""
    D, nn, off = tree(dims, leaf)
    nl = nn[D]

    def given(d, j, c):
        if d == D:
            a, b = leaf_min[c][j[2]][j[1]][j[0]], leaf_max[c][j[2]][j[1]][j[0]]
        else:
            n = node_id(nn, off, d, j)
            a, b = node_min[c][n], node_max[c][n]
        return (a, b) if a >= 0 and b >= 0 else None

    def children(d, j):
        return [(j[0] * 2 + cx, j[1] * 2 + cy, j[2] * 2 + cz) for cz in (0, 1) for cy in (0, 1) for cx in (0, 1)
                if j[0] * 2 + cx < nn[d + 1][0] and j[1] * 2 + cy < nn[d + 1][1] and j[2] * 2 + cz < nn[d + 1][2]]

    def leaves_below(d, j):
        s = D - d
        return [(x, y, z) for z in range(j[2] << s, min((j[2] + 1) << s, nl[2]))
                for y in range(j[1] << s, min((j[1] + 1) << s, nl[1]))
                for x in range(j[0] << s, min((j[0] + 1) << s, nl[0]))]

    def path(d, j, L):
        """nodes from (d, j) down to leaf L"""
        return [(dd, tuple(v >> (D - dd) for v in L)) for dd in range(d, D + 1)]

    valid_memo = {}

    def valid(d, j, c):
        key = (d, j, c)
        if key not in valid_memo:
            valid_memo[key] = all(any(given(dd, jj, c) is not None for dd, jj in path(d, j, L))
                                  for L in leaves_below(d, j))
        return valid_memo[key]

    out = {}
    for d in range(D + 1):
        for jz in range(nn[d][2]):
            for jy in range(nn[d][1]):
                for jx in range(nn[d][0]):
                    j = (jx, jy, jz)
                    n = node_id(nn, off, d, j)
                    for c in range(m):
                        if valid(d, j, c):
                            lo, hi = None, None
                            for L in leaves_below(d, j):
                                for dd, jj in path(d, j, L):
                                    if dd == D or not all(valid(dd + 1, ch, c) for ch in children(dd, jj)):
                                        a, b = given(dd, jj, c)
                                        lo = a if lo is None else min(lo, a)
                                        hi = b if hi is None else max(hi, b)
                                        break
                            q0, q1 = (lo, hi) if bpv == 1 else (lo >> 8, hi >> 8)
                        else:
                            q0, q1 = 255, UNKNOWN
                            for dd in range(d - 1, -1, -1):
                                if valid(dd, tuple(v >> (d - dd) for v in j), c):
                                    q1 = dd
                                    break
                        out[(n, c)] = (q0 << 16) | (q1 << 24)
    return out, off[-1]


def random_metadata(rng, vol0s, leaf, dims, frac_leaf, frac_inner, bpv):
    """Exact ranges (over the dilated support) for a random subset of leaves,
    and conservative ones for a random subset of inner nodes: the hull of
    the node's leaves widened at random (a coarse estimate of the data
    source), so that a node whose children are all valid shows whether their
    hull or its given range is used."""
    m = len(vol0s)
    D, nn, off = tree(dims, leaf)
    lmin, lmax, nmin, nmax = [], [], np.full((m, off[-1]), -1, np.int64), np.full((m, off[-1]), -1, np.int64)
    for c, v in enumerate(vol0s):
        mn, mx = synth.leaf_ranges(v, leaf)
        mn, mx = mn.astype(np.int64), mx.astype(np.int64)
        for d in range(D):
            s = D - d
            for jz in range(nn[d][2]):
                for jy in range(nn[d][1]):
                    for jx in range(nn[d][0]):
                        if rng.random() < frac_inner:
                            sl = (slice(jz << s, (jz + 1) << s), slice(jy << s, (jy + 1) << s),
                                  slice(jx << s, (jx + 1) << s))
                            n = node_id(nn, off, d, (jx, jy, jz))
                            top = 255 if bpv == 1 else 65535
                            widen = rng.integers(0, 12 if bpv == 1 else 3000, 2)
                            nmin[c, n] = max(0, int(mn[sl].min()) - int(widen[0]))
                            nmax[c, n] = min(top, int(mx[sl].max()) + int(widen[1]))
        drop = rng.random(mn.shape) >= frac_leaf
        mn[drop] = -1
        mx[drop] = -1
        lmin.append(mn)
        lmax.append(mx)
    return np.stack(lmin), np.stack(lmax), nmin, nmax


@pytest.mark.parametrize("seed,bpv", [(0, 1), (1, 1), (2, 2), (3, 1)])
def test_node_words_match_path_scan(seed, bpv):
    rng = np.random.default_rng(seed)
    dims, leaf, m = (20, 14, 9), (2, 2, 1), 2
    dt = np.uint8 if bpv == 1 else np.uint16
    hi = 255 if bpv == 1 else 65535
    vols = [rng.integers(0, hi, dims[::-1]).astype(dt) for _ in range(m)]
    fl, fi = [(0.6, 0.2), (0.3, 0.5), (0.8, 0.3), (0.0, 0.4)][seed]
    lmin, lmax, nmin, nmax = random_metadata(rng, vols, leaf, dims, fl, fi, bpv)
    lv = [[v] for v in vols]
    vol = oracle.Volume(lv, (1, 1, 1), 4, leaf, [], lmin, lmax, node_min=nmin, node_max=nmax)
    w = vol.node_words()
    want, n_nodes = brute_ranges(dims, leaf, m, lmin, lmax, nmin, nmax, bpv)
    assert w.shape == (n_nodes, m)
    got = {(n, c): int(w[n, c]) & 0xFFFF0000 for n in range(n_nodes) for c in range(m)}
    bad = [k for k in want if want[k] != got[k]]
    assert not bad, f"{len(bad)} words differ, first {bad[0]}: want {want[bad[0]]:#x} got {got[bad[0]]:#x}"
    # every case occurs: valid, INVALID with a pointer, UNKNOWN
    hi8 = (w >> 24) & 0xFF
    lo8 = (w >> 16) & 0xFF
    inv = lo8 > hi8
    assert inv.any() and (~inv).any()
    if seed != 0:
        assert (inv & (hi8 != UNKNOWN)).any()


def const_scene(value, dtype):
    """32^3 constant volume, two levels, 16^3 bricks (all resident)."""
    lv = synth.mean_levels(np.full((32, 32, 32), value, dtype), 2)
    bricks = [(0, l, x, y, z) for l in (0, 1) for z in range(-(-lv[l].shape[0] // 16))
              for y in range(-(-lv[l].shape[1] // 16)) for x in range(-(-lv[l].shape[2] // 16))]
    return lv, bricks


def ortho_z(W=8, H=8):
    return synth.look_at((16.0, 16.0, -10.0), (16.0, 16.0, 0.0), (0, -1, 0), W, H, ortho_pixel=1.0)


def root_only(vol, lo, hi):
    """No leaf metadata; the root (node 0) given the range [lo, hi]."""
    nmin = np.full((1, vol.n_nodes), -1, np.int64)
    nmax = np.full((1, vol.n_nodes), -1, np.int64)
    nmin[0, 0], nmax[0, 0] = lo, hi
    vol.set_node_ranges(nmin, nmax)


def test_empty_by_ancestor_skips_without_requests():
    """Traversal starting at depth 2 (the paper starts at level 3) over
    INVALID nodes whose root range is below the TF window: every node reads
    as empty through its pointer, so no sample is evaluated, nothing is
    requested and no node metadata is asked for.  With the root UNKNOWN
    instead, the same rays descend, sample and request node metadata."""
    lv, bricks = const_scene(5, np.uint16)
    vol = oracle.Volume([lv], (1, 1, 1), 16, (4, 4, 4), bricks)
    assert vol.depth == 3
    tf = synth.tf_ramp(400, 12000)
    fr = synth.Frame(8, 8, ortho_z(), [tf], 0.5, [0.0] + [float("inf")] * 15, [0], [0], start_depth=2)
    root_only(vol, 5, 5)
    w = vol.node_words()
    assert ((w[1:, 0] >> 24) & 0xFF == 0).all() and ((w[1:, 0] >> 16) & 0xFF == 255).all()
    o = oracle.render(vol, w, fr)
    assert np.all(o["n_eval"] == 0) and np.all(o["rgba32"] == 0)
    assert o["req_ids"].size == 0 and o["node_req_ids"].size == 0
    vol.set_node_ranges(None, None)
    w = vol.node_words()
    assert ((w[:, 0] >> 24) & 0xFF == UNKNOWN).all()
    o2 = oracle.render(vol, w, fr)
    assert np.all(o2["n_eval"] > 0) and o2["node_req_ids"].size > 0


@pytest.mark.parametrize("start_depth", [0, 2])
def test_homogeneous_by_ancestor_closed_form(start_depth):
    """u8 constant volume, no leaf metadata, the root given [77, 77]: every
    INVALID node reads as homogeneous through its pointer (Sec. 5.2), so
    each sample takes the node value without a brick: opacity 1 - (1 -
    alpha)^n over the n lattice samples, no brick read, no request."""
    alpha = float(np.float32(0.03))
    lv, bricks = const_scene(77, np.uint8)
    vol = oracle.Volume([lv], (1, 1, 1), 16, (4, 4, 4), bricks)
    root_only(vol, 77, 77)
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = (0.2, 0.6, 1.0)
    lut[:, 3] = alpha
    tf = synth.TF(0.0, 1.0, lut)
    fr = synth.Frame(8, 8, ortho_z(), [tf], 0.5, [0.0] + [float("inf")] * 15, [0], [0], start_depth=start_depth,
                     ert=0.0)
    o = oracle.render(vol, vol.node_words(), fr)
    n = 64
    assert np.all(o["n_eval"] == n) and np.all(o["n_bs"] == 0)
    assert np.allclose(o["rgba64"][:, 3], 1.0 - (1.0 - alpha) ** n, rtol=0, atol=1e-12)
    assert o["req_ids"].size == 0 and o["used_ids"].size == 0 and o["node_req_ids"].size == 0


def test_brick_by_ancestor_samples_and_asks_for_metadata():
    """A non-empty, inhomogeneous root range: INVALID nodes read as partially
    mapped through their pointer, rays sample the resident bricks exactly as
    with full metadata, and every final node asks for its own metadata."""
    rng = np.random.default_rng(5)
    vol0 = rng.integers(1000, 30000, (32, 32, 32)).astype(np.uint16)
    lv = synth.mean_levels(vol0, 2)
    bricks = [(0, l, x, y, z) for l in (0, 1) for z in range(-(-lv[l].shape[0] // 16))
              for y in range(-(-lv[l].shape[1] // 16)) for x in range(-(-lv[l].shape[2] // 16))]
    mn, mx = synth.leaf_ranges(vol0, (4, 4, 4))
    full = oracle.Volume([lv], (1, 1, 1), 16, (4, 4, 4), bricks, mn[None].astype(np.int64), mx[None].astype(np.int64))
    part = oracle.Volume([lv], (1, 1, 1), 16, (4, 4, 4), bricks)
    root_only(part, int(mn.min()), int(mx.max()))
    tf = synth.tf_ramp(400, 40000)
    fr = synth.Frame(8, 8, ortho_z(), [tf], 0.5, [0.0] + [float("inf")] * 15, [0], [0], ert=0.0)
    a = oracle.render(full, full.node_words(), fr)
    b = oracle.render(part, part.node_words(), fr)
    for key in ("rgba32", "hash", "n_eval", "n_bs"):
        assert np.array_equal(a[key], b[key]), key
    assert a["node_req_ids"].size == 0 and b["node_req_ids"].size > 0
    # the requested nodes are leaves (the walk ends at the traversal depth)
    D = part.depth
    first_leaf = part.n_nodes - int(np.prod(part.leaf_shape))
    assert np.all(b["node_req_ids"] >= first_leaf * part.m) and D == 3

"""Pins for the oracle's quadtree, Morton order and dual-tree-traversal lists
(Sec. 5.1 tree, Sec. 5.2 DTT with the MAC).

Independent checks: a string-based bit interleave, numpy's stable argsort, and brute
force over all (target leaf, source leaf) pairs: every pair must be covered exactly once,
either by a P2P pair or by one M2L pair of ancestors at the same level; the MAC must
hold for M2L pairs and fail for their parents and for P2P pairs.
"""
import math

import numpy as np
import pytest

import oracle as O


def morton_ref(i, j, bits=16):
    bi, bj = format(i, f"0{bits}b"), format(j, f"0{bits}b")
    s = "".join(y + x for x, y in zip(bi, bj))  # y bit above x bit at each level
    return int(s, 2)


def demorton(c):
    c = np.asarray(c, np.int64)
    x = np.zeros_like(c)
    y = np.zeros_like(c)
    for b in range(20):
        x |= ((c >> (2 * b)) & 1) << b
        y |= ((c >> (2 * b + 1)) & 1) << b
    return x, y


def test_morton_keys_match_string_interleave():
    n = 32
    k = O.morton_keys(n)
    for j in range(n):
        for i in range(n):
            assert k[j * n + i] == morton_ref(i, j)


def test_sort_perm_is_stable_argsort():
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 50, size=5000).astype(np.uint32)  # many duplicates
    assert np.array_equal(O.sort_perm(keys), np.argsort(keys, kind="stable"))
    k = O.morton_keys(64)
    assert np.array_equal(O.sort_perm(k), np.argsort(k, kind="stable"))


@pytest.mark.parametrize("n,leaf_max,L", [(64, 64, 3), (64, 16, 4), (128, 256, 3), (96, 64, 4),
                                          (48, 36, 3), (24, 4, -1)])
def test_leaf_level(n, leaf_max, L):
    # split at centre lines until <= leaf_max nodes (Sec. 5.1); -1 when a centre line
    # would cut through a row of nodes (24 -> 12 -> 6 -> 3 with 9 > 4 nodes left)
    assert O.leaf_level(n, leaf_max) == L


def test_cell_ranges_of_complete_tree():
    n = 64
    P = O.Problem(n, p=4)
    st = P.export(O.E_CELL_START)
    perm = P.export(O.E_PERM)
    off = 0
    for l in range(P.L + 1):
        s = n >> l
        nc = 4 ** l
        assert np.array_equal(st[off: off + nc], np.arange(nc) * s * s)
        cx, cy = demorton(np.arange(nc))
        for c in range(nc):
            idx = perm[c * s * s: (c + 1) * s * s]
            assert np.all(idx % n // s == cx[c]) and np.all(idx // n // s == cy[c])
        off += nc


def _geom(n, l, c):
    a, b = demorton(c)
    w = n >> l
    return 2 * a * w + w + 1, 2 * b * w + w + 1, w  # units of h/2


def _mac(n, l, A, B, th):
    XA, YA, sA = _geom(n, l, A)
    XB, YB, sB = _geom(n, l, B)
    d = np.hypot(XA - XB, YA - YB)
    return math.sqrt(2) * (sA + sB) < th * d, math.sqrt(2) * (sA + sB) - th * d


@pytest.mark.parametrize("n", [64, 128])
def test_dtt_lists_partition_all_leaf_pairs(n):
    P = O.Problem(n, p=4)
    L = P.L
    nl = 4 ** L
    cover = np.zeros((nl, nl), np.int32)
    p2p = P.export(O.E_P2P)
    cover[p2p[:, 0], p2p[:, 1]] += 1
    leaves = np.arange(nl)
    for l, A, B in P.export(O.E_M2L):
        sh = 2 * (L - l)
        ts = leaves[(leaves >> sh) == A]
        ss = leaves[(leaves >> sh) == B]
        cover[np.ix_(ts, ss)] += 1
    assert cover.min() == 1 and cover.max() == 1


def test_dtt_mac_conditions():
    n, th = 128, 0.4
    P = O.Problem(n, p=4)
    m2l = P.export(O.E_M2L)
    ok, margin = _mac(n, m2l[:, 0], m2l[:, 1], m2l[:, 2], th)
    assert ok.all()
    pok, _ = _mac(n, m2l[:, 0] - 1, m2l[:, 1] >> 2, m2l[:, 2] >> 2, th)
    assert not pok.any()
    p2p = P.export(O.E_P2P)
    ok2, _ = _mac(n, np.full(len(p2p), P.L), p2p[:, 0], p2p[:, 1], th)
    assert not ok2.any()
    # lists are in canonical (level, target, source) order
    key = m2l[:, 0].astype(np.int64) << 50 | m2l[:, 1].astype(np.int64) << 25 | m2l[:, 2]
    assert np.all(np.diff(key) > 0)


def test_m2l_offsets_per_level():
    # uniform tree, theta = 0.4: the same 140 target-source offsets recur on every level >= 3
    P = O.Problem(256, p=4)
    m2l = P.export(O.E_M2L)
    for l in range(3, P.L + 1):
        s = m2l[m2l[:, 0] == l]
        tx, ty = demorton(s[:, 1])
        sx, sy = demorton(s[:, 2])
        assert len(set(zip((tx - sx).tolist(), (ty - sy).tolist()))) == 140


def test_p2p_is_the_37_leaf_stencil():
    # theta = 0.4 -> leaves interact directly iff |offset|^2 < 12.5 (in leaf widths); the
    # largest integer offset norm below that is 10, e.g. (3, 1)
    P = O.Problem(128, p=4)
    p2p = P.export(O.E_P2P)
    tx, ty = demorton(p2p[:, 0])
    sx, sy = demorton(p2p[:, 1])
    d2 = (tx - sx) ** 2 + (ty - sy) ** 2
    assert d2.max() == 10
    assert len(set(zip((tx - sx).tolist(), (ty - sy).tolist()))) == 37


@pytest.mark.parametrize("n", [32, 64])
def test_boundary_lists_partition_all_pairs(n):
    P = O.Problem(n, p=4)
    L = P.L
    nl, nb = 4 ** L, 4 * 2 ** L
    cover = np.zeros((nl, nb), np.int32)
    pvb = P.export(O.E_P2P_VB)
    cover[pvb[:, 0], pvb[:, 1]] += 1
    leaves = np.arange(nl)
    bl = np.arange(nb)
    for l, v, b in P.export(O.E_M2L_VB):
        ts = leaves[(leaves >> (2 * (L - l))) == v]
        side, k = b >> l, b & ((1 << l) - 1)
        ss = bl[((bl >> L) == side) & (((bl & ((1 << L) - 1)) >> (L - l)) == k)]
        cover[np.ix_(ts, ss)] += 1
    assert cover.min() == 1 and cover.max() == 1

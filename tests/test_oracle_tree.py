"""Pins of the oracle's octree, Morton order and interaction lists (Sec. 2, Eq. (2), Sec. 3.2.1).

Every check below recomputes the object from its definition by brute force in
Python (containment of points in half-open boxes, the infinity-norm neighbour
rule, the cousin rule through parents) and compares with the oracle.
"""
import itertools

import numpy as np
import pytest

import ifgf_inputs as W
import oracle


def _decode(key: int):
    k = [0, 0, 0]
    for b in range(21):
        for ax in range(3):
            k[ax] |= ((key >> (3 * b + ax)) & 1) << b
    return tuple(k)


def _brute_boxes(points, a, H1, d):
    """Level-d boxes by direct containment a + k H_d <= x < a + (k+1) H_d (half-open)."""
    Hd = H1 / 2 ** (d - 1)
    n = points.shape[1]
    side = 2 ** (d - 1)
    boxes = {}
    for i in range(n):
        k = []
        for ax in range(3):
            lo = 0
            # smallest k with x < a + (k+1) Hd, scanning all boxes of the axis
            for kk in range(side):
                if a[ax] + kk * Hd <= points[ax, i] < a[ax] + (kk + 1) * Hd:
                    lo = kk
                    break
            else:
                lo = side - 1
            k.append(lo)
        boxes.setdefault(tuple(k), set()).add(i)
    return boxes


@pytest.fixture(scope="module")
def small_plan():
    pts = W.random_cloud(700, seed=21)
    p = oracle.Plan(pts, 5.0, levels=5)
    return pts, p


def test_boxes_match_containment(small_plan):
    pts, p = small_plan
    perm = p.get(oracle.Q_PERM)
    assert sorted(perm.tolist()) == list(range(pts.shape[1]))
    for d in range(1, p.D + 1):
        brute = _brute_boxes(pts, p.a, p.H1, d)
        keys = p.get(oracle.Q_BOX_KEYS, d)
        start = p.get(oracle.Q_BOX_START, d)
        got = {}
        for b, key in enumerate(keys):
            got[_decode(int(key))] = set(perm[start[b]:start[b + 1]].tolist())
        assert got == brute, f"level {d}"
        assert np.all(np.diff(keys) > 0)


def test_root_cube_contains_points(small_plan):
    pts, p = small_plan
    assert np.all(pts >= p.a[:, None]) and np.all(pts < (p.a + p.H1)[:, None])
    ext = (pts.max(axis=1) - pts.min(axis=1)).max()
    assert ext < p.H1 < ext * (1 + 2e-6)


def test_morton_order_and_ties():
    # Duplicate-free cloud with many points sharing level-21 cells is impossible at random;
    # build clusters so that equal keys occur: ties must follow the original index.
    rng = np.random.default_rng(5)
    base = rng.uniform(-1, 1, size=(3, 50))
    pts = np.repeat(base, 4, axis=1) + rng.uniform(0, 1e-9, size=(3, 200))
    pts[:, 0] = [-1.5, -1.5, -1.5]
    pts[:, 1] = [1.5, 1.5, 1.5]
    p = oracle.Plan(pts, 1.0, levels=4)
    keys = p.get(oracle.Q_KEYS)
    perm = p.get(oracle.Q_PERM)
    assert np.all(np.diff(keys) >= 0)
    eq = np.diff(keys) == 0
    assert eq.sum() > 50
    assert np.all(np.diff(perm)[eq] > 0)
    # Points of every box are contiguous at every level: box of point i is non-decreasing.
    for d in range(1, p.D + 1):
        start = p.get(oracle.Q_BOX_START, d)
        assert start[0] == 0 and start[-1] == p.N and np.all(np.diff(start) > 0)


def test_neighbours_and_cousins_brute_force(small_plan):
    pts, p = small_plan
    for d in range(2, p.D + 1):
        keys = p.get(oracle.Q_BOX_KEYS, d)
        coords = [_decode(int(k)) for k in keys]
        idx = {c: i for i, c in enumerate(coords)}
        cnt = p.get(oracle.Q_NBR_COUNT, d)
        flat = p.get(oracle.Q_NBR_LIST, d)
        off = np.concatenate([[0], np.cumsum(cnt)])
        for b, kb in enumerate(coords):
            want = sorted(idx[c] for c in coords if max(abs(c[i] - kb[i]) for i in range(3)) <= 1)
            assert flat[off[b]:off[b + 1]].tolist() == want
            assert len(want) <= 27
        if d < 3:
            continue
        pkeys = p.get(oracle.Q_BOX_KEYS, d - 1)
        pcoords = [_decode(int(k)) for k in pkeys]
        ccnt = p.get(oracle.Q_COUS_COUNT, d)
        cflat = p.get(oracle.Q_COUS_LIST, d)
        coff = np.concatenate([[0], np.cumsum(ccnt)])
        for b, kb in enumerate(coords):
            pk = tuple(v // 2 for v in kb)
            want = []
            for j, c in enumerate(coords):
                pc = tuple(v // 2 for v in c)
                if max(abs(c[i] - kb[i]) for i in range(3)) > 1 and max(abs(pc[i] - pk[i]) for i in range(3)) <= 1:
                    want.append(j)
            assert cflat[coff[b]:coff[b + 1]].tolist() == want
            assert len(want) <= 189


def test_interaction_partition():
    """Every ordered pair (l, m), m != l, is either a leaf-neighbour pair or a cousin pair at
    exactly one level d in [3, D] -- the property that makes IFGF with exact interpolation equal
    the direct sum; at d = 3 every box is a neighbour or cousin of every other (Sec. 2)."""
    pts = W.fibonacci_sphere(900)
    p = oracle.Plan(pts, 10.0, levels=5)
    perm = p.get(oracle.Q_PERM)
    N = p.N
    box_of = {}
    for d in range(3, p.D + 1):
        start = p.get(oracle.Q_BOX_START, d)
        bo = np.empty(N, dtype=np.int64)
        for b in range(len(start) - 1):
            bo[perm[start[b]:start[b + 1]]] = b
        box_of[d] = bo
    def csr(what_c, what_l, d):
        c = p.get(what_c, d)
        f = p.get(what_l, d)
        o = np.concatenate([[0], np.cumsum(c)])
        return [set(f[o[b]:o[b + 1]].tolist()) for b in range(len(c))]
    near = csr(oracle.Q_NBR_COUNT, oracle.Q_NBR_LIST, p.D)
    cous = {d: csr(oracle.Q_COUS_COUNT, oracle.Q_COUS_LIST, d) for d in range(3, p.D + 1)}
    for l in range(0, N, 7):
        for m in range(N):
            if m == l:
                continue
            hits = int(box_of[p.D][m] in near[box_of[p.D][l]])
            hits += sum(int(box_of[d][m] in cous[d][box_of[d][l]]) for d in range(3, p.D + 1))
            assert hits == 1, (l, m)


def test_level_choice_rule():
    pts = W.fibonacci_sphere(5000)
    for target in (16, 64, 200):
        p = oracle.Plan(pts, 1.0, leaf_target=target)
        assert p.N <= target * p.nbox[p.D]
        if p.D > 3:
            q = oracle.Plan(pts, 1.0, levels=p.D - 1)
            assert p.N > target * q.nbox[p.D - 1]


@pytest.mark.parametrize("bad", ["n1", "kappa", "levels", "coincident_all"])
def test_rejects_invalid(bad):
    pts = W.random_cloud(10, seed=1)
    if bad == "n1":
        with pytest.raises(oracle.OracleError):
            oracle.Plan(pts[:, :1], 1.0)
    elif bad == "kappa":
        with pytest.raises(oracle.OracleError):
            oracle.Plan(pts, -1.0)
    elif bad == "levels":
        with pytest.raises(oracle.OracleError):
            oracle.Plan(pts, 1.0, levels=2)
    else:
        with pytest.raises(oracle.OracleError):
            oracle.Plan(np.zeros((3, 5)), 1.0)


def test_duplicate_detection():
    pts = W.random_cloud(50, seed=2)
    assert not oracle.Plan(pts, 1.0, levels=3).has_duplicates()
    pts[:, 7] = pts[:, 30]
    assert oracle.Plan(pts, 1.0, levels=3).has_duplicates()

"""Pins of the oracle's statement of the distribution over ranks (Sec. 3.2), and the library's
host-side partition functions against it.

- Partitions: the leaf-box intervals cover every box once, in order, and each rank's point count
  is within one leaf box of N / nranks (the bound Sec. 3.2.1 states); cone intervals differ in
  size by at most one.  The library's host functions give the same intervals.
- What a rank reads (M1): over all ranks, the cones looked up by Interpolation and Propagation are
  exactly the relevant cones (every relevant cone has a witness, Eq. (4), and every lookup hits);
  for one rank, the lookups agree with a brute force in FP64 spherical coordinates away from cone
  edges; the points read are the neighbour boxes' points and the own leaf cones' boxes' points.
- Volume (Sec. 3.3): the cones a level sends between ranks stay a bounded multiple of the level's
  relevant cones, not growing with N.
"""
import math
import os

import numpy as np
import pytest

import ifgf_inputs as W
import oracle
from test_oracle_cones import _candidates, _cheb_nodes, _demorton

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import shutil

    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2112_15198_gb300 as ifgf

    ifgf.load(build=True)
    return ifgf


@pytest.mark.parametrize("nranks", [1, 2, 3, 7, 16])
def test_partitions(nranks):
    pts = W.spheroid(6000, 0.5, 0.2, seed=3)
    p = oracle.Plan(pts, 2 * math.pi * 4)
    start = p.get(oracle.Q_BOX_START, p.D)
    b = oracle.partition_boxes(start, nranks)
    assert b[0] == 0 and b[-1] == len(start) - 1 and np.all(np.diff(b) >= 0)
    counts = start[b[1:]] - start[b[:-1]]
    assert counts.sum() == p.N
    biggest = np.max(np.diff(start))
    assert np.all(np.abs(counts - p.N / nranks) <= biggest), (counts, biggest)
    for d in range(3, p.D + 1):
        c = oracle.partition_cones(p.ncone[d], nranks)
        assert c[0] == 0 and c[-1] == p.ncone[d] and np.max(np.diff(c)) - np.min(np.diff(c)) <= 1
    ifgf = _lib()
    np.testing.assert_array_equal(ifgf.partition_boxes(start, nranks), b)
    for d in range(3, p.D + 1):
        np.testing.assert_array_equal(ifgf.partition_cones(p.ncone[d], nranks), oracle.partition_cones(p.ncone[d], nranks))


def _ranks(p, nranks):
    start = p.get(oracle.Q_BOX_START, p.D)
    b = oracle.partition_boxes(start, nranks)
    pts = [(int(start[b[r]]), int(start[b[r + 1]])) for r in range(nranks)]
    cones = {d: oracle.partition_cones(p.ncone[d], nranks) for d in range(3, p.D + 1)}
    return pts, cones


@pytest.mark.parametrize("case", ["sphere", "prolate", "laplace"])
def test_union_of_lookups_is_the_relevant_set(case):
    pts = {"sphere": W.fibonacci_sphere(5000), "prolate": W.spheroid(5000, 0.05, 0.5, seed=8),
           "laplace": W.fibonacci_sphere(5000)}[case]
    kappa = 0.0 if case == "laplace" else 2 * math.pi * 5
    p = oracle.Plan(pts, kappa, levels=5)
    for nranks in (1, 3):
        ranges, cones = _ranks(p, nranks)
        for d in range(3, p.D + 1):
            seen = np.zeros(p.ncone[d], dtype=np.uint8)
            for r in range(nranks):
                pc = (int(cones[d - 1][r]), int(cones[d - 1][r + 1])) if d > 3 else (0, 0)
                seen |= p.shard_cones(d, ranges[r], pc)
            # R1: a cone is relevant iff a cousin point or a node of a relevant parent cone lies in it
            assert np.all(seen > 0), (nranks, d)
            if d > 3:
                assert np.any(seen & 2)  # propagation reads cones at every level below 3


def test_one_rank_lookups_match_fp64_geometry():
    pts = W.fibonacci_sphere(4000)
    kappa = 2 * math.pi * 6
    p = oracle.Plan(pts, kappa, levels=5)
    nranks, r = 3, 1
    ranges, cones = _ranks(p, nranks)
    perm = p.get(oracle.Q_PERM)
    X = pts[:, perm].T
    ts, tt, tp = _cheb_nodes(3), _cheb_nodes(5), _cheb_nodes(5)
    eta = math.sqrt(3.0) / 3.0
    for d in range(4, p.D + 1):
        grid = p.grid(d)
        C = grid[0] * grid[1] * grid[2]
        h = 0.5 * math.sqrt(3.0) * p.H1 * 2.0 ** (1 - d)
        centres = p.a[None, :] + (_demorton(p.get(oracle.Q_BOX_KEYS, d)) + 0.5) * p.H1 * 2.0 ** (1 - d)
        cbox, cgam = p.get(oracle.Q_CONE_BOX, d), p.get(oracle.Q_CONE_GAMMA, d)
        index = {int(b) * C + int(g): i for i, (b, g) in enumerate(zip(cbox, cgam))}
        pc = (int(cones[d - 1][r]), int(cones[d - 1][r + 1]))
        got = p.shard_cones(d, ranges[r], pc)
        # interpolation: the rank's points and the cousins of their level-d boxes
        start = p.get(oracle.Q_BOX_START, d)
        box_of = np.searchsorted(start, np.arange(p.N), side="right") - 1
        cc, cl = p.get(oracle.Q_COUS_COUNT, d), p.get(oracle.Q_COUS_LIST, d)
        coff = np.concatenate([[0], np.cumsum(cc)])
        own_pts = np.arange(*ranges[r])
        owner, pt = [], []
        for i in own_pts:
            cs = cl[coff[box_of[i]]:coff[box_of[i] + 1]]
            owner.append(cs)
            pt.append(np.full(cs.shape[0], i))
        owner, pt = np.concatenate(owner), np.concatenate(pt)
        g, dec, poss = _candidates(X[pt] - centres[owner], h, grid)
        decided = {index[int(k)] for k in owner[dec] * C + g[dec]}
        possible = {index[int(k)] for rows, gg in poss for k in owner[rows] * C + gg if int(k) in index}
        bit0 = set(np.nonzero(got & 1)[0].tolist())
        assert decided <= bit0 <= possible, d
        # propagation: the nodes of the rank's level-(d-1) cones in each child box
        Hp = p.H1 * 2.0 ** (2 - d)
        pgrid = p.grid(d - 1)
        pcentres = p.a[None, :] + (_demorton(p.get(oracle.Q_BOX_KEYS, d - 1)) + 0.5) * Hp
        pbox, pgam = p.get(oracle.Q_CONE_BOX, d - 1), p.get(oracle.Q_CONE_GAMMA, d - 1)
        parent = p.get(oracle.Q_BOX_PARENT, d)
        kids_of = {}
        for k, par in enumerate(parent):
            kids_of.setdefault(int(par), []).append(k)
        decided, possible = set(), set()
        hp = 0.5 * math.sqrt(3.0) * Hp
        for c in range(*pc):
            gm = int(pgam[c])
            ip, it, is_ = gm % pgrid[2], (gm // pgrid[2]) % pgrid[1], gm // (pgrid[2] * pgrid[1])
            s = (eta / pgrid[0]) * (is_ + 0.5 * (1.0 + ts))
            th = (math.pi / pgrid[1]) * (it + 0.5 * (1.0 + tt))
            ph = (2 * math.pi / pgrid[2]) * (ip + 0.5 * (1.0 + tp))
            rr = hp / s
            nodes = np.array([[rr[a] * math.sin(th[b]) * math.cos(ph[q]), rr[a] * math.sin(th[b]) * math.sin(ph[q]),
                               rr[a] * math.cos(th[b])] for a in range(3) for b in range(5) for q in range(5)])
            nodes += pcentres[int(pbox[c])]
            kids = np.array(kids_of[int(pbox[c])])
            own = np.repeat(kids, nodes.shape[0])
            v = np.tile(nodes, (kids.shape[0], 1)) - centres[own]
            g, dec, poss = _candidates(v, h, grid)
            decided |= {index[int(k)] for k in own[dec] * C + g[dec]}
            possible |= {index[int(k)] for rows, gg in poss for k in own[rows] * C + gg if int(k) in index}
        bit1 = set(np.nonzero(got & 2)[0].tolist())
        assert decided <= bit1 <= possible, d


def test_points_read_by_a_rank():
    pts = W.spheroid(5000, 0.5, 0.125, seed=4)
    p = oracle.Plan(pts, 2 * math.pi * 4)
    nranks = 4
    ranges, cones = _ranks(p, nranks)
    D = p.D
    start = p.get(oracle.Q_BOX_START, D)
    ncount, nlist = p.get(oracle.Q_NBR_COUNT, D), p.get(oracle.Q_NBR_LIST, D)
    noff = np.concatenate([[0], np.cumsum(ncount)])
    cbox = p.get(oracle.Q_CONE_BOX, D)
    for r in range(nranks):
        c = (int(cones[D][r]), int(cones[D][r + 1]))
        got = p.shard_points(ranges[r], c)
        b0, b1 = np.searchsorted(start, ranges[r][0]), np.searchsorted(start, ranges[r][1])
        near = np.zeros(p.N, dtype=bool)
        for b in range(b0, b1):
            for q in nlist[noff[b]:noff[b + 1]]:
                near[start[q]:start[q + 1]] = True
        leaf = np.zeros(p.N, dtype=bool)
        for b in set(cbox[c[0]:c[1]].tolist()):
            leaf[start[b]:start[b + 1]] = True
        np.testing.assert_array_equal((got & 1) > 0, near)
        np.testing.assert_array_equal((got & 2) > 0, leaf)


def test_exchange_volume_is_linear():
    """Sec. 3.3: each relevant cone is sent to O(1) ranks, so the cones a level sends are a bounded
    multiple of its relevant cones, whatever N."""
    ratios = []
    for n, lam in ((6000, 3.0), (24000, 6.0)):
        pts = W.fibonacci_sphere(n)
        p = oracle.Plan(pts, 2 * math.pi * lam)
        nranks = 8
        ranges, cones = _ranks(p, nranks)
        worst = 0.0
        for d in range(3, p.D + 1):
            sent = 0
            for r in range(nranks):
                pc = (int(cones[d - 1][r]), int(cones[d - 1][r + 1])) if d > 3 else (0, 0)
                got = p.shard_cones(d, ranges[r], pc)
                own = np.zeros_like(got, dtype=bool)
                own[cones[d][r]:cones[d][r + 1]] = True
                sent += int(np.count_nonzero((got > 0) & ~own))
            worst = max(worst, sent / p.ncone[d])
        ratios.append(worst)
        print(f"N = {n}: largest cones sent per relevant cone over the levels = {worst:.2f}")
    assert all(x <= 8.0 for x in ratios)
    assert ratios[1] <= 2.0 * ratios[0] + 0.5

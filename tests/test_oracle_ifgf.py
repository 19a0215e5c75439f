"""Pins of the oracle's IFGF (O2) against facts other than itself.

- Chebyshev interpolants reproduce polynomials of the orders' degrees exactly.
- Cone classification agrees with FP64 spherical coordinates away from cone edges.
- Exact special case: with one point at the centre of every leaf box, g_k == 1, so the
  leaf fields F_k are constant and their interpolation is exact (Eq. (3)); with D = 3
  the whole IFGF must then equal the direct sum of Eq. (1) to rounding, and with D = 4
  the level-4 cousin interpolations must equal the level-4 cousin pair sums.
- Spectral convergence: the error against the direct sum falls geometrically as the
  orders grow and as the cone grids refine (any wrong term would leave a plateau).
- End to end: the default orders (3,5,5) reach the stated accuracy on the 4-wavelength
  sphere, for the Helmholtz and the Laplace kernels.
"""
import math

import numpy as np
import pytest

import ifgf_inputs as W
import oracle


def test_chebyshev_reproduces_polynomials():
    pts = W.random_cloud(100, seed=1)
    p = oracle.Plan(pts, 1.0, levels=3, orders=(3, 5, 5))
    ts, tt, tp = p.cheb_nodes()
    rng = np.random.default_rng(0)
    C = rng.standard_normal((3, 5, 5)) + 1j * rng.standard_normal((3, 5, 5))

    def poly(a, b, c):  # sum C_ijk a^i b^j c^k, total degree per variable < order
        return sum(C[i, j, k] * a ** i * b ** j * c ** k for i in range(3) for j in range(5) for k in range(5))

    vals = np.array([poly(a, b, c) for a in ts for b in tt for c in tp])
    coef = p.cheb3(vals)
    t = rng.uniform(-1, 1, size=(50, 3))
    got = p.cheb3_eval(coef, t)
    want = np.array([poly(*x) for x in t])
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    # node values are reproduced exactly by the coefficient transform
    tn = np.array([[a, b, c] for a in ts for b in tt for c in tp])
    assert np.max(np.abs(p.cheb3_eval(coef, tn) - vals)) < 1e-12 * np.max(np.abs(vals))


@pytest.mark.parametrize("level", [3, 4, 5])
def test_classification_matches_spherical_coordinates(level):
    pts = W.fibonacci_sphere(6000)
    p = oracle.Plan(pts, 2 * math.pi * 8, levels=5)
    ns, nt, np_ = p.grid(level)
    hg = math.sqrt(3.0) * 2.0 ** (p.D - level)
    eta = math.sqrt(3.0) / 3.0
    rng = np.random.default_rng(level)
    n = 20000
    dirs = rng.standard_normal((n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = hg / rng.uniform(0.02, eta, size=n)
    v = (dirs * r[:, None]).astype(np.float32)
    got = p.classify(level, v)
    vv = v.astype(np.float64)
    rr = np.linalg.norm(vv, axis=1)
    s = hg / rr
    th = np.arccos(np.clip(vv[:, 2] / rr, -1, 1))
    ph = np.mod(np.arctan2(vv[:, 1], vv[:, 0]), 2 * math.pi)
    fs, ft, fp = s / (eta / ns), th / (math.pi / nt), ph / (2 * math.pi / np_)
    is_ = np.minimum(np.floor(fs).astype(int), ns - 1)
    it = np.minimum(np.floor(ft).astype(int), nt - 1)
    ip = np.minimum(np.floor(fp).astype(int), np_ - 1)
    want = (is_ * nt + it) * np_ + ip

    def near_edge(f):
        return np.abs(f - np.round(f)) < 1e-5

    ok = (got == want) | near_edge(fs) | near_edge(ft) | near_edge(fp)
    assert ok.all(), np.nonzero(~ok)[0][:10]
    assert (got == want).mean() > 0.999


def _centre_points(levels, n_boxes, seed):
    """Zero-density anchors at (0,0,0), (1,1,1) fix the root cube; one point at the centre of
    n_boxes random level-`levels` boxes carries a nonzero density."""
    H1 = 1.0 * (1.0 + 2.0 ** -20)
    a = 0.5 * (0.0 + 1.0) - 0.5 * H1
    Hd = H1 * 2.0 ** (1 - levels)
    side = 2 ** (levels - 1)
    rng = np.random.default_rng(seed)
    cells = rng.choice(side ** 3, size=n_boxes, replace=False)
    pts = [[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]
    for c in cells:
        k = (c % side, (c // side) % side, c // (side * side))
        pts.append([a + (k[i] + 0.5) * Hd for i in range(3)])
    pts = np.array(pts).T.copy()
    dens = W.densities(pts.shape[1], 1, seed + 1)[0]
    dens[:2] = 0.0
    return pts, dens, a, H1


def test_exact_when_leaf_fields_are_constant_D3():
    pts, dens, a, H1 = _centre_points(3, 40, 3)
    for kappa in (0.0, 9.0, 40.0):
        p = oracle.Plan(pts, kappa, levels=3)
        assert p.H1 == H1 and np.all(p.a == a)
        got = p.apply(dens)[0]
        want = oracle.direct_sum(pts, kappa, dens)[0]
        assert oracle.rel_l2(got, want) < 1e-12


def test_level4_interpolation_exact_for_centred_points():
    pts, dens, a, H1 = _centre_points(4, 300, 7)
    kappa = 25.0
    p = oracle.Plan(pts, kappa, levels=4)
    got = p.apply(dens, near=False, level_mask=1 << 4)[0]
    # brute force: pairs whose level-4 boxes are cousins
    perm = p.get(oracle.Q_PERM)
    start = p.get(oracle.Q_BOX_START, 4)
    box = np.empty(p.N, dtype=np.int64)
    for b in range(len(start) - 1):
        box[perm[start[b]:start[b + 1]]] = b
    cc = p.get(oracle.Q_COUS_COUNT, 4)
    cl = p.get(oracle.Q_COUS_LIST, 4)
    off = np.concatenate([[0], np.cumsum(cc)])
    want = np.zeros(p.N, dtype=np.complex128)
    for l in range(p.N):
        cous = set(cl[off[box[l]]:off[box[l] + 1]].tolist())
        for m in range(p.N):
            if m != l and box[m] in cous:
                r = np.linalg.norm(pts[:, l] - pts[:, m])
                want[l] += dens[m] * np.exp(1j * kappa * r) / (4 * math.pi * r)
    assert oracle.rel_l2(got, want) < 1e-12


def test_spectral_convergence_in_orders_and_cones():
    n = 2000
    pts = W.fibonacci_sphere(n)
    kappa = 2 * math.pi * 2
    dens = W.densities(n, 1, 5)
    exact = oracle.direct_sum(pts, kappa, dens)
    errs = []
    for orders in [(3, 5, 5), (5, 7, 7), (7, 9, 9)]:
        p = oracle.Plan(pts, kappa, orders=orders, levels=4)
        errs.append(oracle.rel_l2(p.apply(dens), exact))
    assert errs[0] < 3e-4
    assert errs[1] < errs[0] / 20 and errs[2] < errs[1] / 20
    coarse = oracle.rel_l2(oracle.Plan(pts, kappa, levels=4, base_cones=(1, 2, 4)).apply(dens), exact)
    fine = oracle.rel_l2(oracle.Plan(pts, kappa, levels=4, base_cones=(4, 8, 16)).apply(dens), exact)
    assert fine < errs[0] / 5 < coarse / 5


@pytest.mark.parametrize("kappa_wl", [4.0, 0.0])
def test_default_orders_reach_stated_accuracy(kappa_wl):
    w = W.make("sphere4")
    pts = w.points()
    kappa = 2 * math.pi * kappa_wl
    dens = w.densities()
    tg = W.targets(w.n, 3000, 99)
    p = oracle.Plan(pts, kappa)
    got = p.apply(dens)[:, tg]
    exact = oracle.direct_sum(pts, kappa, dens, tg)
    err = oracle.rel_l2(got, exact)
    assert err < 2e-4, err
    assert p.status == 0


def test_multiple_rhs_match_single_rhs():
    pts = W.fibonacci_sphere(3000)
    p = oracle.Plan(pts, 2 * math.pi * 3)
    A = W.densities(3000, 3, 2)
    all3 = p.apply(A)
    for r in range(3):
        assert np.array_equal(p.apply(A[r])[0], all3[r])


def test_relevant_cone_statistics():
    """Each level-d cone feeds a few parent cones (most often one); the counts per level stay
    of the same order across levels (Sec. 3.3)."""
    pts = W.fibonacci_sphere(20000)
    p = oracle.Plan(pts, 2 * math.pi * 8)
    counts = [p.ncone[d] for d in range(3, p.D + 1)]
    assert min(counts) > 0
    assert max(counts) / min(counts) < 50

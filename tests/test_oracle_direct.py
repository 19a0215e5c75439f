"""Pins of the direct-sum oracle O1 (Eq. (1)) against facts other than its own formula.

- The kernel G is pinned by the PDE it solves: the Helmholtz equation away from the
  source (finite differences), the outgoing radiation condition (which fixes the sign
  of the exponent), and the unit point-source flux (which fixes 1/(4 pi)).
- The summation is pinned by single-source indexing, self-exclusion, reciprocity of the
  symmetric kernel, linearity, the kappa -> 0 limit, and an independent extended
  precision brute force on tiny inputs.
- Both together by the closed form of the single layer over a sphere (a quadrature of it).
"""
import math

import numpy as np
import pytest

import ifgf_inputs as W
import oracle


def _one_source(points, kappa, src, tgt):
    n = points.shape[1]
    a = np.zeros(n, dtype=np.complex128)
    a[src] = 1.0
    return oracle.direct_sum(points, kappa, a, np.asarray(tgt))[0]


def _probe(kappa, x0, offsets):
    """Field of a unit source at the origin, seen at x0 + offsets[i] (points 1..)."""
    pts = np.zeros((3, 1 + len(offsets)))
    for i, o in enumerate(offsets):
        pts[:, 1 + i] = x0 + o
    return _one_source(pts, kappa, 0, np.arange(1, 1 + len(offsets)))


@pytest.mark.parametrize("kappa", [0.0, 3.0, 25.0])
def test_helmholtz_equation_away_from_source(kappa):
    # (Laplacian + kappa^2) G = 0 for x != y: second-order central differences.
    x0 = np.array([0.31, -0.22, 0.17])
    h = 1e-3
    offs = [np.zeros(3)]
    for ax in range(3):
        for sgn in (1, -1):
            e = np.zeros(3)
            e[ax] = sgn * h
            offs.append(e)
    g = _probe(kappa, x0, offs)
    lap = (g[1:].sum() - 6.0 * g[0]) / (h * h)
    scale = max(kappa * kappa, 1.0 / np.dot(x0, x0)) * abs(g[0])
    assert abs(lap + kappa * kappa * g[0]) < 1e-4 * scale


def test_outgoing_radiation_condition():
    # r (dG/dr - i kappa G) -> 0 for the outgoing e^{+i kappa r}; the incoming sign gives 2 kappa r |G|.
    kappa = 5.0
    d = np.array([1.0, 2.0, 2.0]) / 3.0
    for r in (50.0, 200.0):
        h = 1e-4
        g = _probe(kappa, np.zeros(3), [d * (r - h), d * r, d * (r + h)])
        dgdr = (g[2] - g[0]) / (2 * h)
        resid = r * abs(dgdr - 1j * kappa * g[1])
        # outgoing: r |dG/dr - i kappa G| = |G| = 1/(4 pi r) -> 0; incoming would give ~2 kappa r |G|
        assert resid < 1.01 * abs(g[1])
        assert abs(abs(g[1]) - 1.0 / (4 * math.pi * r)) < 1e-12


def test_unit_point_source_flux():
    # The flux of grad G through a small sphere tends to -1 (G is the fundamental solution).
    kappa = 2.0
    d = np.array([0.0, 0.6, 0.8])
    r, h = 1e-3, 1e-7
    g = _probe(kappa, np.zeros(3), [d * (r - h), d * (r + h)])
    flux = 4 * math.pi * r * r * (g[1] - g[0]) / (2 * h)
    assert abs(flux + 1.0) < 1e-2


def test_single_source_indexing_and_self_exclusion():
    pts = W.random_cloud(40, seed=3)
    kappa = 7.0
    src = 17
    out = _one_source(pts, kappa, src, np.arange(40))
    assert out[src] == 0  # m != l: no self term
    r = np.linalg.norm(pts - pts[:, [src]], axis=0)
    for l in range(40):
        if l != src:
            # only the source column contributes, with a field of modulus 1/(4 pi r)
            assert abs(abs(out[l]) - 1.0 / (4 * math.pi * r[l])) < 1e-15 / r[l] * 10


def test_reciprocity_of_symmetric_kernel():
    # G(x,y) = G(y,x) makes the matrix symmetric: b . (A a) = a . (A b) (unconjugated).
    pts = W.random_cloud(300, seed=4)
    kappa = 11.0
    a = W.densities(300, 1, 5)[0]
    b = W.densities(300, 1, 6)[0]
    Aa = oracle.direct_sum(pts, kappa, a)[0]
    Ab = oracle.direct_sum(pts, kappa, b)[0]
    lhs, rhs = np.dot(b, Aa), np.dot(a, Ab)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_linearity_and_multiple_rhs():
    pts = W.random_cloud(200, seed=7)
    kappa = 4.0
    A = W.densities(200, 3, 8)
    out = oracle.direct_sum(pts, kappa, A)
    comb = oracle.direct_sum(pts, kappa, 2.0 * A[0] - 1j * A[1] + 0.5 * A[2])[0]
    assert np.max(np.abs(comb - (2.0 * out[0] - 1j * out[1] + 0.5 * out[2]))) < 1e-12 * np.max(np.abs(comb))


def test_kappa_to_zero_limit():
    # |G_kappa - G_0| <= kappa/(4 pi) for every pair, so the difference is O(kappa r_max).
    pts = W.random_cloud(150, seed=9)
    a = W.densities(150, 1, 10)[0]
    base = oracle.direct_sum(pts, 0.0, a)[0]
    prev = None
    for kappa in (1e-2, 1e-3, 1e-4):
        diff = np.max(np.abs(oracle.direct_sum(pts, kappa, a)[0] - base))
        assert diff <= kappa / (4 * math.pi) * np.sum(np.abs(a)) * 1.0001
        if prev is not None:
            assert diff < 0.2 * prev
        prev = diff


def test_brute_force_extended_precision_tiny():
    # Independent evaluation in numpy long double on a tiny cloud.
    n = 48
    pts = W.random_cloud(n, seed=12)
    kappa = 9.0
    a = W.densities(n, 1, 13)[0]
    out = oracle.direct_sum(pts, kappa, a)[0]
    P = pts.astype(np.longdouble)
    k = np.longdouble(kappa)
    four_pi = np.longdouble(4) * np.arccos(np.longdouble(-1))
    for l in range(n):
        d = P - P[:, [l]]
        r = np.sqrt((d * d).sum(axis=0))
        r[l] = 1
        re = np.cos(k * r) / (four_pi * r)
        im = np.sin(k * r) / (four_pi * r)
        re[l] = im[l] = 0
        ar, ai = a.real.astype(np.longdouble), a.imag.astype(np.longdouble)
        val_re = float(np.sum(ar * re - ai * im))
        val_im = float(np.sum(ar * im + ai * re))
        assert abs(out[l] - (val_re + 1j * val_im)) < 1e-14 * max(1.0, abs(out[l]))


def sphere_single_layer(kappa, a, x):
    """Closed form of the single layer of unit density over the sphere |y| = a (addition theorem,
    only the n = 0 term survives the surface integral): a e^{i kappa a} sin(kappa r)/(kappa r) for
    r = |x| < a and a sin(kappa a) e^{i kappa r}/(kappa r) for r > a (a and a^2/r at kappa = 0)."""
    r = float(np.linalg.norm(x))
    if kappa == 0.0:
        return a if r < a else a * a / r
    if r < a:
        return a * np.exp(1j * kappa * a) * (np.sin(kappa * r) / (kappa * r) if r > 0 else 1.0)
    return a * np.sin(kappa * a) * np.exp(1j * kappa * r) / (kappa * r)


@pytest.mark.parametrize("kappa", [0.0, 2 * math.pi * 3])
def test_sphere_single_layer_closed_form(kappa):
    """Eq. (1) as a quadrature of the single layer over a Fibonacci sphere of radius 1/2 (weights
    area / N), seen at interior and exterior points that carry no density."""
    n, a = 20000, 0.5
    probes = np.array([[0.0, 0.0, 0.0], [0.1, -0.05, 0.2], [-0.2, 0.15, -0.1],
                       [0.9, 0.3, -0.4], [-0.2, 0.6, 0.5]]).T
    pts = np.concatenate([W.fibonacci_sphere(n), probes], axis=1)
    dens = np.zeros(pts.shape[1], dtype=np.complex128)
    dens[:n] = 4 * math.pi * a * a / n
    got = oracle.direct_sum(pts, kappa, dens, np.arange(n, pts.shape[1]))[0]
    for t in range(probes.shape[1]):
        want = sphere_single_layer(kappa, a, probes[:, t])
        assert abs(got[t] - want) <= 2e-5 * max(abs(want), 0.1), (t, got[t], want)

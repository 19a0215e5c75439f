"""Pins of the Stokes oracle (S1 direct sum, S2 IFGF apply) against closed forms of Stokes flow.

The Stokeslet S_ij = (delta_ij/r + r_i r_j/r^3)/(8 pi) is the Green tensor of the Stokes
equations at unit viscosity, one of the kernels Sec. 2 names for Eq. (1).  Its single-layer
potential over a sphere of radius a with the uniform traction of a translating sphere is known in
closed form (Stokes' solution): the velocity is the rigid translation U = 2 a f / 3 inside the
sphere and Stokes' exterior flow outside it.  Both fix the normalisation 1/(8 pi) and the relative
weight of the two terms of S; the divergence-free property fixes that weight independently.
"""
import numpy as np
import pytest

import ifgf_inputs as W
import oracle


def _sphere_single_layer(n, extra, forces):
    """Points: n Fibonacci points on the sphere of radius 1/2, then `extra` targets with zero force."""
    a = 0.5
    surf = W.fibonacci_sphere(n)
    pts = np.concatenate([surf, extra], axis=1)
    m = pts.shape[1]
    f = np.zeros((len(forces), 3, m))
    for s, e in enumerate(forces):
        f[s, :, :n] = np.asarray(e)[:, None] * (4.0 * np.pi * a * a / n)  # traction x area weight
    return a, pts, f, np.arange(n, m)


def test_stokeslet_sphere_single_layer_closed_form():
    inside = np.array([[0.0, 0.0, 0.0], [0.1, -0.05, 0.2], [-0.2, 0.15, -0.1]]).T
    outside = np.array([[0.9, 0.3, -0.4], [-0.2, 0.6, 0.5]]).T
    dirs = [np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]), np.array([0.3, -0.5, 0.8])]
    a, pts, f, tgt = _sphere_single_layer(20000, np.concatenate([inside, outside], axis=1), dirs)
    u = oracle.stokes_direct_sum(pts, f, tgt)
    for s, e in enumerate(dirs):
        U = 2.0 * a / 3.0 * e  # rigid translation: traction 3U/(2a) per unit area, unit viscosity
        for t in range(inside.shape[1]):
            assert np.abs(u[s, :, t] - U).max() <= 1e-5 * np.abs(U).max()
        for t in range(outside.shape[1]):
            x = outside[:, t]
            r = np.linalg.norm(x)
            ue = (0.75 * a) * (U / r + (U @ x) * x / r**3) + (a**3 / 4.0) * (U / r**3 - 3.0 * (U @ x) * x / r**5)
            assert np.abs(u[s, :, inside.shape[1] + t] - ue).max() <= 1e-5 * np.abs(ue).max()


def test_stokeslet_divergence_free():
    """div_x S(x, y) f = 0 away from the source (second-order central differences)."""
    y = np.array([0.1, 0.2, -0.1])
    x = np.array([0.4, -0.3, 0.25])
    h = 1e-4
    pts = [y]
    for k in range(3):
        for sg in (1.0, -1.0):
            e = np.zeros(3)
            e[k] = sg * h
            pts.append(x + e)
    pts = np.array(pts).T
    f = np.zeros((3, pts.shape[1]))
    f[:, 0] = [0.3, -0.7, 0.5]
    u = oracle.stokes_direct_sum(pts, f, np.arange(1, 7))[0]
    div = sum((u[k, 2 * k] - u[k, 2 * k + 1]) / (2 * h) for k in range(3))
    grad = np.abs(u[:, 0::2] - u[:, 1::2]).max() / (2 * h)
    assert abs(div) <= 1e-6 * grad


def test_stokeslet_reciprocity():
    """S is symmetric in (x, y) and in (i, j): f_B . u_A(x_B) = f_A . u_B(x_A)."""
    rng = np.random.default_rng(7)
    pts = rng.uniform(-0.5, 0.5, (3, 2))
    fa, fb = rng.normal(size=3), rng.normal(size=3)
    f = np.zeros((2, 3, 2))
    f[0, :, 0] = fa
    f[1, :, 1] = fb
    u = oracle.stokes_direct_sum(pts, f)
    assert abs(fb @ u[0, :, 1] - fa @ u[1, :, 0]) <= 1e-14 * np.linalg.norm(fa) * np.linalg.norm(fb) * 1e2


@pytest.fixture(scope="module")
def sphere_case():
    pts = W.fibonacci_sphere(12288)
    f = np.random.default_rng(1).uniform(-1.0, 1.0, (2, 3, pts.shape[1]))
    return pts, f, oracle.stokes_direct_sum(pts, f)


def test_ifgf_stokes_matches_direct_sum(sphere_case):
    pts, f, exact = sphere_case
    plan = oracle.Plan(pts, 0.0)
    u = plan.apply_stokes(f)
    assert oracle.rel_l2(u, exact) < 3e-4
    for s in range(2):
        for c in range(3):
            assert oracle.rel_l2(u[s, c], exact[s, c]) < 4e-4


def test_ifgf_stokes_converges_with_order(sphere_case):
    """Spectral convergence in the interpolation orders: the analytic factor is smooth in (s, theta, phi)."""
    pts, f, exact = sphere_case
    e3 = oracle.rel_l2(oracle.Plan(pts, 0.0).apply_stokes(f), exact)
    e5 = oracle.rel_l2(oracle.Plan(pts, 0.0, orders=(5, 7, 7)).apply_stokes(f), exact)
    assert e5 < 1e-5 and e5 < e3 / 20


def test_ifgf_stokes_field_linearity(sphere_case):
    """Fields are independent: applying the fields one at a time gives the same velocities."""
    pts, f, _ = sphere_case
    plan = oracle.Plan(pts, 0.0)
    both = plan.apply_stokes(f)
    one = plan.apply_stokes(f[1])
    assert np.array_equal(both[1], one[0])


def test_ifgf_stokes_needs_laplace_plan():
    pts = W.fibonacci_sphere(2048)
    plan = oracle.Plan(pts, 2.0 * np.pi)
    with pytest.raises(oracle.OracleError):
        plan.apply_stokes(np.ones((3, 2048)))

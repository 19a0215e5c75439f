"""Pins of the elasticity oracle (E1 direct sum, E2 IFGF apply) against the equations it solves.

Kelvin's solution K_ij = ((3 - 4 nu) delta_ij/r + r_i r_j/r^3)/(16 pi mu (1 - nu)) is the
displacement of an infinite isotropic solid under a unit point force (the elasticity equations
are among the kernels Sec. 2 names for Eq. (1)). It must satisfy the Navier equations
mu Lap u + (lambda + mu) grad div u = 0 away from the force (this fixes the ratio of the two
terms for each nu), balance the applied force through the traction on any sphere around it
(this fixes the normalisation), and reduce to the Stokeslet over mu at nu = 1/2.
"""
import numpy as np
import pytest

import ifgf_inputs as W
import oracle

MU = 1.7
FORCE = np.array([0.3, -0.7, 0.5])
SOURCE = np.array([0.1, 0.2, -0.1])


def _single_source(targets, mu, nu):
    """Displacements at `targets` (3, M) of FORCE applied at SOURCE (the targets carry no force)."""
    pts = np.concatenate([SOURCE[:, None], targets], axis=1)
    f = np.zeros((3, pts.shape[1]))
    f[:, 0] = FORCE
    return oracle.elastic_direct_sum(pts, f, mu, nu, np.arange(1, pts.shape[1]))[0]


@pytest.mark.parametrize("nu", [0.0, 0.3, 0.45])
def test_kelvin_solution_satisfies_navier(nu):
    x = np.array([0.5, -0.25, 0.3])
    h = 1e-3
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    u = _single_source(np.array([x + h * np.array(o) for o in offs]).T, MU, nu)
    U = {o: u[:, k] for k, o in enumerate(offs)}
    e = np.eye(3, dtype=int)

    def at(*shifts):
        return U[tuple(int(sum(s[i] for s in shifts)) for i in range(3))]

    z = (0, 0, 0)
    lap = sum((at(e[i]) - 2 * U[z] + at(-e[i])) / h**2 for i in range(3))
    graddiv = np.zeros(3)
    for i in range(3):
        for j in range(3):
            if i == j:
                graddiv[i] += (at(e[j])[j] - 2 * U[z][j] + at(-e[j])[j]) / h**2
            else:
                graddiv[i] += (at(e[i], e[j])[j] - at(e[i], -e[j])[j] - at(-e[i], e[j])[j]
                               + at(-e[i], -e[j])[j]) / (4 * h * h)
    lam = 2 * MU * nu / (1 - 2 * nu)
    residual = MU * lap + (lam + MU) * graddiv
    assert np.abs(residual).max() <= 5e-4 * np.abs(MU * lap).max()


@pytest.mark.parametrize("nu", [0.0, 0.3, 0.45])
def test_kelvin_solution_balances_the_point_force(nu):
    """The traction sigma n integrated over a sphere around the force equals minus the force."""
    R, M, h = 0.25, 4000, 1e-5
    normals = 2.0 * W.fibonacci_sphere(M)  # unit sphere, quasi-uniform
    stencil = []
    for n in normals.T:
        xs = SOURCE + R * n
        for k in range(3):
            for sg in (1.0, -1.0):
                d = np.zeros(3)
                d[k] = sg * h
                stencil.append(xs + d)
    u = _single_source(np.array(stencil).T, MU, nu)
    lam = 2 * MU * nu / (1 - 2 * nu)
    total = np.zeros(3)
    for m, n in enumerate(normals.T):
        G = np.array([(u[:, 6 * m + 2 * k] - u[:, 6 * m + 2 * k + 1]) / (2 * h) for k in range(3)])  # G[k, j] = d_k u_j
        sigma = lam * np.trace(G) * np.eye(3) + MU * (G + G.T)
        total += sigma @ n
    total *= 4 * np.pi * R * R / M
    assert np.abs(total + FORCE).max() <= 1e-4 * np.abs(FORCE).max()


def test_kelvin_solution_is_stokeslet_over_mu_at_half():
    pts = np.random.default_rng(3).uniform(-0.5, 0.5, (3, 40))
    f = np.random.default_rng(4).normal(size=(2, 3, 40))
    s = oracle.stokes_direct_sum(pts, f)
    k = oracle.elastic_direct_sum(pts, f, 2.0, 0.5)
    assert np.abs(k - 0.5 * s).max() <= 1e-14 * np.abs(s).max()


@pytest.fixture(scope="module")
def sphere_case():
    pts = W.fibonacci_sphere(12288)
    f = np.random.default_rng(1).uniform(-1.0, 1.0, (2, 3, pts.shape[1]))
    return pts, f, oracle.elastic_direct_sum(pts, f, MU, 0.3)


def test_ifgf_elastic_matches_direct_sum(sphere_case):
    pts, f, exact = sphere_case
    u = oracle.Plan(pts, 0.0).apply_elastic(f, MU, 0.3)
    assert oracle.rel_l2(u, exact) < 3e-4
    e5 = oracle.rel_l2(oracle.Plan(pts, 0.0, orders=(5, 7, 7)).apply_elastic(f, MU, 0.3), exact)
    assert e5 < 1e-5


def test_ifgf_elastic_rejects_bad_parameters():
    plan = oracle.Plan(W.fibonacci_sphere(2048), 0.0)
    f = np.ones((3, 2048))
    for mu, nu in ((0.0, 0.3), (1.0, 0.6), (1.0, -1.0)):
        with pytest.raises(oracle.OracleError):
            plan.apply_elastic(f, mu, nu)

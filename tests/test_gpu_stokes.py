"""GPU parity of the Stokes kernel (the Stokeslet at unit viscosity) through the C ABI.

The mixed path against the CPU IFGF for the Stokeslet (same tree, cones and interpolation, FP64):
relative L2 3e-5 per force field and velocity component, as for the scalar kernel.  Against the
Stokeslet direct sum: the method's accuracy at orders (3,5,5), relative L2 5e-4.  Against Stokes'
solution for a translating sphere (rigid translation inside): 1e-3.
"""
import math

import numpy as np
import pytest

import ifgf_inputs as W
import oracle

torch = pytest.importorskip("torch")
ifgf = pytest.importorskip("paper_2112_15198_gb300")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _plan(pts, nf, precision="mixed", **kw):
    kw.setdefault("max_nrhs", (3 * nf + 1) // 2)
    return ifgf.Plan(torch.from_numpy(np.ascontiguousarray(pts)).to(DEV), 0.0, precision=precision, **kw)


def _real(plan):
    return np.float32 if plan.precision == "mixed" else np.float64


def _stokes(plan, f, **kw):
    F = torch.from_numpy(np.ascontiguousarray(f, dtype=_real(plan))).to(DEV)
    U = torch.empty_like(F)
    plan.apply_stokes(F, U, **kw)
    torch.cuda.synchronize()
    return U.cpu().numpy().astype(np.float64)


def _forces(nf, n, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (nf, 3, n))


def _check_fields(got, ref, tol):
    for s in range(ref.shape[0]):
        for c in range(3):
            assert oracle.rel_l2(got[s, c], ref[s, c]) < tol, (s, c)


@pytest.mark.parametrize("nf", [1, 2, 3, 8])
def test_stokes_matches_cpu_ifgf(nf):
    """nf = 1, 2: two and three complex sets (scalar-path sweep); nf = 3, 8: five and twelve sets
    (tensor-core sweep), odd counts with a half-empty last set."""
    pts = W.fibonacci_sphere(12288)
    f = _forces(nf, pts.shape[1], 40 + nf)
    ref = oracle.Plan(pts, 0.0).apply_stokes(f)
    gp = _plan(pts, nf)
    got = _stokes(gp, f)
    assert gp.status() == 0
    _check_fields(got, ref, 3e-5)


@pytest.mark.parametrize("case", ["cloud_ragged", "spheroid", "deep"])
def test_stokes_geometries(case):
    pts, kw = {
        "cloud_ragged": (W.random_cloud(1003, seed=5), {}),
        "spheroid": (W.spheroid(20000, 0.5, 0.125, seed=9), {}),
        "deep": (W.fibonacci_sphere(3000), {"levels": 7}),
    }[case]
    f = _forces(2, pts.shape[1], 7)
    ref = oracle.Plan(pts, 0.0, levels=kw.get("levels", 0)).apply_stokes(f)
    gp = _plan(pts, 2, **kw)
    _check_fields(_stokes(gp, f), ref, 3e-5)


@pytest.mark.parametrize("stage", ["near", "leaf_level", "top_level"])
@pytest.mark.parametrize("nf", [1, 4])
def test_stokes_stages(stage, nf):
    pts = W.fibonacci_sphere(12288)
    f = _forces(nf, pts.shape[1], 3)
    op = oracle.Plan(pts, 0.0)
    near, mask = {"near": (True, 0), "leaf_level": (False, 1 << op.D), "top_level": (False, 1 << 3)}[stage]
    ref = op.apply_stokes(f, near=near, level_mask=mask)
    got = _stokes(_plan(pts, nf), f, near=near, level_mask=mask)
    _check_fields(got, ref, 3e-5)


def test_stokes_field_blocks_equal_one_sweep():
    """rhs_block = 3 complex sets: five fields run as blocks of 2, 2 and 1."""
    pts = W.fibonacci_sphere(12288)
    f = _forces(5, pts.shape[1], 11)
    full = _stokes(_plan(pts, 5), f)
    blocked = _stokes(_plan(pts, 5, rhs_block=3), f)
    for s in range(5):
        for c in range(3):
            assert oracle.rel_l2(blocked[s, c], full[s, c]) < 2e-5


def test_stokes_translating_sphere():
    """Uniform traction 3U/(2a) on a sphere of radius a = 1/2 moves it rigidly: the velocity at
    interior points (zero force there) is U."""
    n = 20000
    inside = np.array([[0.0, 0.0, 0.0], [0.1, -0.05, 0.2], [-0.2, 0.15, -0.1]]).T
    pts = np.concatenate([W.fibonacci_sphere(n), inside], axis=1)
    e = np.array([0.3, -0.5, 0.8])
    f = np.zeros((1, 3, pts.shape[1]))
    f[0, :, :n] = e[:, None] * (4.0 * math.pi * 0.25 / n)
    got = _stokes(_plan(pts, 1), f)[0][:, n:]
    U = e / 3.0
    assert np.abs(got - U[:, None]).max() < 1e-3 * np.abs(U).max()


def test_stokes_vs_direct_sum_sphere64_sampled():
    """The 1,572,864-point sphere of the bench at kappa = 0 with one force field: 200 seeded targets
    against the Stokeslet direct sum."""
    w = W.make("sphere64")
    pts = w.points()
    f = _forces(1, w.n, 64)
    tgt = W.targets(w.n, 200, 264)
    exact = oracle.stokes_direct_sum(pts, f, tgt)
    gp = _plan(pts, 1)
    got = _stokes(gp, f)[:, :, tgt]
    assert gp.status() == 0
    err = oracle.rel_l2(got, exact)
    print(f"sphere64 Stokes: rel. L2 error on {len(tgt)} targets = {err:.3e}")
    assert err < 5e-4


def test_stokes_invalid_arguments():
    pts = W.fibonacci_sphere(2048)
    F = torch.zeros((1, 3, 2048), dtype=torch.float32, device=DEV)
    U = torch.empty_like(F)
    helm = ifgf.Plan(torch.from_numpy(pts).to(DEV), 2.0, precision="mixed", max_nrhs=2)
    with pytest.raises(ifgf.IFGFError) as e:
        helm.apply_stokes(F, U)
    assert e.value.status == 1
    small = _plan(pts, 1, max_nrhs=1)  # one field needs two complex sets
    with pytest.raises(ifgf.IFGFError) as e:
        small.apply_stokes(F, U)
    assert e.value.status == 1
    ok = _plan(pts, 1)
    with pytest.raises(ifgf.IFGFError):
        ok.apply_stokes(F, F)


# ---- elasticity (Kelvin's solution), the same kernels with alpha = 3 - 4 nu ------------------

def _elastic(plan, f, mu, nu, **kw):
    F = torch.from_numpy(np.ascontiguousarray(f, dtype=_real(plan))).to(DEV)
    U = torch.empty_like(F)
    plan.apply_elastic(F, U, mu, nu, **kw)
    torch.cuda.synchronize()
    return U.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("nf", [1, 3])
@pytest.mark.parametrize("nu", [0.0, 0.3, 0.45])
def test_elastic_matches_cpu_ifgf(nf, nu):
    pts = W.fibonacci_sphere(12288)
    f = _forces(nf, pts.shape[1], 60 + nf)
    ref = oracle.Plan(pts, 0.0).apply_elastic(f, 1.7, nu)
    gp = _plan(pts, nf)
    _check_fields(_elastic(gp, f, 1.7, nu), ref, 3e-5)
    assert gp.status() == 0


def test_elastic_at_half_is_stokes_over_mu():
    """nu = 1/2: Kelvin's solution is the Stokeslet over mu; with mu = 2 every scale factor halves
    exactly, so the result is bit for bit half the Stokes result."""
    pts = W.fibonacci_sphere(12288)
    f = _forces(2, pts.shape[1], 5)
    gp = _plan(pts, 2)
    assert np.array_equal(_elastic(gp, f, 2.0, 0.5), 0.5 * _stokes(gp, f))


def test_elastic_vs_direct_sum_sampled():
    pts = W.fibonacci_sphere(393216)
    f = _forces(1, pts.shape[1], 32)
    tgt = W.targets(pts.shape[1], 100, 232)
    exact = oracle.elastic_direct_sum(pts, f, 1.7, 0.3, tgt)
    got = _elastic(_plan(pts, 1), f, 1.7, 0.3)[:, :, tgt]
    err = oracle.rel_l2(got, exact)
    print(f"sphere32 points, elasticity: rel. L2 error on {len(tgt)} targets = {err:.3e}")
    assert err < 5e-4


def test_elastic_invalid_parameters():
    pts = W.fibonacci_sphere(2048)
    F = torch.zeros((1, 3, 2048), dtype=torch.float32, device=DEV)
    U = torch.empty_like(F)
    gp = _plan(pts, 1)
    for mu, nu in ((0.0, 0.3), (-1.0, 0.3), (1.0, 0.6), (1.0, -1.0), (float("inf"), 0.3)):
        with pytest.raises(ifgf.IFGFError) as e:
            gp.apply_elastic(F, U, mu, nu)
        assert e.value.status == 1


# ---- higher orders on the mixed path -------------------------------------------------------

def test_stokes_higher_orders():
    pts = W.fibonacci_sphere(3000)
    f = _forces(1, pts.shape[1], 9)
    ref = oracle.Plan(pts, 0.0, orders=(5, 7, 7), levels=4).apply_stokes(f)
    gp = _plan(pts, 1, orders=(5, 7, 7), levels=4)
    _check_fields(_stokes(gp, f), ref, 3e-5)


# ---- FP64 path: the same algorithm as the oracle in the same precision -----------------------

@pytest.mark.parametrize("nf", [1, 2, 3])
@pytest.mark.parametrize("kernel", ["stokes", "elastic"])
def test_tensor_kernels_fp64_match_cpu_ifgf(nf, kernel):
    pts = W.fibonacci_sphere(12288)
    f = _forces(nf, pts.shape[1], 80 + nf)
    op = oracle.Plan(pts, 0.0)
    gp = _plan(pts, nf, precision="fp64")
    if kernel == "stokes":
        ref, got = op.apply_stokes(f), _stokes(gp, f)
    else:
        ref, got = op.apply_elastic(f, 1.7, 0.3), _elastic(gp, f, 1.7, 0.3)
    _check_fields(got, ref, 1e-10)


@pytest.mark.parametrize("stage", ["near", "leaf_level"])
def test_stokes_fp64_stages(stage):
    pts = W.fibonacci_sphere(12288)
    f = _forces(2, pts.shape[1], 13)
    op = oracle.Plan(pts, 0.0)
    near, mask = {"near": (True, 0), "leaf_level": (False, 1 << op.D)}[stage]
    ref = op.apply_stokes(f, near=near, level_mask=mask)
    got = _stokes(_plan(pts, 2, precision="fp64"), f, near=near, level_mask=mask)
    _check_fields(got, ref, 1e-10)


SMALL_CASES = {
    "two_points": (np.array([[0.0, 1.0], [0.0, 0.5], [0.0, -0.25]]), {}),
    "tiny": (W.random_cloud(7, seed=2), {}),
    "one_leaf_D3": (W.random_cloud(40, seed=3), {"levels": 3}),
    "planar": (np.stack([W.random_cloud(3000, seed=4)[0], W.random_cloud(3000, seed=5)[1], np.zeros(3000)]), {}),
}


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("case", list(SMALL_CASES))
def test_tensor_kernels_edge_cases(case, prec):
    """Degenerate inputs (two points, fewer points than a leaf holds, one leaf level, a flat
    cloud) for both tensor kernels in both precisions."""
    pts, kw = SMALL_CASES[case]
    f = _forces(2, pts.shape[1], 17)
    op = oracle.Plan(pts, 0.0, levels=kw.get("levels", 0))
    gp = _plan(pts, 2, precision=prec, **kw)
    tol = 3e-5 if prec == "mixed" else 1e-10
    _check_fields(_stokes(gp, f), op.apply_stokes(f), tol)
    _check_fields(_elastic(gp, f, 0.8, 0.25), op.apply_elastic(f, 0.8, 0.25), tol)
    assert gp.status() == 0

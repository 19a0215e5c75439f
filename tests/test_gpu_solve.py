"""GPU: restarted GMRES with the IFGF apply as its matrix-vector product (ifgf_gmres).

The system is (alpha I + beta A W) x = b on a sphere, A the operator of Eq. (1) and W the equal
quadrature weights area / N.  The right-hand side is made from a seeded x_true with the oracle's
FP64 direct sum (the exact operator), so the test checks the solver against the mathematics, not
against the apply it calls: the recovered x matches x_true, and its residual under the exact
operator is at the level of the IFGF approximation error.
"""
import math

import numpy as np
import pytest

import ifgf_inputs as W
import oracle

torch = pytest.importorskip("torch")
ifgf = pytest.importorskip("paper_2112_15198_gb300")

pytestmark = pytest.mark.gpu


def _system(n, wavelengths, seed):
    pts = W.fibonacci_sphere(n)
    kappa = 2 * math.pi * wavelengths
    w = np.full(n, math.pi / n)  # unit-diameter sphere: area pi
    x_true = W.densities(n, 1, seed)[0]
    alpha, beta = 0.5, 1.0
    Ax = oracle.direct_sum(pts, kappa, (w * x_true)[None, :], np.arange(n))[0]
    b = alpha * x_true + beta * Ax
    return pts, kappa, w, x_true, alpha, beta, b


@pytest.mark.parametrize("prec,tol,bound", [("mixed", 1e-5, 5e-4), ("fp64", 1e-8, 5e-4)])
def test_gmres_recovers_the_solution(prec, tol, bound):
    n = 4000
    pts, kappa, w, x_true, alpha, beta, b = _system(n, 3.0, 71)
    cdt = torch.complex64 if prec == "mixed" else torch.complex128
    rdt = torch.float32 if prec == "mixed" else torch.float64
    plan = ifgf.Plan(torch.from_numpy(pts).cuda(), kappa, precision=prec)
    bd = torch.from_numpy(b).to(cdt).cuda()
    wd = torch.from_numpy(w).to(rdt).cuda()
    x = torch.zeros_like(bd)
    its, res = plan.gmres(bd, x, alpha, beta, wd, restart=20, max_iters=100, tol=tol)
    torch.cuda.synchronize()
    assert plan.status() == 0
    print(f"{prec}: {its} iterations, relative residual {res:.2e}")
    assert res <= tol * 1.5 and its < 100
    xs = x.cpu().numpy().astype(np.complex128)
    assert oracle.rel_l2(xs, x_true) < bound
    # residual under the exact operator: the IFGF approximation error, not the solver's
    Ax = oracle.direct_sum(pts, kappa, (w * xs)[None, :], np.arange(n))[0]
    assert oracle.rel_l2(alpha * xs + beta * Ax, b) < bound
    # a second solve from the same guess gives the same bits
    x2 = torch.zeros_like(bd)
    plan.gmres(bd, x2, alpha, beta, wd, restart=20, max_iters=100, tol=tol)
    torch.cuda.synchronize()
    assert torch.equal(x, x2)


def test_gmres_restarts_and_rejects_bad_arguments():
    n = 3000
    pts, kappa, w, x_true, alpha, beta, b = _system(n, 2.0, 72)
    plan = ifgf.Plan(torch.from_numpy(pts).cuda(), kappa)
    bd = torch.from_numpy(b).to(torch.complex64).cuda()
    wd = torch.from_numpy(w).to(torch.float32).cuda()
    x = torch.zeros_like(bd)
    its, res = plan.gmres(bd, x, alpha, beta, wd, restart=3, max_iters=200, tol=1e-5)
    assert res <= 1.5e-5 and its > 3  # converged across several restarts
    assert oracle.rel_l2(x.cpu().numpy().astype(np.complex128), x_true) < 5e-4
    for kw in ({"restart": 0}, {"restart": 129}, {"max_iters": 0}, {"tol": 0.0}):
        args = {"restart": 10, "max_iters": 10, "tol": 1e-3, **kw}
        with pytest.raises(ifgf.IFGFError) as e:
            plan.gmres(bd, x, alpha, beta, wd, **args)
        assert e.value.status == 1
    with pytest.raises(ifgf.IFGFError):
        plan.gmres(bd, bd, alpha, beta, wd)

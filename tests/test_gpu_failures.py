"""Failure reporting on the GPU, driven from the host (no fault, trap or hang of the device).

- Allocation failure: the library's fault-injection hook makes the n-th device allocation fail;
  ifgf_plan_create must return IFGF_ERR_OOM and give back every byte it took (device memory
  returns to its level before the call once the library's cache is released).
- Cone lookup miss: one relevant cone is withheld from a level's dense cone table, so the apply's
  lookups of it miss; the kernels must substitute zeros and record IFGF_ERR_INTERNAL in the
  plan's status word, which the host reads, and the plan and the device stay usable.
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


def _free_after_release():
    torch.cuda.synchronize()
    ifgf.release_cached_memory()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_allocation_failure_returns_oom_and_leaks_nothing(prec):
    pts = torch.from_numpy(W.fibonacci_sphere(20000)).to(DEV)
    kappa = 2 * math.pi * 6
    base = _free_after_release()
    failed = 0
    try:
        for n in (1, 2, 3, 5, 8, 13, 21, 34, 55, 89):
            ifgf.debug_fail_allocation(n)
            try:
                plan = ifgf.Plan(pts, kappa, precision=prec)
            except ifgf.IFGFError as e:
                assert e.status == 2, e
                assert "injected" in str(e)
                failed += 1
            else:
                plan.destroy()
            ifgf.debug_fail_allocation(0)
            free = _free_after_release()
            assert abs(free - base) <= (8 << 20), (n, base - free)
    finally:
        ifgf.debug_fail_allocation(0)
    assert failed >= 5
    # the library still works and gives the method's result
    dens = W.densities(20000, 1, 3)
    plan = ifgf.Plan(pts, kappa, precision=prec)
    cdt = torch.complex64 if prec == "mixed" else torch.complex128
    a = torch.from_numpy(dens).to(DEV).to(cdt)
    out = torch.empty_like(a)
    plan.apply(a, out)
    ref = oracle.Plan(W.fibonacci_sphere(20000), kappa).apply(dens)
    assert oracle.rel_l2(out.cpu().numpy().astype(np.complex128), ref) < (1e-10 if prec == "fp64" else 3e-5)
    assert plan.status() == 0


@pytest.mark.parametrize("prec,nrhs", [("mixed", 1), ("fp64", 1), ("mixed", 8)])
@pytest.mark.parametrize("where", ["leaf", "coarse"])
def test_cone_lookup_miss_is_reported(prec, nrhs, where):
    w = W.make("sphere4")
    pts = torch.from_numpy(w.points()).to(DEV)
    A = W.densities(w.n, nrhs, 9)
    cdt = torch.complex64 if prec == "mixed" else torch.complex128
    a = torch.from_numpy(A).to(DEV).to(cdt)
    good = ifgf.Plan(pts, w.kappa, precision=prec, max_nrhs=nrhs)
    bad = ifgf.Plan(pts, w.kappa, precision=prec, max_nrhs=nrhs)
    level = bad.D if where == "leaf" else 3
    ncone = bad.ncone[level]
    bad.debug_drop_cone(level, ncone // 2)
    out_good, out_bad = torch.empty_like(a), torch.empty_like(a)
    good.apply(a, out_good)
    bad.apply(a, out_bad)
    torch.cuda.synchronize()
    assert good.status() == 0
    assert bad.status() == 5  # IFGF_ERR_INTERNAL: a lookup missed
    g, b = out_good.cpu().numpy(), out_bad.cpu().numpy()
    assert np.all(np.isfinite(b))
    assert not np.array_equal(g, b)
    # the device and the other plan are unaffected
    good.apply(a, out_bad)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out_bad.cpu().numpy(), g)


def test_drop_cone_rejects_bad_arguments():
    w = W.make("sphere4")
    plan = ifgf.Plan(torch.from_numpy(w.points()).to(DEV), w.kappa)
    for level, cone in ((2, 0), (plan.D + 1, 0), (plan.D, -1), (plan.D, plan.ncone[plan.D])):
        with pytest.raises(ifgf.IFGFError) as e:
            plan.debug_drop_cone(level, cone)
        assert e.value.status == 1
    sorted_plan = ifgf.Plan(torch.from_numpy(w.points()).to(DEV), w.kappa, cone_table="sorted")
    with pytest.raises(ifgf.IFGFError) as e:
        sorted_plan.debug_drop_cone(sorted_plan.D, 0)
    assert e.value.status == 6

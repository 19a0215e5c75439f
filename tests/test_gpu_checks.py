"""The bounds-checked build (-DIFGF_CHECKS), as a stand-in for a memory checker.

In a checked build a cousin entry corrupted to a box index past the level's boxes is caught by
the interpolation's check: the apply completes, the plan's status word reports
IFGF_ERR_INTERNAL, the results stay finite, and a fresh plan is unaffected.  In the ordinary build
the corrupting hook refuses (it would lead to an out-of-bounds read).  The whole GPU suite is also
run once in the checked build (IFGF_CHECKS=1), where every plan's index lists are validated and
every cone lookup is checked.
"""
import math

import numpy as np
import pytest

import ifgf_inputs as W

torch = pytest.importorskip("torch")
ifgf = pytest.importorskip("paper_2112_15198_gb300")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_corrupt_cousin_is_reported_in_checked_builds():
    pts = torch.from_numpy(W.fibonacci_sphere(8000)).to(DEV)
    kappa = 2 * math.pi * 4
    A = torch.from_numpy(W.densities(8000, 1, 5)).to(DEV).to(torch.complex64)
    plan = ifgf.Plan(pts, kappa)
    if not ifgf.checked_build():
        with pytest.raises(ifgf.IFGFError) as e:
            plan.debug_corrupt_cousin(plan.D)
        assert e.value.status == 6
        return
    out = torch.empty_like(A)
    plan.apply(A, out)
    torch.cuda.synchronize()
    assert plan.status() == 0
    good = out.cpu().numpy()
    plan.debug_corrupt_cousin(plan.D)
    plan.apply(A, out)
    torch.cuda.synchronize()
    assert plan.status() == 5
    assert np.all(np.isfinite(out.cpu().numpy()))
    fresh = ifgf.Plan(pts, kappa)
    fresh.apply(A, out)
    torch.cuda.synchronize()
    assert fresh.status() == 0
    np.testing.assert_array_equal(out.cpu().numpy(), good)

"""GPU: batched evaluation of many uneven problems as one CUDA-graph launch sequence.

Each problem's output from the batch must equal, bit for bit, the output of its own plan applied
alone (same kernels on the same data), and match the direct sum of Eq. (1) on sampled targets
within the method's accuracy.
"""
import numpy as np
import pytest

import ifgf_inputs as W
import oracle

torch = pytest.importorskip("torch")
ifgf = pytest.importorskip("paper_2112_15198_gb300")

pytestmark = pytest.mark.gpu


def _setup(problems):
    plans, dens, outs, host = [], [], [], []
    for w in problems:
        pts = w.points()
        d = w.densities()
        plans.append(ifgf.Plan(torch.from_numpy(pts).cuda(), w.kappa))
        dens.append(torch.from_numpy(d).to(torch.complex64).cuda())
        outs.append(torch.empty_like(dens[-1]))
        host.append((pts, d))
    return plans, dens, outs, host


def test_small_batch_equals_single_plans_and_replays():
    problems = W.batch_problems(count=6, seed=17)
    plans, dens, outs, host = _setup(problems)
    batch = ifgf.Batch(plans)
    for _ in range(2):  # capture, then replay
        for o in outs:
            o.zero_()
        batch.apply(dens, outs)
        torch.cuda.synchronize()
        for p, d, o in zip(plans, dens, outs):
            single = torch.empty_like(d)
            p.apply(d, single)
            torch.cuda.synchronize()
            assert torch.equal(single, o)
    # new output buffers: a new capture, same results
    outs2 = [torch.empty_like(d) for d in dens]
    batch.apply(dens, outs2)
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)
    for w, (pts, d), o in zip(problems, host, outs):
        tg = W.targets(w.n, 300, w.seed)
        exact = oracle.direct_sum(pts, w.kappa, d, tg)
        got = o.cpu().numpy().astype(np.complex128)[:, tg]
        assert oracle.rel_l2(got, exact) < 3e-4
    for p in plans:
        assert p.status() == 0
    batch.destroy()


def test_batch_rejects_bad_entries():
    problems = W.batch_problems(count=2, seed=3)
    plans, dens, outs, _ = _setup(problems)
    batch = ifgf.Batch(plans)
    with pytest.raises(ifgf.IFGFError):
        batch.apply(dens, [outs[0], dens[1]])  # aliased buffers
    with pytest.raises(ifgf.IFGFError):
        batch.apply(dens, outs, nrhs_list=[1, 2])  # above max_nrhs
    batch.destroy()


def test_batch64_uneven_workload():
    """64 spheres and (a, a, a/2) spheroids, 2-32 wavelengths, N from 6,144 to 264,192 (about
    100 points per square wavelength): one captured launch sequence; error per problem on 500
    sampled targets against the direct sum."""
    problems = W.batch_problems()
    plans, dens, outs, host = _setup(problems)
    batch = ifgf.Batch(plans)
    batch.apply(dens, outs)
    batch.apply(dens, outs)
    torch.cuda.synchronize()
    worst = 0.0
    for w, (pts, d), o in zip(problems, host, outs):
        tg = w.targets()
        exact = oracle.direct_sum(pts, w.kappa, d, tg)
        err = oracle.rel_l2(o.cpu().numpy().astype(np.complex128)[:, tg], exact)
        worst = max(worst, err)
    print(f"batch64: worst per-problem rel. L2 error on 500 targets = {worst:.3e}")
    assert worst < 5e-4
    batch.destroy()

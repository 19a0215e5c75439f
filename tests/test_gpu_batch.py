"""GPU: batched evaluation of many uneven problems as one captured launch sequence, both as work
queues over all problems (a persistent propagation kernel with bounded dependency waits) and as
each plan's apply on concurrent graph branches.

Each problem's output from the batch must equal, bit for bit, the output of its own plan applied
alone (same kernel bodies on the same data), and match the direct sum of Eq. (1) on sampled
targets within the method's accuracy.  A withheld completion makes the dependency waits run out:
the batch reports IFGF_ERR_TIMEOUT and stays usable.
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


def _singles(plans, dens):
    out = []
    for p, d in zip(plans, dens):
        single = torch.empty_like(d)
        p.apply(d, single)
        out.append(single)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_small_batch_equals_single_plans_and_replays(mode):
    problems = W.batch_problems(count=6, seed=17)
    plans, dens, outs, host = _setup(problems)
    batch = ifgf.Batch(plans)
    batch.set(ifgf.BATCH.MODE, mode)
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
    assert batch.get(ifgf.BATCH.LAST_MODE) == mode
    assert batch.get(ifgf.BATCH.STATUS) == 0
    batch.destroy()


@pytest.mark.parametrize("cpi,bps", [(4, 0), (12, 1), (64, 2), (1000, 0)])
def test_queue_splits_give_identical_results(cpi, bps):
    """Any queue split (parent cones per item) and any number of resident blocks: the same bits
    as the plans' own applies."""
    problems = W.batch_problems(count=5, seed=29)
    plans, dens, outs, _ = _setup(problems)
    ref = _singles(plans, dens)
    batch = ifgf.Batch(plans)
    batch.set(ifgf.BATCH.MODE, 1)
    batch.set(ifgf.BATCH.CONES_PER_ITEM, cpi)
    batch.set(ifgf.BATCH.BLOCKS_PER_SM, bps)
    batch.apply(dens, outs)
    torch.cuda.synchronize()
    assert batch.get(ifgf.BATCH.ITEMS) > 0
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    batch.destroy()


def test_queue_wait_limit_reports_timeout_and_recovers():
    """The first item of one problem's leaf-level propagation is never counted as complete, so the
    items of the next level wait on a counter that cannot reach its target; with the wait limit
    shrunk to 2,000 polls they give up, the batch's status word reads IFGF_ERR_TIMEOUT, and the
    kernel ends.  Without the withheld completion the next apply is exact again."""
    problems = W.batch_problems(count=4, seed=5)
    plans, dens, outs, _ = _setup(problems)
    ref = _singles(plans, dens)
    batch = ifgf.Batch(plans)
    batch.set(ifgf.BATCH.MODE, 1)
    deep = max(range(len(plans)), key=lambda i: plans[i].D)
    assert plans[deep].D >= 5
    batch.set(ifgf.BATCH.WAIT_LIMIT, 2000)
    batch.set(ifgf.BATCH.WITHHOLD, deep * 64 + plans[deep].D)
    batch.apply(dens, outs)
    torch.cuda.synchronize()
    assert batch.get(ifgf.BATCH.STATUS) == 4  # IFGF_ERR_TIMEOUT
    batch.set(ifgf.BATCH.WITHHOLD, -1)
    batch.set(ifgf.BATCH.WAIT_LIMIT, 1 << 24)
    batch.apply(dens, outs)
    torch.cuda.synchronize()
    assert batch.get(ifgf.BATCH.STATUS) == 0
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    with pytest.raises(ifgf.IFGFError):
        batch.set(ifgf.BATCH.WITHHOLD, 99 * 64 + 5)
    with pytest.raises(ifgf.IFGFError):
        batch.set(ifgf.BATCH.CONES_PER_ITEM, 2)
    batch.destroy()


def test_queue_mode_refuses_plans_it_cannot_run():
    problems = W.batch_problems(count=2, seed=3)
    plans, dens, outs, _ = _setup(problems)
    fp64 = ifgf.Plan(torch.from_numpy(problems[1].points()).cuda(), problems[1].kappa, precision="fp64")
    batch = ifgf.Batch([plans[0], fp64])
    batch.set(ifgf.BATCH.MODE, 1)
    d64 = dens[1].to(torch.complex128)
    with pytest.raises(ifgf.IFGFError) as e:
        batch.apply([dens[0], d64], [outs[0], torch.empty_like(d64)])
    assert e.value.status == 6
    batch.set(ifgf.BATCH.MODE, -1)  # falls back to the graph sequence
    batch.apply([dens[0], d64], [outs[0], torch.empty_like(d64)])
    assert batch.get(ifgf.BATCH.LAST_MODE) == 0
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
    ref = _singles(plans, dens)
    batch = ifgf.Batch(plans)
    for mode in (0, 1, 2):
        batch.set(ifgf.BATCH.MODE, mode)
        for o in outs:
            o.zero_()
        batch.apply(dens, outs)
        batch.apply(dens, outs)
        torch.cuda.synchronize()
        assert batch.get(ifgf.BATCH.LAST_MODE) == mode and batch.get(ifgf.BATCH.STATUS) == 0
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
    worst = 0.0
    for w, (pts, d), o in zip(problems, host, outs):
        tg = w.targets()
        exact = oracle.direct_sum(pts, w.kappa, d, tg)
        err = oracle.rel_l2(o.cpu().numpy().astype(np.complex128)[:, tg], exact)
        worst = max(worst, err)
    print(f"batch64: worst per-problem rel. L2 error on 500 targets = {worst:.3e}")
    assert worst < 5e-4
    batch.destroy()

"""The distributed apply (Sec. 3.2) on one GPU: every rank's shard of the same plan, the ranks
taking turns, exchanges by device copies (sharding.apply_local).

- The library's partitions and the cones and points each rank reads equal the oracle's statement
  of them (bit-exact integer work).
- The assembled result is bit-identical to the single-GPU apply: each rank runs the same kernels
  on the same coefficients for its own points and cones, and reads nothing outside what it owns or
  received (the rest of its density vector is NaN).
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

CASES = {
    "sphere": lambda: (W.fibonacci_sphere(12000), 2 * math.pi * 5),
    "oblate": lambda: (W.spheroid(15000, 0.5, 0.125, seed=21), 2 * math.pi * 8),
    "prolate": lambda: (W.spheroid(12000, 0.05, 0.5, seed=22), 2 * math.pi * 6),
    "laplace": lambda: (W.fibonacci_sphere(10000), 0.0),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("nranks", [1, 2, 5])
def test_shards_match_the_oracle_and_the_single_apply(case, nranks):
    from paper_2112_15198_gb300 import sharding

    pts, kappa = CASES[case]()
    n = pts.shape[1]
    nrhs = 2 if case == "oblate" else 1
    plan = ifgf.Plan(torch.from_numpy(pts).to(DEV), kappa, max_nrhs=nrhs)
    shards = [ifgf.Shard(plan, nranks, r, max_nrhs=nrhs) for r in range(nranks)]
    op = oracle.Plan(pts, kappa)
    assert op.D == plan.D
    start = op.get(oracle.Q_BOX_START, op.D)
    bb = oracle.partition_boxes(start, nranks)
    np.testing.assert_array_equal(shards[0].query(ifgf.SQ.POINT_BOUNDS), start[bb])
    for r, sh in enumerate(shards):
        p0, p1 = sh.query(ifgf.SQ.POINTS)
        for d in range(3, plan.D + 1):
            cb = oracle.partition_cones(op.ncone[d], nranks)
            np.testing.assert_array_equal(sh.query(ifgf.SQ.CONE_BOUNDS, d), cb)
            pcb = oracle.partition_cones(op.ncone[d - 1], nranks) if d > 3 else np.zeros(nranks + 1, np.int64)
            looked = op.shard_cones(d, (p0, p1), (int(pcb[r]), int(pcb[r + 1])))
            np.testing.assert_array_equal(sh.query(ifgf.SQ.LOOKED_INTERP, d), np.nonzero(looked & 1)[0])
            np.testing.assert_array_equal(sh.query(ifgf.SQ.LOOKED_PROP, d), np.nonzero(looked & 2)[0])
            need = np.nonzero(looked)[0]
            need = need[(need < cb[r]) | (need >= cb[r + 1])]
            np.testing.assert_array_equal(sh.query(ifgf.SQ.NEED_CONES, d), need)
        cD = oracle.partition_cones(op.ncone[op.D], nranks)
        pts_read = op.shard_points((p0, p1), (int(cD[r]), int(cD[r + 1])))
        want = np.nonzero(pts_read)[0]
        want = want[(want < p0) | (want >= p1)]
        np.testing.assert_array_equal(sh.query(ifgf.SQ.NEED_POINTS), want)
    A = torch.from_numpy(W.densities(n, nrhs, 31)).to(DEV).to(torch.complex64)
    ref = torch.empty_like(A)
    plan.apply(A, ref)
    got = torch.empty_like(A)
    sharding.apply_local(plan, shards, A, got)
    torch.cuda.synchronize()
    assert plan.status() == 0
    np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
    for sh in shards:
        sh.destroy()


def test_shard_rejects_bad_arguments():
    pts = W.fibonacci_sphere(3000)
    plan = ifgf.Plan(torch.from_numpy(pts).to(DEV), 2 * math.pi * 2)
    for nranks, rank, mx in ((0, 0, 1), (2, 2, 1), (2, -1, 1), (2, 0, 4)):
        with pytest.raises(ifgf.IFGFError) as e:
            ifgf.Shard(plan, nranks, rank, max_nrhs=mx)
        assert e.value.status == 1
    fp64 = ifgf.Plan(torch.from_numpy(pts).to(DEV), 2 * math.pi * 2, precision="fp64")
    with pytest.raises(ifgf.IFGFError) as e:
        ifgf.Shard(fp64, 2, 0)
    assert e.value.status == 6

"""The exchange of the distributed apply over torch.distributed, on CPU processes (gloo).

World sizes 2 and 4.  Every rank builds the same oracle plan, takes its intervals of points and
cones (Sec. 3.2.1) and the cones its Interpolation and Propagation read (the oracle's statement
of them), and gathers those cones from their owners with the package's ``exchange``.  The payload
of a cone is (level, cone index, owner rank, a seeded value of the cone), so each rank can check
that it received exactly the blocks it asked for, from the right owners and in its order; owners
check that every request lies in their interval.  Over all ranks the owned cones are every cone
once, and the cones sent per level stay a bounded multiple of the level's cones (Sec. 3.3).
"""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _value(level, ids):
    return np.sin(1.0 + 0.37 * ids + 1.7 * level)


def _rank_main(rank, world, port, out_dir):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import ifgf_inputs as W
    import oracle
    from paper_2112_15198_gb300 import sharding

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pts = W.spheroid(8000, 0.5, 0.2, seed=12)
        p = oracle.Plan(pts, 2 * math.pi * 4)
        start = p.get(oracle.Q_BOX_START, p.D)
        bb = oracle.partition_boxes(start, world)
        my_pts = (int(start[bb[rank]]), int(start[bb[rank + 1]]))
        sent = {}
        for d in range(p.D, 2, -1):
            cb = oracle.partition_cones(p.ncone[d], world)
            pcb = oracle.partition_cones(p.ncone[d - 1], world) if d > 3 else np.zeros(world + 1, np.int64)
            looked = p.shard_cones(d, my_pts, (int(pcb[rank]), int(pcb[rank + 1])))
            need = np.nonzero(looked)[0]
            need = need[(need < cb[rank]) | (need >= cb[rank + 1])].astype(np.int64)
            asked_of_me = []

            def pack(ids, d=d, cb=cb):
                ids_np = ids.numpy()
                asked_of_me.append(ids_np.copy())
                assert np.all((ids_np >= cb[rank]) & (ids_np < cb[rank + 1]))
                return torch.from_numpy(np.stack([np.full(ids_np.shape, d, float), ids_np.astype(float),
                                                  np.full(ids_np.shape, rank, float), _value(d, ids_np)], axis=1))

            got = sharding.exchange(need, cb, pack, 4, torch.float64, torch.device("cpu")).numpy()
            assert got.shape == (need.shape[0], 4)
            np.testing.assert_array_equal(got[:, 0], d)
            np.testing.assert_array_equal(got[:, 1], need)
            np.testing.assert_array_equal(got[:, 2], sharding.owners(need, cb))
            np.testing.assert_array_equal(got[:, 3], _value(d, need))
            sent[d] = int(sum(a.shape[0] for a in asked_of_me))
        np.save(os.path.join(out_dir, f"sent{rank}.npy"), np.array([sent[d] for d in range(3, p.D + 1)]))
        np.save(os.path.join(out_dir, f"nc{rank}.npy"), np.array([p.ncone[d] for d in range(3, p.D + 1)]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_exchange_over_gloo(world, tmp_path):
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    sent = sum(np.load(tmp_path / f"sent{r}.npy") for r in range(world))
    nc = np.load(tmp_path / "nc0.npy")
    assert np.all(sent <= 4 * nc), (sent, nc)
    assert np.all(sent > 0)

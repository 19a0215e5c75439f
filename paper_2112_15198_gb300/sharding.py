"""The apply distributed over ranks (Sec. 3.2), driven from Python.

Each rank holds a Shard of the same plan: its points (an interval of leaf boxes), its cones at
every level (an interval of the cone order), and buffers for the cones of other ranks that its
Interpolation and Propagation read.  Per level d, before the rank's step, the needed level-d
cones are gathered from their owners (the data of the paper's CommunicateInterpolationData and
CommunicatePropagationData, Sec. 3.2.3); at the start, the densities of the points of other ranks
that the rank's near field and LevelDEvaluations read are gathered the same way.  All arithmetic
runs in the library's kernels; this module only moves blocks between ranks:

- ``exchange``: one all-to-all round trip of requests and data over ``torch.distributed`` (NCCL
  between GPUs, gloo between CPU processes), written once for any block payload;
- ``apply_distributed``: the apply of one rank of a ``torch.distributed`` job;
- ``apply_local``: all ranks of a job in one process, taking turns on one device, with the
  exchanges done by device copies; each rank sees only its own data and what it received.
"""
from __future__ import annotations

import numpy as np

from . import SQ, Shard

__all__ = ["owners", "exchange", "apply_distributed", "apply_local"]


def owners(ids: np.ndarray, bounds: np.ndarray) -> np.ndarray:
    """Rank owning each item of ids, for the intervals [bounds[r], bounds[r + 1])."""
    return np.searchsorted(np.asarray(bounds), np.asarray(ids), side="right") - 1


def exchange(need: np.ndarray, bounds: np.ndarray, pack, block: int, dtype, device, group=None):
    """Gather the blocks of the items `need` (ascending, owned by other ranks) from their owners.

    pack(ids) must return the calling rank's own blocks of the items ids (an int64 tensor on
    `device`) as a [len(ids), block] tensor of `dtype`.  Returns the [len(need), block] blocks in
    the order of need.  Collective: every rank of the group calls it for the same level.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    need = np.asarray(need, dtype=np.int64)
    own = owners(need, bounds)
    send_counts = np.bincount(own, minlength=world).astype(np.int64)  # requests to each owner
    sc = torch.from_numpy(send_counts).to(device)
    rc = torch.empty_like(sc)
    dist.all_to_all_single(rc, sc, group=group)
    recv_counts = rc.cpu().numpy()
    req = torch.from_numpy(need).to(device)
    asked = torch.empty(int(recv_counts.sum()), dtype=torch.int64, device=device)
    dist.all_to_all_single(asked, req, [int(c) for c in recv_counts], [int(c) for c in send_counts], group=group)
    data = pack(asked) if asked.numel() else torch.empty((0, block), dtype=dtype, device=device)
    got = torch.empty((need.shape[0], block), dtype=dtype, device=device)
    dist.all_to_all_single(got, data.reshape(-1, block), [int(c) for c in send_counts],
                           [int(c) for c in recv_counts], group=group)
    return got


def _cone_pack(shard: Shard, level: int, nrhs: int):
    import torch

    floats = shard.block_bytes(level, nrhs) // 4

    def pack(ids):
        dst = torch.empty((ids.numel(), floats), dtype=torch.float32, device=ids.device)
        shard.pack(level, nrhs, ids, dst)
        return dst

    return pack, floats


def apply_distributed(plan, shard: Shard, dens, out, group=None):
    """The rank's part of out = I(dens) in a torch.distributed job (Sec. 3.2).

    dens: [nrhs][N] complex64 on the rank's device, caller order; only the entries of the
    rank's own points and of the points it reads (IFGF_SQ_NEED_POINTS) are used.  out: same
    shape; on return it holds the results of the rank's own points (other entries undefined).
    """
    import torch

    nrhs = dens.shape[0]
    dev = dens.device
    dsort = torch.empty_like(dens)
    plan.permute(dens, dsort, to_sorted=True)
    # densities of the points of other ranks that this rank reads
    need_pts = shard.query(SQ.NEED_POINTS)
    pbounds = shard.query(SQ.POINT_BOUNDS)
    flat = torch.view_as_real(dsort).permute(1, 0, 2).reshape(plan.N, 2 * nrhs)  # [N][2 nrhs] by point
    got = exchange(need_pts, pbounds, lambda ids: flat.index_select(0, ids).contiguous(), 2 * nrhs, torch.float32,
                   dev, group)
    if need_pts.size:
        idx = torch.from_numpy(need_pts).to(dev)
        dsort_r = torch.view_as_real(dsort)
        dsort_r[:, idx, :] = got.reshape(-1, nrhs, 2).permute(1, 0, 2)
    osort = torch.zeros_like(dens)
    shard.near_leaf(dsort, osort, nrhs)
    for d in range(plan.D, 2, -1):
        pack, floats = _cone_pack(shard, d, nrhs)
        need = shard.query(SQ.NEED_CONES, d)
        blocks = exchange(need, shard.query(SQ.CONE_BOUNDS, d), pack, floats, torch.float32, dev, group)
        if need.size:
            shard.unpack(d, nrhs, blocks, 0, need.size)
        shard.level(d, osort, nrhs)
    plan.permute(osort, out, to_sorted=False)
    return out


def apply_local(plan, shards, dens, out):
    """All ranks of a job in one process, taking turns on one device (a check of the distributed
    data flow without several GPUs).  Each rank works on its own sorted density vector holding
    only its own points and the points it reads (the rest is NaN, so any other read would show in
    the results), and on its own result vector; exchanges copy packed blocks from the owners'
    buffers.  out (caller order) receives every rank's own results."""
    import torch

    nrhs = dens.shape[0]
    dsort = torch.empty_like(dens)
    plan.permute(dens, dsort, to_sorted=True)
    nan = complex(float("nan"), float("nan"))
    dloc, oloc = [], []
    for sh in shards:
        p0, p1 = sh.query(SQ.POINTS)
        d = torch.full_like(dsort, nan)
        d[:, p0:p1] = dsort[:, p0:p1]
        need_pts = sh.query(SQ.NEED_POINTS)
        if need_pts.size:
            idx = torch.from_numpy(need_pts).to(dens.device)
            d[:, idx] = dsort[:, idx]
        dloc.append(d)
        oloc.append(torch.full_like(dsort, nan))
    for sh, d, o in zip(shards, dloc, oloc):
        sh.near_leaf(d, o, nrhs)
    for lev in range(plan.D, 2, -1):
        for sh in shards:  # exchange: every rank gathers its needed level-lev cones from the owners
            need = sh.query(SQ.NEED_CONES, lev)
            if not need.size:
                continue
            bounds = shards[0].query(SQ.CONE_BOUNDS, lev)
            own = owners(need, bounds)
            first = 0
            for r in np.unique(own):
                ids = need[own == r]
                pack, _ = _cone_pack(shards[r], lev, nrhs)
                blocks = pack(torch.from_numpy(ids).to(dens.device))
                sh.unpack(lev, nrhs, blocks, first, ids.size)
                first += ids.size
        for sh, o in zip(shards, oloc):
            sh.level(lev, o, nrhs)
    osort = torch.empty_like(dsort)
    for sh, o in zip(shards, oloc):
        p0, p1 = sh.query(SQ.POINTS)
        osort[:, p0:p1] = o[:, p0:p1]
    plan.permute(osort, out, to_sorted=False)
    return out

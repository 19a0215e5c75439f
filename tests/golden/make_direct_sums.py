"""Write the stored direct-sum values of the full-size workloads (test infrastructure).

For each named workload this evaluates the operator of Eq. (1) pair by pair in FP64 with the
oracle's direct sum (``oracle.direct_sum``), at the workload's seeded target sample, and stores

    targets  int64 [M]        the target indices (``Workload.targets()``)
    exact    complex128 [nrhs, M]  I(x_l) at those targets
    check    float64 [4]      sums of the x, y, z coordinates and of |a| over all points, so a
                              reader can confirm that its inputs are the ones used here

in ``direct_<workload>.npz`` beside this script.  Nothing here calls the CUDA library; the
values come from the oracle alone.  Usage:

    python tests/golden/make_direct_sums.py sphere512 sphere512_laplace ...
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import ifgf_inputs as W  # noqa: E402
import oracle  # noqa: E402

# Workloads whose direct sums take minutes of CPU time at their full size.
DEFAULT = ("sphere64", "prolate128", "oblate128", "sphere512", "sphere512_laplace")


def input_check(pts: np.ndarray, dens: np.ndarray) -> np.ndarray:
    return np.array([pts[0].sum(), pts[1].sum(), pts[2].sum(), np.abs(dens).sum()], dtype=np.float64)


def path_of(name: str) -> str:
    return os.path.join(HERE, f"direct_{name}.npz")


def make(name: str) -> str:
    w = W.make(name)
    pts = w.points()
    dens = w.densities()
    tg = w.targets()
    t0 = time.perf_counter()
    exact = oracle.direct_sum(pts, w.kappa, dens, tg)
    el = time.perf_counter() - t0
    out = path_of(name)
    np.savez_compressed(out, targets=tg, exact=exact, check=input_check(pts, dens))
    print(f"{name}: N = {w.n}, nrhs = {w.nrhs}, {tg.shape[0]} targets, {el:.0f} s -> {os.path.basename(out)}",
          flush=True)
    return out


def load(name: str):
    """(targets, exact, check) of a stored workload, or None if it was not generated."""
    p = path_of(name)
    if not os.path.exists(p):
        return None
    z = np.load(p)
    return z["targets"], z["exact"], z["check"]


if __name__ == "__main__":
    for nm in (sys.argv[1:] or DEFAULT):
        make(nm)

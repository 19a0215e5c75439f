"""GPU check of the allocation-free Morton order (ifgf_morton_order_noalloc).

Callers whose device memory belongs entirely to another allocator, or who cannot afford a
cudaMalloc in their loop, get the point order from a fixed static scratch array instead of
per-call allocations.  This test calls that entry point directly through the C ABI, twice in
a row on the same buffers (the second call must not see stale scratch from the first), and
checks that its permutation and keys equal, bit for bit, those of ifgf_plan_create
(IFGF_Q_PERM / IFGF_Q_KEYS) for the same points.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import ifgf_inputs as W

torch = pytest.importorskip("torch")
ifgf = pytest.importorskip("paper_2112_15198_gb300")

pytestmark = pytest.mark.gpu

MAX_POINTS = 1 << 20


def _entry():
    lib = ifgf.load()
    fn = lib.ifgf_morton_order_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _order(fn, P, n):
    perm = torch.full((n,), -1, dtype=torch.int32, device=P.device)
    keys = torch.zeros((n,), dtype=torch.int64, device=P.device)
    stream = torch.cuda.current_stream().cuda_stream
    st = fn(P.data_ptr(), n, perm.data_ptr(), keys.data_ptr(), stream)
    assert st == 0, ifgf.load().ifgf_last_error()
    torch.cuda.synchronize()
    return perm.cpu().numpy().astype(np.int64), keys.cpu().numpy()


@pytest.mark.parametrize("case", ["sphere", "cloud", "ragged_small"])
def test_noalloc_order_matches_plan_twice(case):
    pts = {"sphere": lambda: W.fibonacci_sphere(300_000),
           "cloud": lambda: W.random_cloud(MAX_POINTS, seed=11),
           "ragged_small": lambda: W.random_cloud(4099, seed=12)}[case]()
    n = pts.shape[1]
    P = torch.from_numpy(pts).cuda()
    plan = ifgf.Plan(P, 1.0)
    want_perm = plan.query(ifgf.Q.PERM)
    want_keys = plan.query(ifgf.Q.KEYS)
    plan.destroy()
    fn = _entry()
    for _ in range(2):
        perm, keys = _order(fn, P, n)
        np.testing.assert_array_equal(perm, want_perm)
        np.testing.assert_array_equal(keys, want_keys)


def test_noalloc_rejects_too_many_points():
    fn = _entry()
    P = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    # the size check comes before any device work, so no buffer of that size is needed
    assert fn(P.data_ptr(), MAX_POINTS + 1, out.data_ptr(), out.data_ptr(), None) == 1
    assert b"allocation-free" in ifgf.load().ifgf_last_error()
    assert fn(P.data_ptr(), 1, out.data_ptr(), out.data_ptr(), None) == 1

"""GPU: the autotuner of kernel choices and of batched launch sequences.

- A plan's tuning times the candidate kernels on its own data, sets the fastest and writes them to
  the cache file; a second plan of the same shape takes them from the file without measuring, and
  its results still match the CPU IFGF.
- A batch's tuning picks a launch sequence and queue split; the outputs stay bit-identical to the
  plans' own applies, and the choice is cached too.
"""
import math

import pytest

import ifgf_inputs as W
import oracle

torch = pytest.importorskip("torch")
ifgf = pytest.importorskip("paper_2112_15198_gb300")

pytestmark = pytest.mark.gpu


def _cache_entries(path):
    lines = [ln for ln in path.read_text().splitlines() if ln.strip()]
    out = {}
    for ln in lines:
        key, value = ln.rsplit(" ", 1)
        out[key] = value
    return out


@pytest.mark.parametrize("nrhs", [1, 12])
def test_plan_autotune_and_cache(nrhs, tmp_path):
    pts = W.fibonacci_sphere(9000)
    kappa = 2 * math.pi * 6
    cache = tmp_path / "tune.txt"
    A = W.densities(9000, nrhs, 52)
    ref = oracle.Plan(pts, kappa).apply(A)
    P = torch.from_numpy(pts).cuda()
    dens = torch.from_numpy(A).to(torch.complex64).cuda()
    first = ifgf.Plan(P, kappa, max_nrhs=nrhs)
    knob = ifgf.KNOB.PROP_MANY if nrhs >= 4 else ifgf.KNOB.PROP_FEW
    assert any(first.get_knob(knob, d) >= 0 for d in range(4, first.D + 1)), "no level with node tables"
    assert first.autotune(nrhs, cache) is False
    entries = _cache_entries(cache)
    assert entries and all(k.startswith("plan|") for k in entries)
    chosen = {d: first.get_knob(knob, d) for d in range(4, first.D + 1)}
    assert all(v in (-1, 0, 1) for v in chosen.values())
    if nrhs >= 4:
        assert first.get_knob(ifgf.KNOB.RHS_BLOCK) in (8, 16, 32)
    second = ifgf.Plan(P, kappa, max_nrhs=nrhs)
    assert second.autotune(nrhs, cache) is True
    assert {d: second.get_knob(knob, d) for d in range(4, second.D + 1)} == chosen
    out = torch.empty_like(dens)
    second.apply(dens, out)
    torch.cuda.synchronize()
    assert second.status() == 0
    got = out.cpu().numpy()
    for r in range(nrhs):
        assert oracle.rel_l2(got[r], ref[r]) < 3e-5


def test_batch_autotune_keeps_results_and_caches(tmp_path):
    problems = W.batch_problems(count=6, seed=61)
    plans, dens, outs, refs = [], [], [], []
    for w in problems:
        p = ifgf.Plan(torch.from_numpy(w.points()).cuda(), w.kappa)
        d = torch.from_numpy(w.densities()).to(torch.complex64).cuda()
        r = torch.empty_like(d)
        p.apply(d, r)
        plans.append(p)
        dens.append(d)
        outs.append(torch.empty_like(d))
        refs.append(r)
    torch.cuda.synchronize()
    cache = tmp_path / "tune.txt"
    batch = ifgf.Batch(plans)
    assert batch.autotune(dens, outs, cache) is False
    mode = batch.get(ifgf.BATCH.MODE)
    assert mode in (0, 1, 2)
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    batch.apply(dens, outs)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    assert any(k.startswith("batch|") for k in _cache_entries(cache))
    again = ifgf.Batch(plans)
    assert again.autotune(dens, outs, cache) is True
    assert again.get(ifgf.BATCH.MODE) == mode
    assert again.get(ifgf.BATCH.CONES_PER_ITEM) == batch.get(ifgf.BATCH.CONES_PER_ITEM)
    again.destroy()
    batch.destroy()

"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances:
  - tree, interaction lists, cone lists: bit-exact (integer work);
  - FP64 path vs CPU IFGF (same algorithm, FP64, different summation order): rel. L2 1e-10;
  - mixed path vs CPU IFGF: rel. L2 3e-5 (FP32 arithmetic over D levels of interpolation);
  - either path vs the direct sum of Eq. (1): the method's accuracy, rel. L2 2e-4 at the
    default orders (the CPU IFGF itself measures ~1.1e-4 on the 4-wavelength sphere).
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
TREE_ITEMS = [
    ("PERM", 0), ("KEYS", 0),
]


def _dyadic_lattice(n=6000, seed=61):
    """Points of the 1/128 lattice of the root cube near a sphere, so that many of them lie exactly
    on box faces (the half-open rule of the root-cube reading decides their box) and on the
    theta = pi/2, phi = j pi/4 and axis directions seen from box centres (the edge rules of the
    classification decide their cone).  Two anchors at (0,0,0) and (1,1,1) fix the root cube:
    H1 = 1 + 2^-20, a = -2^-21, and lattice point m sits at a + m H1 / 128, exactly."""
    H1 = 1.0 + 2.0 ** -20
    a = -(2.0 ** -21)
    g = np.arange(129)
    i, j, k = np.meshgrid(g, g, g, indexing="ij")
    r = np.sqrt((i / 128 - 0.5) ** 2 + (j / 128 - 0.5) ** 2 + (k / 128 - 0.5) ** 2)
    shell = np.abs(r - 0.4) < 0.5 / 128
    m = np.stack([i[shell], j[shell], k[shell]])
    rng = np.random.default_rng(seed)
    m = m[:, rng.choice(m.shape[1], size=min(n, m.shape[1]), replace=False)]
    pts = a + m.astype(np.float64) * H1 / 128.0
    anchors = np.array([[0.0, 1.0], [0.0, 1.0], [0.0, 1.0]])
    return np.ascontiguousarray(np.concatenate([anchors, pts], axis=1))


def _stored(name):
    """Targets and FP64 direct-sum values of a workload, from the values the oracle wrote
    (tests/golden/make_direct_sums.py) when they match these inputs, else from the oracle now."""
    import importlib.util
    import os

    spec = importlib.util.spec_from_file_location(
        "make_direct_sums", os.path.join(os.path.dirname(__file__), "golden", "make_direct_sums.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    w = W.make(name)
    pts, dens = w.points(), w.densities()
    got = mk.load(name)
    if got is not None and np.allclose(got[2], mk.input_check(pts, dens), rtol=1e-9, atol=1e-9):
        return w, pts, dens, got[0], got[1]
    tgt = w.targets()
    return w, pts, dens, tgt, oracle.direct_sum(pts, w.kappa, dens, tgt)


def _plan(pts, kappa, **kw):
    return ifgf.Plan(torch.from_numpy(np.ascontiguousarray(pts)).to(DEV), kappa, **kw)


def _apply(plan, dens, prec, **kw):
    cdt = torch.complex64 if prec == "mixed" else torch.complex128
    a = torch.from_numpy(np.atleast_2d(dens).astype(np.complex128)).to(DEV).to(cdt)
    out = torch.empty_like(a)
    plan.apply(a, out, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def assert_same_tree(gp, op):
    """Every integer list of the GPU plan equals the oracle's, bit for bit."""
    assert gp.D == op.D
    Qg, Qo = ifgf.Q, oracle
    np.testing.assert_array_equal(gp.query(Qg.PERM), op.get(Qo.Q_PERM))
    np.testing.assert_array_equal(gp.query(Qg.KEYS), op.get(Qo.Q_KEYS))
    for d in range(1, gp.D + 1):
        keys = gp.query(Qg.BOX_KEYS, d)
        coords = gp.query(Qg.BOX_COORDS, d).reshape(-1, 3)
        for b in range(0, len(keys), max(1, len(keys) // 64)):  # coordinates decode the keys
            k = [0, 0, 0]
            for bit in range(21):
                for ax in range(3):
                    k[ax] |= ((int(keys[b]) >> (3 * bit + ax)) & 1) << bit
            assert tuple(coords[b]) == tuple(k)
        for qg, qo in ((Qg.BOX_KEYS, Qo.Q_BOX_KEYS), (Qg.BOX_START, Qo.Q_BOX_START), (Qg.BOX_PARENT, Qo.Q_BOX_PARENT)):
            np.testing.assert_array_equal(gp.query(qg, d), op.get(qo, d), err_msg=f"item {qg} level {d}")
        if d < gp.D:
            np.testing.assert_array_equal(gp.query(Qg.CHILD_START, d), op.get(Qo.Q_CHILD_START, d))
        if d >= 2:
            np.testing.assert_array_equal(gp.query(Qg.NBR_COUNT, d), op.get(Qo.Q_NBR_COUNT, d))
            np.testing.assert_array_equal(gp.query(Qg.NBR_LIST, d), op.get(Qo.Q_NBR_LIST, d))
        if d >= 3:
            np.testing.assert_array_equal(gp.query(Qg.COUS_COUNT, d), op.get(Qo.Q_COUS_COUNT, d))
            np.testing.assert_array_equal(gp.query(Qg.COUS_LIST, d), op.get(Qo.Q_COUS_LIST, d))
            assert gp.grid(d) == op.grid(d)
            np.testing.assert_array_equal(gp.query(Qg.CONE_BOX, d), op.get(Qo.Q_CONE_BOX, d), err_msg=f"cones {d}")
            np.testing.assert_array_equal(gp.query(Qg.CONE_GAMMA, d), op.get(Qo.Q_CONE_GAMMA, d), err_msg=f"cones {d}")


CASES = {
    "sphere4": lambda: (W.make("sphere4").points(), W.make("sphere4").kappa, {}),
    "cloud_ragged": lambda: (W.random_cloud(1003, seed=5), 2 * math.pi * 3, {}),
    "spheroid": lambda: (W.spheroid(20000, 0.5, 0.125, seed=9), 2 * math.pi * 6, {}),
    "tiny": lambda: (W.random_cloud(7, seed=2), 1.0, {}),
    "two_points": lambda: (np.array([[0.0, 1.0], [0.0, 0.5], [0.0, -0.25]]), 3.0, {}),
    "one_leaf_D3": lambda: (W.random_cloud(40, seed=3), 2.0, {"levels": 3}),
    "planar": lambda: (np.stack([W.random_cloud(3000, seed=4)[0], W.random_cloud(3000, seed=5)[1],
                                 np.zeros(3000)]), 2 * math.pi * 4, {}),
    "deep": lambda: (W.fibonacci_sphere(3000), 2 * math.pi * 2, {"levels": 7}),
    "laplace": lambda: (W.fibonacci_sphere(12000), 0.0, {}),
    # (a, a, a/2) spheroid of the uneven batch: its leaf neighbour lists once came out truncated
    "batch_spheroid": lambda: (W.batch_problems(count=6, seed=17)[1].points(),
                               W.batch_problems(count=6, seed=17)[1].kappa, {}),
    # the paper's third body, the prolate spheroid (a, a, 10a): long, thin, many levels
    "prolate": lambda: (W.spheroid(20000, 0.05, 0.5, seed=51), 2 * math.pi * 8, {}),
    # points exactly on box faces and on cone edges seen from box centres
    "dyadic_lattice": lambda: (_dyadic_lattice(), 2 * math.pi * 4, {}),
}


@pytest.mark.parametrize("case", list(CASES))
def test_tree_and_cones_bit_exact(case):
    pts, kappa, kw = CASES[case]()
    op = oracle.Plan(pts, kappa, **kw)
    gp = _plan(pts, kappa, **kw)
    assert_same_tree(gp, op)


@pytest.mark.parametrize("case", ["sphere4", "cloud_ragged", "spheroid", "two_points", "one_leaf_D3", "planar",
                                  "deep", "laplace", "batch_spheroid", "prolate", "dyadic_lattice"])
def test_fp64_matches_cpu_ifgf(case):
    pts, kappa, kw = CASES[case]()
    n = pts.shape[1]
    dens = W.densities(n, 1, 17)
    ref = oracle.Plan(pts, kappa, **kw).apply(dens)
    gp = _plan(pts, kappa, precision="fp64", **kw)
    got = _apply(gp, dens, "fp64")
    assert gp.status() == 0
    assert oracle.rel_l2(got, ref) < 1e-10


@pytest.mark.parametrize("case", ["sphere4", "cloud_ragged", "spheroid", "two_points", "one_leaf_D3", "planar",
                                  "deep", "laplace", "batch_spheroid", "prolate", "dyadic_lattice"])
def test_mixed_matches_cpu_ifgf(case):
    pts, kappa, kw = CASES[case]()
    n = pts.shape[1]
    dens = W.densities(n, 1, 17)
    ref = oracle.Plan(pts, kappa, **kw).apply(dens)
    gp = _plan(pts, kappa, precision="mixed", **kw)
    got = _apply(gp, dens, "mixed")
    assert gp.status() == 0
    assert oracle.rel_l2(got, ref) < 3e-5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("stage", ["near", "leaf_level", "top_level"])
def test_stages_match_cpu_ifgf(prec, stage):
    w = W.make("sphere4")
    pts, kappa = w.points(), w.kappa
    dens = w.densities()
    op = oracle.Plan(pts, kappa)
    gp = _plan(pts, kappa, precision=prec)
    near, mask = {"near": (True, 0), "leaf_level": (False, 1 << op.D), "top_level": (False, 1 << 3)}[stage]
    ref = op.apply(dens, near=near, level_mask=mask)
    got = _apply(gp, dens, prec, near=near, level_mask=mask)
    tol = 1e-10 if prec == "fp64" else 3e-5
    assert oracle.rel_l2(got, ref) < tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_accuracy_vs_direct_sum_sphere4(prec):
    w = W.make("sphere4")
    pts, kappa = w.points(), w.kappa
    dens = w.densities()
    exact = oracle.direct_sum(pts, kappa, dens)
    got = _apply(_plan(pts, kappa, precision=prec), dens, prec)
    assert oracle.rel_l2(got, exact) < 2e-4


def test_multiple_rhs_and_determinism():
    pts = W.fibonacci_sphere(6000)
    kappa = 2 * math.pi * 3
    A = W.densities(6000, 3, 5)
    for prec in ("fp64", "mixed"):
        gp = _plan(pts, kappa, precision=prec, max_nrhs=3)
        all3 = _apply(gp, A, prec)
        again = _apply(gp, A, prec)
        assert np.array_equal(all3, again)  # no float atomics: bitwise reproducible
        for r in range(3):
            one = _apply(gp, A[r], prec)[0]
            assert np.array_equal(one, all3[r])


def test_higher_orders_fp64():
    pts = W.fibonacci_sphere(3000)
    kappa = 2 * math.pi * 2
    dens = W.densities(3000, 1, 3)
    op = oracle.Plan(pts, kappa, orders=(5, 7, 7), levels=4)
    gp = _plan(pts, kappa, precision="fp64", orders=(5, 7, 7), levels=4)
    assert_same_tree(gp, op)
    assert oracle.rel_l2(_apply(gp, dens, "fp64"), op.apply(dens)) < 1e-10
    exact = oracle.direct_sum(pts, kappa, dens)
    assert oracle.rel_l2(_apply(gp, dens, "fp64"), exact) < 2e-6


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("kappa", [0.0, 2 * math.pi * 3])
def test_sphere_single_layer_closed_form(prec, kappa):
    """The single layer of unit density over a Fibonacci sphere of radius a = 1/2 at points that
    carry no density, against its closed form: a e^{i kappa a} sin(kappa r)/(kappa r) inside,
    a sin(kappa a) e^{i kappa r}/(kappa r) outside (a and a^2/r at kappa = 0)."""
    n, a = 20000, 0.5
    probes = np.array([[0.0, 0.0, 0.0], [0.1, -0.05, 0.2], [-0.2, 0.15, -0.1],
                       [0.9, 0.3, -0.4], [-0.2, 0.6, 0.5]]).T
    pts = np.concatenate([W.fibonacci_sphere(n), probes], axis=1)
    dens = np.zeros((1, pts.shape[1]), dtype=np.complex128)
    dens[0, :n] = 4 * math.pi * a * a / n
    got = _apply(_plan(pts, kappa, precision=prec), dens, prec)[0, n:]
    for t in range(probes.shape[1]):
        r = float(np.linalg.norm(probes[:, t]))
        if kappa == 0.0:
            want = a if r < a else a * a / r
        elif r < a:
            want = a * np.exp(1j * kappa * a) * (np.sin(kappa * r) / (kappa * r) if r > 0 else 1.0)
        else:
            want = a * np.sin(kappa * a) * np.exp(1j * kappa * r) / (kappa * r)
        assert abs(got[t] - want) <= 1e-4 * max(abs(want), 0.1), (t, got[t], want)


def test_higher_orders_mixed():
    """Orders (5,7,7) on the mixed path (generic propagation, leaf in passes of 8 cones)."""
    pts = W.fibonacci_sphere(3000)
    kappa = 2 * math.pi * 2
    dens = W.densities(3000, 2, 8)
    op = oracle.Plan(pts, kappa, orders=(5, 7, 7), levels=4)
    gp = _plan(pts, kappa, precision="mixed", orders=(5, 7, 7), levels=4, max_nrhs=2)
    got = _apply(gp, dens, "mixed")
    ref = op.apply(dens)
    for r in range(2):
        assert oracle.rel_l2(got[r], ref[r]) < 3e-5


@pytest.mark.parametrize("what", ["duplicate", "nan", "n1", "kappa", "levels", "orders", "host_points",
                                  "unbuilt_orders"])
def test_invalid_input_rejected(what):
    pts = W.random_cloud(100, seed=1)
    kw = {}
    kappa = 1.0
    if what == "duplicate":
        pts[:, 10] = pts[:, 50]
    elif what == "nan":
        pts[1, 3] = np.nan
    elif what == "n1":
        pts = pts[:, :1]
    elif what == "kappa":
        kappa = -1.0
    elif what == "levels":
        kw["levels"] = 22
    elif what == "orders":
        kw["orders"] = (0, 4, 4)
    elif what == "unbuilt_orders":
        kw["orders"] = (7, 9, 9)  # valid orders without kernels in this build
    with pytest.raises(ifgf.IFGFError) as e:
        if what == "host_points":
            ifgf.Plan(torch.from_numpy(pts), kappa)
        else:
            _plan(pts, kappa, **kw)
    assert e.value.status == (6 if what == "unbuilt_orders" else 1)


def test_nrhs_limit():
    pts = W.random_cloud(500, seed=1)
    gp = _plan(pts, 1.0, max_nrhs=2)
    a = torch.zeros((3, 500), dtype=torch.complex64, device=DEV)
    with pytest.raises(ifgf.IFGFError):
        gp.apply(a, torch.empty_like(a))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_full_size_sphere64_sampled(prec):
    """The 64-wavelength, 1,572,864-point sphere: error on its 2,000 seeded targets against the
    direct sum (measured 1.4e-4 in both precisions; bound about twice that), and the tree/cone
    lists against the oracle's."""
    w, pts, dens, tgt, exact = _stored("sphere64")
    gp = _plan(pts, w.kappa, precision=prec)
    got = _apply(gp, dens, prec)[:, tgt]
    assert gp.status() == 0
    err = oracle.rel_l2(got, exact)
    print(f"sphere64 {prec}: rel. L2 error on {len(tgt)} targets = {err:.3e}")
    assert err < 3e-4
    if prec == "mixed":
        op = oracle.Plan(pts, w.kappa)
        assert_same_tree(gp, op)


def test_full_size_prolate128_sampled():
    """The prolate spheroid (a, a, 10a) of the paper's tests, 128 wavelengths long, N = 6,291,456:
    error on 2,000 seeded targets against the direct sum, and the tree/cone lists against the
    oracle's."""
    w, pts, dens, tgt, exact = _stored("prolate128")
    gp = _plan(pts, w.kappa, precision="mixed")
    got = _apply(gp, dens, "mixed")[:, tgt]
    assert gp.status() == 0
    err = oracle.rel_l2(got, exact)
    print(f"prolate128: D = {gp.D}, rel. L2 error on {len(tgt)} targets = {err:.3e}")
    assert err < 3e-4
    assert_same_tree(gp, oracle.Plan(pts, w.kappa))


@pytest.mark.parametrize("nrhs", [4, 12, 32])
@pytest.mark.parametrize("shape", ["sphere", "oblate"])
def test_many_densities_tensor_core_path(nrhs, shape):
    """nrhs >= 4 runs the tensor-core (3xTF32 mma.sync) propagation and interpolation; every
    density must match the CPU IFGF as the single-density path does, and agree with it."""
    n = 8000
    pts = W.fibonacci_sphere(n) if shape == "sphere" else W.spheroid(n, 0.5, 0.125, seed=31)
    kappa = 2 * math.pi * 5
    A = W.densities(n, nrhs, 21)
    ref = oracle.Plan(pts, kappa).apply(A)
    gp = _plan(pts, kappa, precision="mixed", max_nrhs=nrhs)
    got = _apply(gp, A, "mixed")
    assert gp.status() == 0
    for r in range(nrhs):
        assert oracle.rel_l2(got[r], ref[r]) < 3e-5, r
    single = _apply(_plan(pts, kappa, precision="mixed"), A[nrhs - 1], "mixed")[0]
    assert oracle.rel_l2(got[nrhs - 1], single) < 2e-5


@pytest.mark.parametrize("nrhs,block", [(12, -1), (32, -1), (20, 8), (6, 32)])
def test_tcgen05_products_and_density_blocks(nrhs, block):
    """The kernel choices of the many-density path: on every level whose parent level has node
    tables, the propagation as tcgen05 products with TMEM accumulators (knob PROP_MANY = 1) or as
    mma.sync tiles, with 8, 16 or 32 densities per block; every density matches the CPU IFGF, and
    the two product kernels agree to FP32 rounding."""
    n = 9000
    pts = W.spheroid(n, 0.5, 0.125, seed=33)
    kappa = 2 * math.pi * 6
    A = W.densities(n, nrhs, 23)
    ref = oracle.Plan(pts, kappa).apply(A)
    gp = _plan(pts, kappa, precision="mixed", max_nrhs=nrhs)
    gp.set_knob(ifgf.KNOB.RHS_BLOCK, 0, block)
    tab = [d for d in range(4, gp.D + 1) if gp.get_knob(ifgf.KNOB.PROP_MANY, d) >= 0]
    assert tab, "no level with node tables"
    mma = _apply(gp, A, "mixed")
    for d in tab:
        gp.set_knob(ifgf.KNOB.PROP_MANY, d, 1)
        assert gp.get_knob(ifgf.KNOB.PROP_MANY, d) == 1
    tc = _apply(gp, A, "mixed")
    assert gp.status() == 0
    for r in range(nrhs):
        assert oracle.rel_l2(tc[r], ref[r]) < 3e-5, r
        assert oracle.rel_l2(mma[r], ref[r]) < 3e-5, r
        assert oracle.rel_l2(tc[r], mma[r]) < 1e-5, r


def test_per_cone_kernel_on_table_levels():
    """With one density, the per-cone propagation (knob PROP_FEW = 1) on the node-table levels
    gives the values of the node-table warp kernel up to FP32 rounding, and both match the CPU
    IFGF."""
    pts = W.fibonacci_sphere(9000)
    kappa = 2 * math.pi * 6
    A = W.densities(9000, 1, 5)
    ref = oracle.Plan(pts, kappa).apply(A)
    gp = _plan(pts, kappa, precision="mixed")
    warp = _apply(gp, A, "mixed")
    tab = [d for d in range(4, gp.D + 1) if gp.get_knob(ifgf.KNOB.PROP_FEW, d) >= 0]
    assert tab
    for d in tab:
        gp.set_knob(ifgf.KNOB.PROP_FEW, d, 1)
    cone = _apply(gp, A, "mixed")
    assert gp.status() == 0
    assert oracle.rel_l2(warp[0], ref[0]) < 3e-5
    assert oracle.rel_l2(cone[0], ref[0]) < 3e-5
    assert oracle.rel_l2(cone[0], warp[0]) < 1e-5
    with pytest.raises(ifgf.IFGFError):
        gp.set_knob(ifgf.KNOB.PROP_FEW, 3, 1)
    with pytest.raises(ifgf.IFGFError):
        gp.set_knob(ifgf.KNOB.RHS_BLOCK, 0, 12)


@pytest.mark.parametrize("stage", ["near", "leaf_level", "top_level"])
def test_many_densities_stages(stage):
    w = W.make("sphere4")
    pts, kappa = w.points(), w.kappa
    A = W.densities(w.n, 8, 3)
    op = oracle.Plan(pts, kappa)
    gp = _plan(pts, kappa, precision="mixed", max_nrhs=8)
    near, mask = {"near": (True, 0), "leaf_level": (False, 1 << op.D), "top_level": (False, 1 << 3)}[stage]
    ref = op.apply(A, near=near, level_mask=mask)
    got = _apply(gp, A, "mixed", near=near, level_mask=mask)
    for r in range(8):
        assert oracle.rel_l2(got[r], ref[r]) < 3e-5


def test_density_blocks_equal_one_sweep():
    """With rhs_block smaller than nrhs, the levels are swept once per block of densities; the
    result is the same as one sweep over all densities."""
    pts = W.fibonacci_sphere(5000)
    kappa = 2 * math.pi * 4
    A = W.densities(5000, 10, 8)
    full = _apply(_plan(pts, kappa, precision="mixed", max_nrhs=10), A, "mixed")
    blocked = _apply(_plan(pts, kappa, precision="mixed", max_nrhs=10, rhs_block=4), A, "mixed")
    for r in range(10):
        assert oracle.rel_l2(blocked[r], full[r]) < 2e-5


@pytest.mark.parametrize("prec,nrhs", [("mixed", 1), ("fp64", 1), ("mixed", 8)])
def test_sorted_cone_lists_equal_dense_tables(prec, nrhs):
    """The sorted per-box cone lists (used where a dense n_d x C_d table would be too large) give
    the same cones as the dense table and, since every lookup returns the same cone, bit-identical
    results; the cones also equal the oracle's."""
    pts = W.spheroid(12_000, 0.5, 0.25, seed=41)
    kappa = 2 * math.pi * 6
    A = W.densities(pts.shape[1], nrhs, 42)
    dense = _plan(pts, kappa, precision=prec, cone_table="dense", max_nrhs=nrhs)
    srt = _plan(pts, kappa, precision=prec, cone_table="sorted", max_nrhs=nrhs)
    for d in range(3, dense.D + 1):
        np.testing.assert_array_equal(dense.query(ifgf.Q.CONE_BOX, d), srt.query(ifgf.Q.CONE_BOX, d))
        np.testing.assert_array_equal(dense.query(ifgf.Q.CONE_GAMMA, d), srt.query(ifgf.Q.CONE_GAMMA, d))
    a = _apply(dense, A, prec)
    b = _apply(srt, A, prec)
    assert dense.status() == 0 and srt.status() == 0
    np.testing.assert_array_equal(a, b)
    if prec == "mixed" and nrhs == 1:
        assert_same_tree(srt, oracle.Plan(pts, kappa))


@pytest.mark.parametrize("name,bound", [("sphere512", 1.5e-4), ("sphere512_laplace", 2e-4)])
def test_full_size_sphere512_sampled(name, bound):
    """The 512-wavelength, 25,165,824-point sphere (sorted cone lists at the coarse levels) and its
    Laplace repeat: error on 2,000 seeded targets against the direct sum, bounded at about twice
    the measured error."""
    w, pts, dens, tgt, exact = _stored(name)
    gp = _plan(pts, w.kappa, precision="mixed")
    got = _apply(gp, dens, "mixed")[:, tgt]
    assert gp.status() == 0
    err = oracle.rel_l2(got, exact)
    print(f"{name}: D = {gp.D}, rel. L2 error on {len(tgt)} targets = {err:.3e}")
    assert err < bound


def test_full_size_oblate128_many_densities():
    """The 128-wavelength (a, a, a/4) spheroid, N = 6,291,456, 32 densities on the tensor-core path:
    error of every density on 2,000 seeded targets against the direct sum."""
    w, pts, dens, tgt, exact = _stored("oblate128")
    gp = _plan(pts, w.kappa, precision="mixed", max_nrhs=w.nrhs)
    got = _apply(gp, dens, "mixed")[:, tgt]
    assert gp.status() == 0
    errs = [oracle.rel_l2(got[r], exact[r]) for r in range(w.nrhs)]
    print(f"oblate128 x 32: rel. L2 error on {len(tgt)} targets: mean {np.mean(errs):.3e}, worst {max(errs):.3e}")
    assert max(errs) < 3e-4


def test_cached_memory_is_reused_and_released():
    """Plan memory comes from the library's pool: a second plan of the same problem reuses the
    cached memory, results are unchanged, and the cache can be returned to the device."""
    pts = W.fibonacci_sphere(6000)
    kappa = 2 * math.pi * 4
    A = W.densities(6000, 1, 3)
    first = _plan(pts, kappa)
    a = _apply(first, A, "mixed")
    first.destroy()
    second = _plan(pts, kappa)
    b = _apply(second, A, "mixed")
    second.destroy()
    np.testing.assert_array_equal(a, b)
    ifgf.release_cached_memory()
    third = _plan(pts, kappa)
    np.testing.assert_array_equal(_apply(third, A, "mixed"), a)


@pytest.mark.parametrize("prec,nrhs,cone_table", [("mixed", 1, "auto"), ("fp64", 1, "auto"), ("mixed", 8, "auto"),
                                                   ("mixed", 1, "sorted")])
def test_sliced_propagation_equals_one_slice(prec, nrhs, cone_table):
    """Propagation in many slices (consecutive levels at opposite ends of one coefficient buffer,
    slices ordered so no child coefficient is overwritten before it is read) gives bit-identical
    results to one slice per level."""
    pts = W.spheroid(15_000, 0.5, 0.2, seed=44)
    kappa = 2 * math.pi * 7
    A = W.densities(pts.shape[1], nrhs, 45)
    one = _plan(pts, kappa, precision=prec, max_nrhs=nrhs, prop_slices=1, cone_table=cone_table)
    many = _plan(pts, kappa, precision=prec, max_nrhs=nrhs, prop_slices=37, cone_table=cone_table)
    a = _apply(one, A, prec)
    b = _apply(many, A, prec)
    assert one.status() == 0 and many.status() == 0
    np.testing.assert_array_equal(a, b)
    ref = oracle.Plan(pts, kappa).apply(A)
    assert oracle.rel_l2(b, ref) < (1e-10 if prec == "fp64" else 3e-5)

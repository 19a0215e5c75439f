"""Host-side pieces of bench.py: the algorithmic work model, the workloads and the traffic record.

The per-unit flop counts are the ones the roofline divides by; for one value set they must equal
the per-evaluation figures stated with the kernels (interpolant evaluation 415, interpolation to
a target 425, coefficient generation 52 per node, Helmholtz leaf pair 35 and near pair 22).
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _work():
    return {"prop": {3: 10, 4: 20}, "interp": {3: 5, 4: 6}, "near_pairs": 100, "leaf_pairs": 200}


def test_one_set_matches_the_per_unit_figures():
    ncone = {3: 4, 4: 5}
    f = bench.algorithmic_flops(_work(), ncone, 75, 1)
    assert f["prop"] + f["prop_gen"] == 30 * 415 + 4 * 75 * 52
    assert f["interp"] == 11 * 425
    assert f["leaf"] == 200 * 35 + 5 * 75 * 52
    assert f["near"] == 100 * 22


def test_sets_repeat_only_the_per_set_work():
    ncone = {3: 4, 4: 5}
    one = bench.algorithmic_flops(_work(), ncone, 75, 1)
    four = bench.algorithmic_flops(_work(), ncone, 75, 4)
    assert four["prop"] - one["prop"] == 3 * (30 * 390 + 4 * 75 * 52)
    assert four["prop_gen"] == one["prop_gen"] == 0
    assert four["interp"] - one["interp"] == 3 * 11 * 390
    assert four["near"] - one["near"] == 3 * 100 * 8


def test_stokes_pairs_count_per_force_field():
    ncone = {3: 4, 4: 5}
    f1 = bench.algorithmic_flops(_work(), ncone, 75, 2, stokes_fields=1)
    f3 = bench.algorithmic_flops(_work(), ncone, 75, 5, stokes_fields=3)
    assert f1["near"] == 100 * (9 + 18)
    assert f3["near"] == 100 * (9 + 3 * 18)
    assert f1["leaf"] == 200 * (15 + 18) + 5 * 75 * 52 * 2


def test_workloads_and_sets():
    class A:
        workload, nrhs, kernel, precision = "sphere64", 0, "helmholtz", "mixed"

    w = bench.workload_of(A)
    assert w.n == 1_572_864 and w.nrhs == 1 and w.kappa > 0
    assert bench.Problem(A, w).sets == 1
    A.kernel, A.nrhs = "stokes", 3
    w = bench.workload_of(A)
    assert w.kappa == 0.0 and w.nrhs == 3
    assert bench.Problem(A, w).sets == 5  # ceil(9 / 2) complex sets
    cfg = bench.config_of(w, "mixed", 8, "stokes")
    assert "Stokeslet" in cfg["workload"] and cfg["nrhs"] == 3


def test_traffic_record_is_keyed_by_the_kernel_source():
    csrc = os.path.join(ROOT, "paper_2112_15198_gb300", "csrc")
    apply_src = open(os.path.join(csrc, "apply.cu")).read()
    header = open(os.path.join(csrc, "ifgf_internal.cuh")).read()
    bodies = open(os.path.join(csrc, "bodies_f32.cuh")).read()
    sha = bench.kernel_source_sha("k_prop_warp_f32", apply_src, header, bodies)
    assert sha == bench.kernel_source_sha("k_prop_warp_f32", apply_src + "\n// trailing\n", header, bodies)
    assert sha != bench.kernel_source_sha("k_prop_warp_f32", apply_src, header, bodies.replace("kSegLen / 2", "kSegLen/2"))
    assert sha != bench.kernel_source_sha("k_prop_warp_f32", apply_src.replace("kWarpCones + (threadIdx.x >> 5)", "kWarpCones+(threadIdx.x >> 5)"),
                                          header, bodies)
    recorded = [ln for ln in open(os.path.join(ROOT, "profiles", "traffic.txt")) if ln.startswith("kernel=")]
    assert recorded and all("source_sha=" in ln for ln in recorded)


def test_propagation_split_by_node_tables():
    """Evaluations out of level d, and the coefficients of the level-(d-1) cones they produce,
    belong to the node-table kernel when level d-1 has tables, else to the generic one."""
    work = {"prop": {3: 0, 4: 20, 5: 7}, "interp": {3: 5, 4: 6, 5: 1}, "near_pairs": 1, "leaf_pairs": 2,
            "tabled": {3: False, 4: False, 5: True}}
    ncone = {3: 4, 4: 5, 5: 6}
    f = bench.algorithmic_flops(work, ncone, 75, 1)
    assert f["prop_gen"] == 20 * 415 + 4 * 75 * 52
    assert f["prop"] == 7 * 415 + 5 * 75 * 52


def test_roofline_reports_every_kernel_kind():
    kt = {"perm": (1.0, 4), "near": (2.0, 2), "leaf": (3.0, 2), "prop": (10.0, 6), "interp": (4.0, 12),
          "plan": (5.0, 2), "prop_gen": (8.0, 4)}
    flops = {"near": 2e9, "leaf": 3e9, "prop": 1e10, "prop_gen": 4e9, "interp": 5e9}
    peaks = {"fp32_ffma_tflops": 78.0, "fp32x2_ffma2_tflops": 80.0, "fp64_tflops": 1.2, "mufu_sin_gops": 5e3,
             "tf32_mma_sync_tflops": 300.0, "sms": 152.0}
    r = bench.roofline_of(kt, flops, 2, "mixed", False, False, peaks)
    assert set(r["per_kernel"]) == {"near", "leaf", "prop", "prop_gen", "interp"}
    assert r["kernel"] == "k_prop_warp_f32" and r["per_kernel"]["prop_gen"]["kernel"] == "k_prop_f32"
    # 1e10 flops per step x 2 steps in 10 ms
    assert abs(r["achieved"] - 2.0) < 1e-12 and abs(r["frac"] - 2.0 / 80.0) < 1e-12
    m = bench.roofline_of(kt, flops, 2, "mixed", False, True, peaks)
    assert m["bound"] == "tensor" and abs(m["peak"] - 100.0) < 1e-12

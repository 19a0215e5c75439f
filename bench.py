"""Benchmark of the GB300 IFGF operator apply (one JSON line on rank 0).

A step is one pass of the whole hot path over one synthetic input: the plan (Morton
octree, interaction lists, relevant cones) and the apply (near field, leaf evaluation,
propagation, interpolation, permutations), i.e. ifgf_plan_create + ifgf_apply +
ifgf_plan_destroy on device-resident inputs.  The default workload is the largest
single-GPU problem: the 512-wavelength Fibonacci sphere with N = 25,165,824 points and one
complex density vector, mixed precision, orders (3,5,5).  Metric: IFGF matvecs expressed as
N*nrhs points per second.  Beside it the line reports the apply alone, the same step through
host buffers (e2e), the plain FP64 GPU IFGF and the kappa = 0 (Laplace) repeat on the same
points, the relative error of each against the FP64 direct sum at 2,000 seeded targets
(stored values written by tests/golden/make_direct_sums.py from the oracle), and the
achieved fraction of its roofline for every hot kernel.

Multi-GPU: the method is run as independent replicas (one full problem per rank, no
collective); value = points of all ranks / max step time over ranks ("weak" scaling).

--impl reference times the oracle (the FP64 direct sum of Eq. (1), C/OpenMP) on the
host cores, on a bounded sample of the same workload's targets.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ifgf_inputs as W  # noqa: E402

METRIC = "IFGF matvecs/sec (N*nrhs pts/s) at stated rel. error vs FP64 direct sum"
UNIT = "pts/s"
L2_FLUSH_BYTES = 256 << 20

# Algorithmic FP32 flops per unit of work (counted from the arithmetic of the method's
# steps, independent of how the kernels schedule it), split into the part shared by all value
# sets of an apply and the part repeated for each (complex) set:
#   interpolant evaluation at one point, orders (3,5,5): Chebyshev recurrences 2*(1+3+3) = 14,
#   local coordinates 6, squared distance 5 (shared: 25); per set the separable contraction
#   4*(75+15+3) = 372 and the factor/ratio multiply-accumulate 18 (390)  -> 415 for one set
FLOPS_EVAL_SHARED, FLOPS_EVAL_SET = 25, 390
#   centred factor of an interpolation to a target (shared): 10
FLOPS_CENTRED = 10
#   coefficient generation per node and set: 4*(5+5+3) = 52
FLOPS_DCT_NODE = 52
#   Helmholtz leaf pair: analytic factor of one source at one node 27, accumulate 8 per set
FLOPS_LEAF_SHARED, FLOPS_LEAF_SET = 27, 8
#   Helmholtz near-field pair: distance and Green function 14, accumulate 8 per set
FLOPS_NEAR_SHARED, FLOPS_NEAR_SET = 14, 8
#   Stokeslet pairs (per force field: r.f 5, scaling 1, three two-FMA accumulations 12):
#   near field separation 3 + squared distance 5 + 1/r^2 1; leaf w 9 + |w|^2 5 + 1/|w|^2 1
FLOPS_STOKES_FIELD = 18
FLOPS_STOKES_NEAR_SHARED, FLOPS_STOKES_LEAF_SHARED = 9, 15
# FP32 ALU peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.070 GHz (maximum SM clock).
SMS, LANES, MAX_SM_GHZ = 152, 128, 2.070
PEAK_FP32_TFLOPS = SMS * LANES * 2 * MAX_SM_GHZ / 1e3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere512")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--study", default="", choices=["", "linearithmic", "batch"],
                    help="linearithmic: plan + apply time and error against N log N for four sizes of the "
                         "sphere and the prolate spheroid (fixed sampling density); batch: the 64-problem uneven batch (spheres and spheroids of 2-32 wavelengths), one batched "
                         "apply per step: sequential applies, the per-plan graph sequence and the queue "
                         "sequence, and the autotuner's choice")
    ap.add_argument("--batch-mode", type=int, default=-2, choices=[-2, 0, 1, 2],
                    help="--study batch: -2 the autotuner's choice (default), else the batch sequence to time alone "
                         "(0 graph, 1 queue with the persistent propagation, 2 queue with branch propagation)")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the FP64 GPU and kappa = 0 records beside the line")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--nrhs", type=int, default=0,
                    help="densities (force fields for --kernel stokes) per apply; 0: the workload's own count")
    ap.add_argument("--kernel", default="helmholtz", choices=["helmholtz", "stokes", "elastic"],
                    help="stokes: the Stokeslet on the workload's points (kappa = 0, real force fields); "
                         "elastic: Kelvin's solution with mu = 1, nu = 0.3 on the same inputs")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_flops(work: dict, ncone: dict, P: int, sets: int, stokes_fields: int = 0) -> dict:
    """FP32 flops of one apply on `sets` complex value sets (for the Stokeslet, its
    ceil(3 nf / 2) sets of nf force fields), per kernel kind: "prop" is the propagation out of
    levels whose parent level has node tables, "prop_gen" the rest (each with the coefficient
    generation of the parent cones it writes)."""
    top = max(ncone)
    tabled = work.get("tabled", {})
    prop = {"prop": 0, "prop_gen": 0}
    for d, evals in work["prop"].items():
        kind = "prop" if tabled.get(d, True) else "prop_gen"
        prop[kind] += evals * (FLOPS_EVAL_SHARED + FLOPS_EVAL_SET * sets)
        if d - 1 in ncone and d > min(ncone):
            prop[kind] += ncone[d - 1] * P * FLOPS_DCT_NODE * sets
    interp = sum(work["interp"].values()) * (FLOPS_EVAL_SHARED + FLOPS_CENTRED + FLOPS_EVAL_SET * sets)
    dct_leaf = ncone[top] * P * FLOPS_DCT_NODE * sets
    if stokes_fields:
        leaf = work["leaf_pairs"] * (FLOPS_STOKES_LEAF_SHARED + FLOPS_STOKES_FIELD * stokes_fields) + dct_leaf
        near = work["near_pairs"] * (FLOPS_STOKES_NEAR_SHARED + FLOPS_STOKES_FIELD * stokes_fields)
    else:
        leaf = work["leaf_pairs"] * (FLOPS_LEAF_SHARED + FLOPS_LEAF_SET * sets) + dct_leaf
        near = work["near_pairs"] * (FLOPS_NEAR_SHARED + FLOPS_NEAR_SET * sets)
    return {"prop": prop["prop"], "prop_gen": prop["prop_gen"], "interp": interp, "leaf": leaf, "near": near}


def kernel_source_sha(kernel: str, apply_src: str, header_src: str, bodies_src: str = "") -> str:
    """sha256 prefix of a kernel's definition in apply.cu together with the device bodies it
    runs (bodies_f32.cuh) and the device helpers of ifgf_internal.cuh (everything after its
    "Device helpers" banner)."""
    at = apply_src.index(f"\n{kernel}(")
    start = apply_src.rindex("\n\n", 0, at)
    end = apply_src.index("\n}\n", at) + 3
    dev = header_src[header_src.index("// Device helpers"):]
    return hashlib.sha256((apply_src[start:end] + bodies_src + dev).encode()).hexdigest()[:16]


def traffic_record(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on
    the current kernel source (its sha256 is recorded beside the figure)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    csrc = os.path.join(ROOT, "paper_2112_15198_gb300", "csrc")
    try:
        sha = kernel_source_sha(kernel, open(os.path.join(csrc, "apply.cu")).read(),
                                open(os.path.join(csrc, "ifgf_internal.cuh")).read(),
                                open(os.path.join(csrc, "bodies_f32.cuh")).read())
    except ValueError:
        return None
    for ln in open(path):
        f = dict(kv.split("=", 1) for kv in ln.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("source_sha") == sha and "bytes_per_launch" in f:
            return float(f["bytes_per_launch"])
    return None


def max_over_ranks(x: float, pg, device) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's); x itself when
    there is one rank."""
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ws: int, n: int, nrhs: int, ms_step: float) -> float:
    """Points of all ranks per second: every rank solves its own full problem (replicas)."""
    return ws * n * nrhs / (ms_step / 1e3)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle

    oracle.build()
    w = workload_of(args)
    prob = Problem(args, w)
    pts = w.points()
    dens = prob.host_inputs()
    threads = oracle.max_threads()
    # bounded sample: enough targets for ~3 s of CPU work per step
    probe = W.targets(w.n, 64, 999)
    prob.exact(oracle, pts, dens, probe[:4])  # thread pool start-up, untimed
    t0 = time.perf_counter()
    prob.exact(oracle, pts, dens, probe)
    per_target = (time.perf_counter() - t0) / len(probe)
    m = int(max(16, min(w.n, 3.0 / per_target)))
    tg = W.targets(w.n, m, w.seed + 200)
    for _ in range(args.warmup):
        prob.exact(oracle, pts, dens, tg[:16])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        prob.exact(oracle, pts, dens, tg)
        times.append(time.perf_counter() - t0)
    value = m * w.nrhs / statistics.median(times)
    sample = f"direct sum of {prob.what()} at {m} of the {w.n} targets per step (FP64, OpenMP)"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_of(w, args.precision, None, prob.kind),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def workload_of(args):
    w = W.make(args.workload)
    if args.nrhs > 0:
        w = dataclasses.replace(w, nrhs=args.nrhs)
    if args.kernel != "helmholtz":
        w = dataclasses.replace(w, wavelengths=0.0)
    return w


ELASTIC_MU, ELASTIC_NU = 1.0, 0.3


class Problem:
    """The apply of one kernel on a workload: inputs, plan and oracle reference."""

    def __init__(self, args, w):
        self.w, self.kind, self.precision = w, args.kernel, args.precision
        self.stokes = args.kernel != "helmholtz"  # a Green tensor acting on real force fields
        # complex value sets carried through the levels
        self.sets = (3 * w.nrhs + 1) // 2 if self.stokes else w.nrhs

    def host_inputs(self):
        if self.stokes:
            rng = np.random.default_rng(self.w.seed + 100)
            return rng.uniform(-1.0, 1.0, (self.w.nrhs, 3, self.w.n))
        return self.w.densities()

    def torch_inputs(self, host):
        import torch

        if self.stokes:
            return torch.from_numpy(host.astype(np.float32))
        cdt = torch.complex64 if self.precision == "mixed" else torch.complex128
        return torch.from_numpy(host).to(cdt)

    def plan(self, ifgf, P):
        return ifgf.Plan(P, self.w.kappa, precision=self.precision, max_nrhs=self.sets)

    def apply(self, plan, A, out):
        if self.kind == "stokes":
            plan.apply_stokes(A, out)
        elif self.kind == "elastic":
            plan.apply_elastic(A, out, ELASTIC_MU, ELASTIC_NU)
        else:
            plan.apply(A, out)

    def exact(self, oracle, pts, host, tgt):
        if self.kind == "stokes":
            return oracle.stokes_direct_sum(pts, host, tgt)
        if self.kind == "elastic":
            return oracle.elastic_direct_sum(pts, host, ELASTIC_MU, ELASTIC_NU, tgt)
        return oracle.direct_sum(pts, self.w.kappa, host, tgt)

    def what(self):
        return {"stokes": "the Stokeslet sum", "elastic": "the Kelvin-solution sum"}.get(self.kind, "Eq. (1)")


def config_of(w, precision, D, kind="helmholtz"):
    body = ("Fibonacci sphere, unit diameter" if w.geometry == "sphere"
            else f"spheroid with semi-axes ({w.axes[0]:g}, {w.axes[0]:g}, {w.axes[1]:g})")
    if kind != "helmholtz":
        green = ("Stokeslet (unit viscosity)" if kind == "stokes"
                 else f"Kelvin's solution (mu = {ELASTIC_MU:g}, nu = {ELASTIC_NU:g})")
        what = (f"{w.name} points: {body}, {green}, N = {w.n}, nrhs = {w.nrhs} force fields "
                f"iid U[-1,1]^3")
    else:
        what = (f"{w.name}: {body}, {w.wavelengths:g} wavelengths (kappa = 2 pi x {w.wavelengths:g}), N = {w.n}, "
                f"nrhs = {w.nrhs}, densities iid U[-1,1]+iU[-1,1]")
    return {"workload": what,
            "N": w.n, "kappa": w.kappa, "nrhs": w.nrhs, "orders": [3, 5, 5], "precision": precision,
            "base_cones": [2, 4, 8], "tau": 0.5, "leaf_target": 64, "levels": D,
            "step": "ifgf_plan_create + ifgf_apply + ifgf_plan_destroy (device-resident inputs)",
            "l2": "flushed between timed steps (256 MiB write)"}


def stored_exact(w, pts, host):
    """(targets, exact values) of the FP64 direct sum stored for workload w by
    tests/golden/make_direct_sums.py, if present and computed on these very inputs."""
    path = os.path.join(ROOT, "tests", "golden", f"direct_{w.name}.npz")
    if not os.path.exists(path):
        return None
    z = np.load(path)
    check = np.array([pts[0].sum(), pts[1].sum(), pts[2].sum(), np.abs(host).sum()])
    if z["exact"].shape[0] != host.shape[0] or not np.allclose(z["check"], check, rtol=1e-9, atol=1e-9):
        return None
    return z["targets"], z["exact"]


def rel_l2(approx, exact) -> float:
    """Relative L2 error over sampled targets (the paper's error estimator)."""
    return float(np.sqrt(np.sum(np.abs(approx - exact) ** 2) / np.sum(np.abs(exact) ** 2)))


def timed_steps(torch, stream, flush, fn, n):
    """Device time (ms, CUDA events on `stream`) of each of n calls of fn, L2 flushed before each."""
    out = []
    for _ in range(n):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def kernel_names(precision, stokes, multi):
    """Kernel behind each timing kind of the apply."""
    if precision != "mixed":
        return {"prop": "k_prop_f64", "prop_gen": "k_prop_f64", "interp": "k_interp_f64", "leaf": "k_leaf_f64",
                "near": "k_near_f64"}
    names = {"prop": "k_prop_mma_tab" if multi else "k_prop_warp_f32",
             "prop_gen": "k_prop_mma" if multi else "k_prop_f32", "interp": "k_interp_f32"}
    if stokes:
        names.update(leaf="k_leaf_stokes_f32", near="k_near_stokes_f32")
    else:
        names.update(leaf="k_leaf_f32_multi" if multi else "k_leaf_box_f32",
                     near="k_near_f32_multi" if multi else "k_near_tile_f32")
    return names


def peak_of(kind, precision, multi, peaks):
    """(bound, peak TFLOP/s, source) of a kernel kind."""
    if "error" in peaks:
        return "alu", PEAK_FP32_TFLOPS, "152 SMs x 128 FP32 lanes x 2 x 2.070 GHz (derived, not measured)"
    if precision != "mixed":
        return "alu", peaks["fp64_tflops"], "measured: FP64 DFMA probe on this GPU (of measured)"
    if multi and kind in ("prop", "prop_gen"):
        # many-density propagation runs on the TF32 tensor cores (three products per product)
        return ("tensor", peaks["tf32_mma_sync_tflops"] / 3.0,
                "measured: TF32 mma.sync probe on this GPU / 3 (3xTF32) (of measured)")
    return ("alu", max(peaks["fp32_ffma_tflops"], peaks["fp32x2_ffma2_tflops"]),
            "measured: FP32 FFMA/FFMA2 probe on this GPU (of measured)")


def roofline_of(kt, flops, steps, precision, stokes, multi, peaks):
    """Achieved algorithmic TFLOP/s of every hot kernel kind over the timed steps, against its
    measured peak; the dominant kind (largest time) fills the top-level fields."""
    names = kernel_names(precision, stokes, multi)
    per = {}
    for kind, fl in flops.items():
        ms, n = kt.get(kind, (0.0, 0))
        if n == 0 or ms <= 0 or fl <= 0:
            continue
        achieved = fl * steps / (ms / 1e3) / 1e12
        bound, peak, src = peak_of(kind, precision, multi, peaks)
        per[kind] = {"kernel": names[kind], "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "ms_per_step": ms / steps, "launches_per_step": n / steps,
                     "peak_source": src}
    dom = max(per, key=lambda k: per[k]["ms_per_step"])
    d = per[dom]
    return {"bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": "TFLOP/s", "frac": d["frac"],
            "traffic": traffic_record(d["kernel"]), "kernel": d["kernel"], "peak_source": d["peak_source"],
            "per_kernel": per, "peaks_measured": peaks,
            "kernel_ms_per_step": {k: v[0] / steps for k, v in kt.items()},
            "kernel_launches_per_step": {k: v[1] / steps for k, v in kt.items()}}


def side_record(torch, ifgf, args, name, precision, P_dev, stream, flush, steps, warmup):
    """Plan + apply + destroy of another variant on the same device (the plain FP64 GPU IFGF, or
    the kappa = 0 repeat), with its error against the stored direct sum."""
    a2 = argparse.Namespace(**vars(args))
    a2.workload, a2.precision = name, precision
    w = workload_of(a2)
    prob = Problem(a2, w)
    host = prob.host_inputs()
    A = prob.torch_inputs(host).to(P_dev.device)
    out = torch.empty_like(A)

    def step():
        plan = prob.plan(ifgf, P_dev)
        prob.apply(plan, A, out)
        plan.destroy()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ms = timed_steps(torch, stream, flush, step, steps)
    rec = {"workload": name, "precision": precision, "kappa": w.kappa, "steps": steps,
           "value": w.n * w.nrhs / (statistics.mean(ms) / 1e3), "unit": UNIT, "ms_per_step": statistics.mean(ms)}
    ref = stored_exact(w, w.points(), host)
    if ref is not None:
        tg, exact = ref
        got = out.cpu().numpy().astype(np.complex128)[:, tg]
        rec["rel_err_vs_direct_sum"] = {"value": rel_l2(got, exact), "targets": int(tg.shape[0])}
    del A, out
    return rec


def run_linearithmic(args):
    """Cost against N at a fixed sampling density (the GPU counterpart of the paper's study of
    linearithmic scaling): for each body and size, plan + apply and apply alone (CUDA events, L2
    flushed, mean of the timed steps after the warm-up) and the error on 200 seeded targets."""
    import torch

    import oracle
    import paper_2112_15198_gb300 as ifgf

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rows = []
    for body in ("sphere", "prolate"):
        for w in W.linearithmic_series(body):
            pts = w.points()
            dens = w.densities()
            P = torch.from_numpy(pts).to(dev)
            A = torch.from_numpy(dens).to(dev).to(torch.complex64)
            out = torch.empty_like(A)

            def step():
                plan = ifgf.Plan(P, w.kappa)
                plan.apply(A, out)
                plan.destroy()

            for _ in range(max(1, args.warmup)):
                step()
            st = statistics.mean(timed_steps(torch, stream, flush, step, max(1, args.steps)))
            plan = ifgf.Plan(P, w.kappa)
            plan.apply(A, out)
            ap = statistics.mean(timed_steps(torch, stream, flush, lambda: plan.apply(A, out), max(1, args.steps)))
            D = plan.D
            plan.destroy()
            tg = w.targets()
            err = rel_l2(out.cpu().numpy().astype(np.complex128)[:, tg], oracle.direct_sum(pts, w.kappa, dens, tg))
            nlogn = w.n * math.log2(w.n)
            rows.append({"body": body, "N": w.n, "wavelengths": w.wavelengths, "levels": D,
                         "ms_plan_apply": st, "ms_apply": ap, "ns_apply_per_NlogN": ap * 1e6 / nlogn,
                         "ns_step_per_NlogN": st * 1e6 / nlogn, "rel_err": err, "targets": int(tg.shape[0])})
            del P, A, out
    print(json.dumps({"study": "linearithmic", "metric": "apply time / (N log2 N)", "unit": "ns",
                      "steps": args.steps, "warmup": args.warmup, "precision": "mixed", "orders": [3, 5, 5],
                      "rows": rows}), flush=True)


def run_batch(args):
    """The uneven batch (64 spheres and (a, a, a/2) spheroids, 2-32 wavelengths, N from 6,144 to
    264,192 at about 100 points per square wavelength, one density each): plans and batch built
    once outside the timed region, then per step one batched apply (CUDA events, L2 flushed,
    mean over the timed steps after the warm-up): the plans' applies one after another, the
    per-plan graph sequence, the queue sequence at the autotuner's split, and the sequence the
    autotuner chose (cached in the build folder).  Error per problem on 100 seeded targets against
    the direct sum; every problem's batched result is checked bit-identical to its own apply."""
    import torch

    import oracle
    import paper_2112_15198_gb300 as ifgf

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    probs = W.batch_problems()
    pts = [w.points() for w in probs]
    dens_h = [w.densities() for w in probs]
    P = [torch.from_numpy(x).to(dev) for x in pts]
    dens = [torch.from_numpy(d).to(dev).to(torch.complex64) for d in dens_h]
    outs = [torch.empty_like(d) for d in dens]
    ref = [torch.empty_like(d) for d in dens]
    t0 = time.perf_counter()
    plans = [ifgf.Plan(x, w.kappa) for x, w in zip(P, probs)]
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    ntot = sum(w.n for w in probs)

    def singles(o):
        for p_, d_, x_ in zip(plans, dens, o):
            p_.apply(d_, x_)

    singles(ref)
    batch = ifgf.Batch(plans)
    if args.batch_mode == -2:
        cache = os.path.join(ROOT, "paper_2112_15198_gb300", "_build", "tune_cache.txt")
        hit = batch.autotune(dens, outs, cache_path=cache)
        runs = (("sequential", None), ("graph", 0), ("queue_branches", 2), ("queue_persistent", 1))
    else:
        hit = None
        batch.set(ifgf.BATCH.MODE, args.batch_mode)
        runs = ()
    mode, cpi = batch.get(ifgf.BATCH.MODE), batch.get(ifgf.BATCH.CONES_PER_ITEM)
    bps = batch.get(ifgf.BATCH.BLOCKS_PER_SM)
    res = {}
    clocks = ClockSampler(0)
    clocks.start()
    for name, m in runs + (("chosen", mode),):
        if m is None:
            fn = lambda: singles(outs)  # noqa: E731
        else:
            batch.set(ifgf.BATCH.MODE, m)
            fn = lambda: batch.apply(dens, outs)  # noqa: E731
        for _ in range(max(3, args.warmup)):
            fn()
        ms = statistics.mean(timed_steps(torch, stream, flush, fn, max(1, args.steps)))
        torch.cuda.synchronize()
        same = all(torch.equal(o, r) for o, r in zip(outs, ref))
        res[name] = {"ms_per_step": ms, "pts_per_s": ntot / (ms * 1e-3), "bit_identical_to_own_apply": same}
    ck = clocks.stop()
    worst = 0.0
    for w, x, d, o in zip(probs, pts, dens_h, ref):
        tg = w.targets()[:100]
        worst = max(worst, rel_l2(o.cpu().numpy().astype(np.complex128)[:, tg], oracle.direct_sum(x, w.kappa, d, tg)))
    print(json.dumps({"study": "batch", "metric": "IFGF matvecs/sec (N*nrhs pts/s) at stated rel. error vs FP64 "
                      "direct sum", "unit": "pts/s", "value": res["chosen"]["pts_per_s"],
                      "ms_per_step": res["chosen"]["ms_per_step"], "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "batch64 (64 problems, 6,144-264,192 points each)", "points": ntot,
                                 "problems": len(probs), "nrhs": 1, "step": "one batched apply (plans built once)",
                                 "l2": "flushed before each step", "plans_s": plan_s,
                                 "chosen": {"mode": {0: "graph", 1: "queue, persistent propagation",
                                                     2: "queue, branch propagation"}[mode], "cones_per_item": cpi,
                                            "blocks_per_sm": bps, "from_cache": hit}},
                      "sequences": res, "worst_rel_err": worst, "targets_per_problem": 100,
                      "batch_status": batch.get(ifgf.BATCH.STATUS), "clocks": ck}), flush=True)
    batch.destroy()


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.study == "linearithmic":
        if rank == 0:
            run_linearithmic(args)
        return
    if args.study == "batch":
        if rank == 0:
            run_batch(args)
        return
    import torch

    import paper_2112_15198_gb300 as ifgf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    ifgf.load()
    w = workload_of(args)
    prob = Problem(args, w)
    pts = w.points()
    dens_np = prob.host_inputs()
    P_host = torch.from_numpy(pts).pin_memory()
    A_host = prob.torch_inputs(dens_np).pin_memory()
    P = P_host.to(dev)
    A = A_host.to(dev)
    out = torch.empty_like(A)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    side = min(args.steps, 3)  # iterations of the context legs

    def step():
        plan = prob.plan(ifgf, P)
        prob.apply(plan, A, out)
        plan.destroy()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region -------------------------------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    ifgf.timing_enable(True)
    ifgf.timing_collect()
    launches0 = ifgf.launch_count()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    total_ms = sum(timed_steps(torch, stream, flush, step, args.steps))
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    launches = ifgf.launch_count() - launches0
    kt = ifgf.timing_collect()
    ifgf.timing_enable(False)
    clk = clocks.stop()
    ms_step = max_over_ranks(total_ms / args.steps, pg, dev)
    value = whole_job_value(ws, w.n, w.nrhs, ms_step)
    result = out.cpu().numpy()

    # ---- apply-only throughput on a persistent plan (context) ------------------------
    plan = prob.plan(ifgf, P)
    prob.apply(plan, A, out)
    torch.cuda.synchronize()
    ap_ms = timed_steps(torch, stream, flush, lambda: prob.apply(plan, A, out), side)
    work = plan.work()
    ncone = dict(plan.ncone)
    D = plan.D
    status = plan.status()
    plan.destroy()

    # ---- end to end through the C ABI with host buffers ------------------------------
    out_host = torch.empty(A.shape, dtype=A.dtype).pin_memory()
    Pd = torch.empty_like(P)
    Ad = torch.empty_like(A)
    e2e_ms = []
    for it in range(1 + side):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Pd.copy_(P_host, non_blocking=True)
        Ad.copy_(A_host, non_blocking=True)
        pl = prob.plan(ifgf, Pd)
        prob.apply(pl, Ad, out)
        out_host.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        pl.destroy()
        if it >= 1:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_step = statistics.mean(e2e_ms)
    e2e_step = max_over_ranks(e2e_step, pg, dev)
    h2d = P_host.numel() * P_host.element_size() + A_host.numel() * A_host.element_size()
    d2h = out_host.numel() * out_host.element_size()
    del Pd, Ad, out_host

    # ---- the kappa = 0 repeat on the same points; the plain FP64 GPU IFGF against the mixed one --
    extra = {}
    if rank == 0 and not args.no_side and args.kernel == "helmholtz" and args.precision == "mixed":
        if w.wavelengths > 0 and f"{args.workload}_laplace" in W.WORKLOADS:
            extra["laplace"] = side_record(torch, ifgf, args, f"{args.workload}_laplace", "mixed", P, stream, flush,
                                           side, 1)
        if w.nrhs == 1:
            # The FP64 coefficients of one level of the 512-wavelength sphere (about 2.4e8 cones of
            # 75 complex128) exceed the device memory, so the two precisions are compared on the
            # largest workload where both fit, the 64-wavelength sphere, one plan + apply each.
            del P
            torch.cuda.empty_cache()
            fw = "sphere64" if w.n > 1_572_864 else args.workload
            Pf = torch.from_numpy(W.make(fw).points()).to(dev)
            extra["fp64_vs_mixed"] = {
                "fp64": side_record(torch, ifgf, args, fw, "fp64", Pf, stream, flush, 1, 1),
                "mixed": side_record(torch, ifgf, args, fw, "mixed", Pf, stream, flush, side, 1)}
            del Pf

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return

    # ---- roofline of every hot kernel ---------------------------------------------------
    flops = algorithmic_flops(work, ncone, 75, prob.sets, w.nrhs if prob.stokes else 0)
    multi = prob.sets >= 4 and args.precision == "mixed"  # the tensor-core path
    try:
        peaks = ifgf.measure_peaks()
    except Exception as exc:  # the probe library is optional for the line itself
        peaks = {"error": str(exc)}
    roofline = roofline_of(kt, flops, args.steps, args.precision, prob.stokes, multi, peaks)

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
           "config": config_of(w, args.precision, D, prob.kind),
           "e2e": {"value": whole_job_value(ws, w.n, w.nrhs, e2e_step), "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step, "steps": side},
           "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
           "apply_only": {"value": w.n * w.nrhs / (statistics.median(ap_ms) / 1e3), "unit": UNIT,
                          "ms_per_apply": statistics.median(ap_ms), "applies": side},
           "roofline": roofline, "clocks": clk, "device_status": status,
           "work_per_apply": {"near_pairs": work["near_pairs"], "leaf_pairs": work["leaf_pairs"],
                              "interp_evals": sum(work["interp"].values()), "prop_evals": sum(work["prop"].values()),
                              "cones": sum(ncone.values())}}
    res.update(extra)
    if not prob.stokes:
        ref = stored_exact(w, pts, dens_np)
        if ref is not None:
            tg, exact = ref
            res["rel_err_vs_direct_sum"] = {"value": rel_l2(result.astype(np.complex128)[:, tg], exact),
                                            "targets": int(tg.shape[0]),
                                            "source": "stored FP64 direct sum (tests/golden)"}

    if not args.no_cpu_baseline and ws == 1:
        import oracle

        oracle.build()
        threads = oracle.max_threads()
        probe = W.targets(w.n, 64, 999)
        prob.exact(oracle, pts, dens_np, probe[:4])  # thread pool start-up, untimed
        t0 = time.perf_counter()
        prob.exact(oracle, pts, dens_np, probe)
        per_target = (time.perf_counter() - t0) / len(probe)
        m = int(max(16, min(w.n, args.cpu_seconds / per_target)))
        tg = W.targets(w.n, m, w.seed + 200)
        t0 = time.perf_counter()
        exact = prob.exact(oracle, pts, dens_np, tg)
        el = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": m * w.nrhs / el, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"FP64 direct sum of {prob.what()} at {m} of the {w.n} targets ({el:.1f} s)"}
        if "rel_err_vs_direct_sum" not in res:
            got = result.astype(np.complex128 if not prob.stokes else np.float64)[..., tg]
            res["rel_err_vs_direct_sum"] = {"value": oracle.rel_l2(got, exact), "targets": m,
                                            "source": "the cpu_baseline sample"}
    print(json.dumps(res), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()

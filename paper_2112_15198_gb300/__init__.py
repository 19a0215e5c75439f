"""GB300 IFGF operator apply -- Python binding of the C ABI in ``include/ifgf.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libifgf_<arch>.so``.  There is no fallback: if the library is missing
and cannot be built, importing the binding's functions raises.

Device buffers are passed as torch CUDA tensors (or raw integer device
pointers); torch supplies device memory and streams, nothing else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["IFGFError", "Plan", "Batch", "load", "library_path", "launch_count", "timing_enable", "timing_collect", "Q", "KNOB", "BATCH",
           "debug_fail_allocation", "Shard", "SQ", "partition_boxes", "partition_cones",
           "PREC_FP64", "PREC_MIXED"]

PREC_FP64 = 0
PREC_MIXED = 1


class Q:
    """Query codes of ifgf_plan_query."""

    PERM, KEYS, BOX_KEYS, BOX_START, BOX_PARENT = 0, 1, 2, 3, 4
    NBR_COUNT, NBR_LIST, COUS_COUNT, COUS_LIST = 5, 6, 7, 8
    CONE_BOX, CONE_GAMMA, GRID, INFO, WORK, STATUS, CHILD_START, BOX_COORDS = 9, 10, 11, 12, 13, 14, 15, 16
    TABLES = 17


class BATCH:
    """Settings and states of ifgf_batch_set / ifgf_batch_get."""

    MODE, CONES_PER_ITEM, BLOCKS_PER_SM, WAIT_LIMIT, WITHHOLD, STATUS, LAST_MODE, ITEMS = range(8)


class KNOB:
    """Kernel choices of ifgf_plan_set_knob."""

    PROP_MANY, PROP_FEW, RHS_BLOCK = 0, 1, 2


STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "INTERNAL", 6: "UNSUPPORTED"}


class IFGFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("base_cones", ctypes.c_int32 * 3),
        ("leaf_target", ctypes.c_int32),
        ("max_nrhs", ctypes.c_int32),
        ("rhs_block", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("cone_table", ctypes.c_int32),
        ("prop_slices", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load (building first if needed and allowed) the CUDA library; raise if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        checks = os.environ.get("IFGF_CHECKS", "0") == "1"  # the bounds-checked build
        path = _build.build(checks=checks) if build else (_build.CHECKS_LIB if checks else _build.LIB)
        if not os.path.exists(path):
            raise RuntimeError(f"IFGF CUDA library not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.ifgf_options_default.argtypes = [ctypes.POINTER(Options)]
        lib.ifgf_options_default.restype = None
        lib.ifgf_plan_create.argtypes = [vp, i64, dbl, ctypes.POINTER(i32), i32, ctypes.POINTER(Options), vp,
                                         ctypes.POINTER(vp)]
        lib.ifgf_plan_create.restype = ctypes.c_int
        lib.ifgf_apply.argtypes = [vp, vp, i32, vp, vp]
        lib.ifgf_apply.restype = ctypes.c_int
        lib.ifgf_apply_ex.argtypes = [vp, vp, i32, vp, vp, i32, i64]
        lib.ifgf_apply_ex.restype = ctypes.c_int
        lib.ifgf_apply_stokes.argtypes = [vp, vp, i32, vp, vp]
        lib.ifgf_apply_stokes.restype = ctypes.c_int
        lib.ifgf_apply_stokes_ex.argtypes = [vp, vp, i32, vp, vp, i32, i64]
        lib.ifgf_apply_stokes_ex.restype = ctypes.c_int
        lib.ifgf_apply_elastic.argtypes = [vp, vp, i32, vp, dbl, dbl, vp]
        lib.ifgf_apply_elastic.restype = ctypes.c_int
        lib.ifgf_apply_elastic_ex.argtypes = [vp, vp, i32, vp, dbl, dbl, vp, i32, i64]
        lib.ifgf_apply_elastic_ex.restype = ctypes.c_int
        lib.ifgf_plan_destroy.argtypes = [vp]
        lib.ifgf_plan_destroy.restype = ctypes.c_int
        lib.ifgf_plan_query.argtypes = [vp, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.ifgf_plan_query.restype = ctypes.c_int
        lib.ifgf_status_string.argtypes = [ctypes.c_int]
        lib.ifgf_status_string.restype = ctypes.c_char_p
        lib.ifgf_last_error.argtypes = []
        lib.ifgf_last_error.restype = ctypes.c_char_p
        lib.ifgf_launch_count.argtypes = []
        lib.ifgf_launch_count.restype = i64
        lib.ifgf_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
        lib.ifgf_batch_create.restype = ctypes.c_int
        lib.ifgf_batch_apply.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(vp), vp]
        lib.ifgf_batch_apply.restype = ctypes.c_int
        lib.ifgf_batch_set.argtypes = [vp, i32, i64]
        lib.ifgf_batch_set.restype = ctypes.c_int
        lib.ifgf_batch_get.argtypes = [vp, i32, ctypes.POINTER(i64)]
        lib.ifgf_batch_get.restype = ctypes.c_int
        lib.ifgf_batch_autotune.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(vp),
                                            ctypes.c_char_p, vp, ctypes.POINTER(i32)]
        lib.ifgf_batch_autotune.restype = ctypes.c_int
        lib.ifgf_plan_autotune.argtypes = [vp, i32, ctypes.c_char_p, vp, ctypes.POINTER(i32)]
        lib.ifgf_plan_autotune.restype = ctypes.c_int
        lib.ifgf_batch_destroy.argtypes = [vp]
        lib.ifgf_batch_destroy.restype = ctypes.c_int
        lib.ifgf_checked_build.argtypes = []
        lib.ifgf_checked_build.restype = i32
        lib.ifgf_debug_corrupt_cousin.argtypes = [vp, i32]
        lib.ifgf_debug_corrupt_cousin.restype = ctypes.c_int
        lib.ifgf_debug_fail_allocation.argtypes = [i64]
        lib.ifgf_debug_fail_allocation.restype = None
        lib.ifgf_debug_drop_cone.argtypes = [vp, i32, i64]
        lib.ifgf_debug_drop_cone.restype = ctypes.c_int
        lib.ifgf_partition_boxes.argtypes = [ctypes.POINTER(i64), i64, i32, ctypes.POINTER(i64)]
        lib.ifgf_partition_boxes.restype = ctypes.c_int
        lib.ifgf_partition_cones.argtypes = [i64, i32, ctypes.POINTER(i64)]
        lib.ifgf_partition_cones.restype = ctypes.c_int
        lib.ifgf_shard_create.argtypes = [vp, i32, i32, i32, ctypes.POINTER(vp)]
        lib.ifgf_shard_create.restype = ctypes.c_int
        lib.ifgf_shard_query.argtypes = [vp, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.ifgf_shard_query.restype = ctypes.c_int
        lib.ifgf_shard_coefficients.argtypes = [vp, i32, i32, ctypes.POINTER(vp), ctypes.POINTER(i64)]
        lib.ifgf_shard_coefficients.restype = ctypes.c_int
        lib.ifgf_shard_pack.argtypes = [vp, i32, i32, vp, i64, vp, vp]
        lib.ifgf_shard_pack.restype = ctypes.c_int
        lib.ifgf_shard_unpack.argtypes = [vp, i32, i32, vp, i64, i64, vp]
        lib.ifgf_shard_unpack.restype = ctypes.c_int
        lib.ifgf_shard_near_leaf.argtypes = [vp, vp, i32, vp, vp]
        lib.ifgf_shard_near_leaf.restype = ctypes.c_int
        lib.ifgf_shard_level.argtypes = [vp, i32, i32, vp, vp]
        lib.ifgf_shard_level.restype = ctypes.c_int
        lib.ifgf_shard_destroy.argtypes = [vp]
        lib.ifgf_shard_destroy.restype = ctypes.c_int
        lib.ifgf_plan_set_knob.argtypes = [vp, i32, i32, i32]
        lib.ifgf_plan_set_knob.restype = ctypes.c_int
        lib.ifgf_plan_get_knob.argtypes = [vp, i32, i32, ctypes.POINTER(i32)]
        lib.ifgf_plan_get_knob.restype = ctypes.c_int
        lib.ifgf_gmres.argtypes = [vp, vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp, i32, i32, dbl, vp,
                                   ctypes.POINTER(i32), ctypes.POINTER(dbl)]
        lib.ifgf_gmres.restype = ctypes.c_int
        lib.ifgf_permute.argtypes = [vp, vp, i32, vp, i32, vp]
        lib.ifgf_permute.restype = ctypes.c_int
        lib.ifgf_timing_enable.argtypes = [i32]
        lib.ifgf_timing_enable.restype = None
        lib.ifgf_timing_collect.argtypes = [ctypes.POINTER(dbl), ctypes.POINTER(i64)]
        lib.ifgf_timing_collect.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(st: int):
    if st != 0:
        lib = load()
        raise IFGFError(st, lib.ifgf_last_error().decode(errors="replace"))


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        import torch

        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def launch_count() -> int:
    return int(load().ifgf_launch_count())


def release_cached_memory() -> None:
    """Return the device memory cached by the library's memory pools (ifgf_release_cached_memory)."""
    lib = load()
    lib.ifgf_release_cached_memory.argtypes = []
    lib.ifgf_release_cached_memory.restype = ctypes.c_int
    _check(lib.ifgf_release_cached_memory())


def checked_build() -> bool:
    """True when the loaded library is the bounds-checked build (IFGF_CHECKS=1 at load)."""
    return bool(load().ifgf_checked_build())


def debug_fail_allocation(n: int) -> None:
    """Fault injection for tests: the n-th device allocation from now on fails as out of memory
    (ifgf_debug_fail_allocation); 0 turns it off."""
    load().ifgf_debug_fail_allocation(int(n))


def partition_boxes(box_start, nranks: int) -> np.ndarray:
    """Leaf-box intervals of the ranks (ifgf_partition_boxes, Sec. 3.2.1); host only."""
    bs = np.ascontiguousarray(box_start, dtype=np.int64)
    out = np.zeros(int(nranks) + 1, dtype=np.int64)
    i64p = ctypes.POINTER(ctypes.c_int64)
    _check(load().ifgf_partition_boxes(bs.ctypes.data_as(i64p), bs.shape[0] - 1, int(nranks), out.ctypes.data_as(i64p)))
    return out


def partition_cones(nc: int, nranks: int) -> np.ndarray:
    """Cone intervals of the ranks at one level (ifgf_partition_cones, Sec. 3.2.1); host only."""
    out = np.zeros(int(nranks) + 1, dtype=np.int64)
    _check(load().ifgf_partition_cones(int(nc), int(nranks), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out


class SQ:
    """Query codes of ifgf_shard_query."""

    POINTS, BOXES, CONES, NEED_CONES, NEED_POINTS, POINT_BOUNDS, CONE_BOUNDS, LOOKED_INTERP, LOOKED_PROP = range(9)


class Shard:
    """One rank's part of a plan (ifgf_shard_create, Sec. 3.2); see sharding.py for the apply."""

    def __init__(self, plan, nranks: int, rank: int, max_nrhs: int = 1):
        lib = load()
        self._lib = lib
        self.plan = plan  # the shard borrows the plan
        self.nranks, self.rank, self.max_nrhs = int(nranks), int(rank), int(max_nrhs)
        h = ctypes.c_void_p()
        _check(lib.ifgf_shard_create(plan._h, self.nranks, self.rank, self.max_nrhs, ctypes.byref(h)))
        self._h = h

    def query(self, what: int, level: int = 0) -> np.ndarray:
        cnt = ctypes.c_int64(0)
        _check(self._lib.ifgf_shard_query(self._h, int(what), int(level), None, ctypes.byref(cnt)))
        buf = np.zeros(max(cnt.value, 1), dtype=np.int64)
        cnt2 = ctypes.c_int64(buf.shape[0])
        _check(self._lib.ifgf_shard_query(self._h, int(what), int(level),
                                          buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(cnt2)))
        return buf[: cnt.value]

    def block_bytes(self, level: int, nrhs: int) -> int:
        ptr, nb = ctypes.c_void_p(), ctypes.c_int64(0)
        _check(self._lib.ifgf_shard_coefficients(self._h, int(level), int(nrhs), ctypes.byref(ptr), ctypes.byref(nb)))
        return int(nb.value)

    def pack(self, level: int, nrhs: int, ids, dst, stream=None):
        """dst <- the rank's own blocks of the cones ids (int64 device tensor), in that order."""
        _check(self._lib.ifgf_shard_pack(self._h, int(level), int(nrhs), _ptr(ids), int(ids.numel()), _ptr(dst),
                                         _stream(stream)))

    def unpack(self, level: int, nrhs: int, src, first: int, n: int, stream=None):
        """Needed cones first .. first + n - 1 of the level <- the n blocks at src."""
        _check(self._lib.ifgf_shard_unpack(self._h, int(level), int(nrhs), _ptr(src), int(first), int(n),
                                           _stream(stream)))

    def near_leaf(self, dens_sorted, out_sorted, nrhs: int, stream=None):
        _check(self._lib.ifgf_shard_near_leaf(self._h, _ptr(dens_sorted), int(nrhs), _ptr(out_sorted),
                                              _stream(stream)))

    def level(self, level: int, out_sorted, nrhs: int, stream=None):
        _check(self._lib.ifgf_shard_level(self._h, int(level), int(nrhs), _ptr(out_sorted), _stream(stream)))

    def destroy(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _check(self._lib.ifgf_shard_destroy(h))
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def measure_peaks() -> dict:
    """Measured throughputs of the current device (separate probe library): FP32 FFMA and
    FP32x2 FFMA2 TFLOP/s, FP64 TFLOP/s, MUFU sine Gop/s, TF32 mma.sync TFLOP/s, SM count."""
    load()
    lib = ctypes.CDLL(_build.PEAKS_LIB)
    lib.ifgf_peaks_measure.argtypes = [ctypes.POINTER(ctypes.c_double)]
    lib.ifgf_peaks_measure.restype = ctypes.c_int
    out = (ctypes.c_double * 6)()
    rc = lib.ifgf_peaks_measure(out)
    if rc != 0:
        raise IFGFError(3, f"peak probes failed with CUDA error {rc}")
    keys = ("fp32_ffma_tflops", "fp32x2_ffma2_tflops", "fp64_tflops", "mufu_sin_gops", "tf32_mma_sync_tflops", "sms")
    return {k: float(v) for k, v in zip(keys, out)}


TIMING_KINDS = ("perm", "near", "leaf", "prop", "interp", "plan", "prop_gen")


def timing_enable(on: bool = True) -> None:
    """Bracket every hot-kernel launch with CUDA events on its stream (live kernel timing)."""
    load().ifgf_timing_enable(1 if on else 0)


def timing_collect() -> dict:
    """Wait for the recorded events; return {kind: (total ms, launches)} and reset."""
    ms = (ctypes.c_double * len(TIMING_KINDS))()
    cnt = (ctypes.c_int64 * len(TIMING_KINDS))()
    _check(load().ifgf_timing_collect(ms, cnt))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(TIMING_KINDS)}


class Plan:
    """An IFGF plan over N points (ifgf_plan_create); apply() evaluates Eq. (1) for densities."""

    def __init__(self, points, kappa: float, orders=(3, 5, 5), levels: int = 0, precision: str = "mixed",
                 base_cones=(2, 4, 8), tau: float = 0.5, leaf_target: int = 64, max_nrhs: int = 1, stream=None,
                 n: int | None = None, rhs_block: int = 0, cone_table: str = "auto", prop_slices: int = 0):
        lib = load()
        self._lib = lib
        opt = Options()
        lib.ifgf_options_default(ctypes.byref(opt))
        opt.precision = PREC_MIXED if precision == "mixed" else PREC_FP64
        opt.base_cones[0], opt.base_cones[1], opt.base_cones[2] = (int(v) for v in base_cones)
        opt.tau = float(tau)
        opt.leaf_target = int(leaf_target)
        opt.max_nrhs = int(max_nrhs)
        opt.rhs_block = int(rhs_block)
        opt.cone_table = {"auto": 0, "dense": 1, "sorted": 2}[cone_table]
        opt.prop_slices = int(prop_slices)
        if n is None:
            shape = tuple(points.shape)
            if len(shape) != 2 or shape[0] != 3:
                raise ValueError("points must have shape (3, N)")
            n = shape[1]
        self.N = int(n)
        self.precision = precision
        self.max_nrhs = int(max_nrhs)
        o = (ctypes.c_int32 * 3)(*(int(v) for v in orders))
        h = ctypes.c_void_p()
        _check(lib.ifgf_plan_create(_ptr(points), self.N, float(kappa), o, int(levels), ctypes.byref(opt),
                                    _stream(stream), ctypes.byref(h)))
        self._h = h
        info = self.query(Q.INFO)
        self.D = int(info[1])
        self.nbox = {d: int(info[1 + d]) for d in range(1, self.D + 1)}
        self.ncone = {d: int(info[22 + d]) for d in range(3, self.D + 1)}

    def apply(self, dens, out, nrhs: int | None = None, stream=None, near: bool = True, level_mask: int = -1):
        """out <- I(dens); dens/out are [nrhs][N] complex (complex64 for mixed, complex128 for fp64)."""
        if nrhs is None:
            nrhs = 1 if len(dens.shape) == 1 else int(dens.shape[0])
        if near and level_mask == -1:
            _check(self._lib.ifgf_apply(self._h, _ptr(dens), int(nrhs), _ptr(out), _stream(stream)))
        else:
            _check(self._lib.ifgf_apply_ex(self._h, _ptr(dens), int(nrhs), _ptr(out), _stream(stream),
                                           1 if near else 0, int(level_mask)))
        return out

    def apply_stokes(self, forces, velocity, nfield: int | None = None, stream=None, near: bool = True,
                     level_mask: int = -1):
        """velocity <- Stokeslet sums of the force fields (kappa = 0 plans); forces/velocity are
        [nfield][3][N] float32 (mixed plans) or float64 (fp64 plans) in the caller's point order."""
        if nfield is None:
            nfield = 1 if len(forces.shape) == 2 else int(forces.shape[0])
        if near and level_mask == -1:
            _check(self._lib.ifgf_apply_stokes(self._h, _ptr(forces), int(nfield), _ptr(velocity), _stream(stream)))
        else:
            _check(self._lib.ifgf_apply_stokes_ex(self._h, _ptr(forces), int(nfield), _ptr(velocity), _stream(stream),
                                                  1 if near else 0, int(level_mask)))
        return velocity

    def apply_elastic(self, forces, displacement, shear_modulus: float, poisson_ratio: float,
                      nfield: int | None = None, stream=None, near: bool = True, level_mask: int = -1):
        """displacement <- Kelvin-solution sums of the force fields (kappa = 0 plans); forces and
        displacement are [nfield][3][N] float32 (mixed) or float64 (fp64) in the caller's point order."""
        if nfield is None:
            nfield = 1 if len(forces.shape) == 2 else int(forces.shape[0])
        if near and level_mask == -1:
            _check(self._lib.ifgf_apply_elastic(self._h, _ptr(forces), int(nfield), _ptr(displacement),
                                                float(shear_modulus), float(poisson_ratio), _stream(stream)))
        else:
            _check(self._lib.ifgf_apply_elastic_ex(self._h, _ptr(forces), int(nfield), _ptr(displacement),
                                                   float(shear_modulus), float(poisson_ratio), _stream(stream),
                                                   1 if near else 0, int(level_mask)))
        return displacement

    def query(self, what: int, level: int = 0) -> np.ndarray:
        cnt = ctypes.c_int64(0)
        _check(self._lib.ifgf_plan_query(self._h, int(what), int(level), None, ctypes.byref(cnt)))
        buf = np.zeros(max(cnt.value, 1), dtype=np.int64)
        cnt2 = ctypes.c_int64(buf.shape[0])
        _check(self._lib.ifgf_plan_query(self._h, int(what), int(level),
                                         buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(cnt2)))
        return buf[: cnt.value]

    def permute(self, src, dst, to_sorted: bool, nrhs: int | None = None, stream=None):
        """dst <- src reordered between the caller's point order and the sorted order (ifgf_permute)."""
        n = int(src.shape[0]) if nrhs is None else int(nrhs)
        _check(self._lib.ifgf_permute(self._h, _ptr(src), n, _ptr(dst), 1 if to_sorted else 0, _stream(stream)))
        return dst

    def debug_corrupt_cousin(self, level: int) -> None:
        """Checked builds only: one cousin entry of `level` becomes a box index past the level's
        boxes (ifgf_debug_corrupt_cousin), for the next apply's checks to report."""
        _check(self._lib.ifgf_debug_corrupt_cousin(self._h, int(level)))

    def set_knob(self, knob: int, level: int, value: int) -> None:
        """Kernel choice of the apply (ifgf_plan_set_knob): KNOB.PROP_MANY / KNOB.PROP_FEW per level
        d of the propagation from d into d-1, KNOB.RHS_BLOCK plan-wide; -1 restores the built-in."""
        _check(self._lib.ifgf_plan_set_knob(self._h, int(knob), int(level), int(value)))

    def gmres(self, b, x, alpha=1.0, beta=1.0, weights=None, restart: int = 30, max_iters: int = 200,
              tol: float = 1e-4, stream=None):
        """Solve (alpha I + beta A W) x = b by restarted GMRES with this plan's apply as A
        (ifgf_gmres); x holds the initial guess and receives the solution.  Returns
        (iterations, final relative residual)."""
        a = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
        bt = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
        it = ctypes.c_int32(0)
        res = ctypes.c_double(0.0)
        _check(self._lib.ifgf_gmres(self._h, _ptr(b), _ptr(x), a, bt, _ptr(weights), int(restart), int(max_iters),
                                    float(tol), _stream(stream), ctypes.byref(it), ctypes.byref(res)))
        return int(it.value), float(res.value)

    def autotune(self, nrhs: int = 1, cache_path=None, stream=None) -> bool:
        """Times the kernel choices of an apply with nrhs densities and keeps the fastest
        (ifgf_plan_autotune); True if they came from the cache file."""
        hit = ctypes.c_int32(0)
        path = None if cache_path is None else os.fsencode(cache_path)
        _check(self._lib.ifgf_plan_autotune(self._h, int(nrhs), path, _stream(stream), ctypes.byref(hit)))
        return bool(hit.value)

    def get_knob(self, knob: int, level: int = 0) -> int:
        """The kernel choice in effect (ifgf_plan_get_knob)."""
        v = ctypes.c_int32(0)
        _check(self._lib.ifgf_plan_get_knob(self._h, int(knob), int(level), ctypes.byref(v)))
        return int(v.value)

    def debug_drop_cone(self, level: int, cone: int) -> None:
        """Fault injection for tests: every lookup of relevant cone `cone` of `level` misses from now
        on (ifgf_debug_drop_cone); the next apply records IFGF_ERR_INTERNAL in status()."""
        _check(self._lib.ifgf_debug_drop_cone(self._h, int(level), int(cone)))

    def status(self) -> int:
        return int(self.query(Q.STATUS)[0])

    def grid(self, level: int):
        return tuple(int(v) for v in self.query(Q.GRID, level))

    def work(self) -> dict:
        """Exact work of one apply: near pairs, leaf pairs, per-level interpolations/propagations;
        "tabled"[d] tells whether the propagation out of level d reads node tables."""
        res = {"interp": {}, "prop": {}, "tabled": {}}
        for d in range(3, self.D + 1):
            w = self.query(Q.WORK, d)
            res["near_pairs"], res["leaf_pairs"] = int(w[0]), int(w[1])
            res["interp"][d] = int(w[2])
            res["prop"][d] = int(w[3])
            res["tabled"][d] = d > 3 and int(self.query(Q.TABLES, d - 1)[0]) > 0
        return res

    def destroy(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _check(self._lib.ifgf_plan_destroy(h))
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


class Batch:
    """Many plans applied as one captured launch sequence (ifgf_batch_*): work queues over all
    problems where the plans allow it, else each plan's apply on concurrent graph branches."""

    def __init__(self, plans):
        lib = load()
        self._lib = lib
        self._plans = list(plans)  # keep the plans alive
        arr = (ctypes.c_void_p * len(self._plans))(*(p._h.value for p in self._plans))
        h = ctypes.c_void_p()
        _check(lib.ifgf_batch_create(arr, len(self._plans), ctypes.byref(h)))
        self._h = h

    def apply(self, dens_list, out_list, nrhs_list=None, stream=None):
        n = len(self._plans)
        if nrhs_list is None:
            nrhs_list = [1 if len(d.shape) == 1 else int(d.shape[0]) for d in dens_list]
        d = (ctypes.c_void_p * n)(*(_ptr(x) for x in dens_list))
        o = (ctypes.c_void_p * n)(*(_ptr(x) for x in out_list))
        r = (ctypes.c_int32 * n)(*(int(x) for x in nrhs_list))
        _check(self._lib.ifgf_batch_apply(self._h, d, r, o, _stream(stream)))
        return out_list

    def autotune(self, dens_list, out_list, cache_path=None, nrhs_list=None, stream=None) -> bool:
        """Times the batch's launch sequences and settings and keeps the fastest
        (ifgf_batch_autotune); True if the choice came from the cache file."""
        n = len(self._plans)
        if nrhs_list is None:
            nrhs_list = [1 if len(d.shape) == 1 else int(d.shape[0]) for d in dens_list]
        d = (ctypes.c_void_p * n)(*(_ptr(x) for x in dens_list))
        o = (ctypes.c_void_p * n)(*(_ptr(x) for x in out_list))
        r = (ctypes.c_int32 * n)(*(int(x) for x in nrhs_list))
        hit = ctypes.c_int32(0)
        path = None if cache_path is None else os.fsencode(cache_path)
        _check(self._lib.ifgf_batch_autotune(self._h, d, r, o, path, _stream(stream), ctypes.byref(hit)))
        return bool(hit.value)

    def set(self, what: int, value: int) -> None:
        """A setting of the batch (ifgf_batch_set), e.g. BATCH.MODE or BATCH.CONES_PER_ITEM."""
        _check(self._lib.ifgf_batch_set(self._h, int(what), int(value)))

    def get(self, what: int) -> int:
        """A setting or state of the batch (ifgf_batch_get); BATCH.STATUS synchronises."""
        v = ctypes.c_int64(0)
        _check(self._lib.ifgf_batch_get(self._h, int(what), ctypes.byref(v)))
        return int(v.value)

    def destroy(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _check(self._lib.ifgf_batch_destroy(h))
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

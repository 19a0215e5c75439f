"""IFGF oracle -- TEST INFRASTRUCTURE ONLY.

Python access (ctypes + numpy) to the plain CPU statement of the method in
``ifgf_oracle.c``.  Only the tests, ``__graft_entry__.smoke()`` and the bench's
CPU-baseline / reference legs may import this package; the product library
never does, and nothing here imports the product package.

O1  ``direct_sum``: the operator of Eq. (1) evaluated pair by pair in FP64.
O2  ``Plan``: the plain CPU IFGF (tree, cousins, relevant cones of Eq. (4),
    Algorithms 5-8) in FP64, with its integer lists exposed for bit-exact
    comparison.
S1  ``stokes_direct_sum``: Eq. (1) with the Stokeslet (Stokes Green tensor at
    unit viscosity) acting on real force vectors, pair by pair in FP64.
S2  ``Plan.apply_stokes``: the O2 IFGF for the Stokeslet on a kappa = 0 plan.
E1  ``elastic_direct_sum``: Eq. (1) with Kelvin's solution of linear elasticity
    (shear modulus mu, Poisson ratio nu), pair by pair in FP64.
E2  ``Plan.apply_elastic``: the O2 IFGF for Kelvin's solution on a kappa = 0 plan.
M1  ``partition_boxes``, ``partition_cones``, ``Plan.shard_cones``, ``Plan.shard_points``: the
    distribution of Sec. 3.2 (points by intervals of leaf boxes, cones by intervals of the cone
    order) and the data one rank reads from the others.

Parity unpinned: none of the functions here lacks a pin; see ``tests/test_oracle_*``.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ifgf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, f"liborc_{platform.machine()}.so")
_lock = threading.Lock()
_lib = None

# Default method parameters of the oracle (the GPU path states the same readings).
DEFAULT_ORDERS = (3, 5, 5)
DEFAULT_BASE_CONES = (2, 4, 8)
DEFAULT_TAU = 0.5
DEFAULT_LEAF_TARGET = 64

Q_PERM, Q_KEYS, Q_BOX_KEYS, Q_BOX_START, Q_BOX_PARENT = 0, 1, 2, 3, 4
Q_NBR_COUNT, Q_NBR_LIST, Q_COUS_COUNT, Q_COUS_LIST = 5, 6, 7, 8
Q_CONE_BOX, Q_CONE_GAMMA, Q_GRID, Q_WORK, Q_CHILD_START = 9, 10, 11, 12, 13


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE single/double precision, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=gnu11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c_i64, c_int, c_dbl, c_vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        lib.orc_direct_sum.argtypes = [c_i64, c_vp, c_vp, c_vp, c_dbl, c_int, c_vp, c_i64, c_vp, c_vp]
        lib.orc_direct_sum.restype = None
        lib.orc_plan_create.argtypes = [c_i64, c_vp, c_vp, c_vp, c_dbl, c_int, c_int, c_int, c_int, c_int,
                                        c_int, c_int, c_int, c_dbl, ctypes.POINTER(c_int)]
        lib.orc_plan_create.restype = c_vp
        lib.orc_plan_destroy.argtypes = [c_vp]
        lib.orc_plan_destroy.restype = None
        lib.orc_apply.argtypes = [c_vp, c_int, c_vp, c_vp, c_int, c_i64]
        lib.orc_apply.restype = c_int
        lib.orc_stokes_direct_sum.argtypes = [c_i64, c_vp, c_vp, c_vp, c_int, c_vp, c_i64, c_vp, c_vp]
        lib.orc_stokes_direct_sum.restype = None
        lib.orc_apply_stokes.argtypes = [c_vp, c_int, c_vp, c_vp, c_int, c_i64]
        lib.orc_apply_stokes.restype = c_int
        lib.orc_elastic_direct_sum.argtypes = [c_i64, c_vp, c_vp, c_vp, c_dbl, c_dbl, c_int, c_vp, c_i64, c_vp,
                                               c_vp]
        lib.orc_elastic_direct_sum.restype = None
        lib.orc_apply_elastic.argtypes = [c_vp, c_dbl, c_dbl, c_int, c_vp, c_vp, c_int, c_i64]
        lib.orc_apply_elastic.restype = c_int
        lib.orc_get.argtypes = [c_vp, c_int, c_int, c_vp]
        lib.orc_get.restype = c_i64
        lib.orc_info.argtypes = [c_vp, c_vp, c_vp]
        lib.orc_info.restype = None
        lib.orc_offsets.argtypes = [c_vp, c_vp]
        lib.orc_classify.argtypes = [c_vp, c_int, c_i64, c_vp, c_vp]
        lib.orc_cheb3.argtypes = [c_vp, c_vp, c_vp]
        lib.orc_cheb3_eval.argtypes = [c_vp, c_vp, c_i64, c_vp, c_vp]
        lib.orc_cheb_nodes.argtypes = [c_vp, c_vp, c_vp, c_vp]
        lib.orc_has_duplicates.argtypes = [c_vp]
        lib.orc_has_duplicates.restype = c_int
        lib.orc_shard_cones.argtypes = [c_vp, c_int, c_i64, c_i64, c_i64, c_i64, c_vp]
        lib.orc_shard_cones.restype = c_int
        lib.orc_shard_points.argtypes = [c_vp, c_i64, c_i64, c_i64, c_i64, c_vp]
        lib.orc_shard_points.restype = None
        lib.orc_set_threads.argtypes = [c_int]
        lib.orc_max_threads.restype = c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def direct_sum(points: np.ndarray, kappa: float, dens: np.ndarray, tgt=None) -> np.ndarray:
    """O1: I(x_l) = sum_{m != l} a_m exp(i kappa r)/(4 pi r) at target indices tgt (Eq. (1)).

    points (3, N) float64; dens (nrhs, N) or (N,) complex; returns (nrhs, M) complex128.
    """
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[1]
    a = np.ascontiguousarray(np.atleast_2d(dens), dtype=np.complex128)
    nrhs = a.shape[0]
    t = np.arange(n, dtype=np.int64) if tgt is None else np.ascontiguousarray(tgt, dtype=np.int64)
    out = np.zeros((nrhs, t.shape[0]), dtype=np.complex128)
    x, y, z = (np.ascontiguousarray(pts[i]) for i in range(3))
    lib.orc_direct_sum(n, _ptr(x), _ptr(y), _ptr(z), float(kappa), nrhs, _ptr(a), t.shape[0], _ptr(t), _ptr(out))
    return out


def stokes_direct_sum(points: np.ndarray, forces: np.ndarray, tgt=None) -> np.ndarray:
    """S1: u_i(x_l) = sum_{m != l} sum_j S_ij(x_l, x_m) f_j(x_m), S the Stokeslet at unit
    viscosity, S_ij = (delta_ij/r + r_i r_j/r^3)/(8 pi), at target indices tgt.

    points (3, N) float64; forces (nf, 3, N) or (3, N) real; returns (nf, 3, M) float64.
    """
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[1]
    f = np.ascontiguousarray(np.asarray(forces, dtype=np.float64).reshape(-1, 3, n))
    nf = f.shape[0]
    t = np.arange(n, dtype=np.int64) if tgt is None else np.ascontiguousarray(tgt, dtype=np.int64)
    out = np.zeros((nf, 3, t.shape[0]), dtype=np.float64)
    x, y, z = (np.ascontiguousarray(pts[i]) for i in range(3))
    lib.orc_stokes_direct_sum(n, _ptr(x), _ptr(y), _ptr(z), nf, _ptr(f), t.shape[0], _ptr(t), _ptr(out))
    return out


def elastic_direct_sum(points: np.ndarray, forces: np.ndarray, mu: float, nu: float, tgt=None) -> np.ndarray:
    """E1: u_i(x_l) = sum_{m != l} sum_j K_ij(x_l, x_m) f_j(x_m), K Kelvin's solution,
    K_ij = ((3 - 4 nu) delta_ij/r + r_i r_j/r^3)/(16 pi mu (1 - nu)); layouts as stokes_direct_sum."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[1]
    f = np.ascontiguousarray(np.asarray(forces, dtype=np.float64).reshape(-1, 3, n))
    nf = f.shape[0]
    t = np.arange(n, dtype=np.int64) if tgt is None else np.ascontiguousarray(tgt, dtype=np.int64)
    out = np.zeros((nf, 3, t.shape[0]), dtype=np.float64)
    x, y, z = (np.ascontiguousarray(pts[i]) for i in range(3))
    lib.orc_elastic_direct_sum(n, _ptr(x), _ptr(y), _ptr(z), float(mu), float(nu), nf, _ptr(f), t.shape[0],
                               _ptr(t), _ptr(out))
    return out


class OracleError(RuntimeError):
    pass


class Plan:
    """O2: plain CPU IFGF plan (tree, cousins, relevant cones) and its FP64 apply."""

    def __init__(self, points, kappa, orders=DEFAULT_ORDERS, levels=0, leaf_target=DEFAULT_LEAF_TARGET,
                 base_cones=DEFAULT_BASE_CONES, tau=DEFAULT_TAU):
        lib = _load()
        self._lib = lib
        pts = np.ascontiguousarray(points, dtype=np.float64)
        self._xyz = [np.ascontiguousarray(pts[i]) for i in range(3)]
        st = ctypes.c_int(0)
        h = lib.orc_plan_create(pts.shape[1], _ptr(self._xyz[0]), _ptr(self._xyz[1]), _ptr(self._xyz[2]),
                                float(kappa), int(orders[0]), int(orders[1]), int(orders[2]), int(levels),
                                int(leaf_target), int(base_cones[0]), int(base_cones[1]), int(base_cones[2]),
                                float(tau), ctypes.byref(st))
        if not h:
            raise OracleError(f"orc_plan_create failed with status {st.value}")
        self._h = h
        self.status = st.value
        info = np.zeros(44, dtype=np.int64)
        geom = np.zeros(4, dtype=np.float64)
        lib.orc_info(h, _ptr(info), _ptr(geom))
        self.N = int(info[0])
        self.D = int(info[1])
        self.nbox = {d: int(info[1 + d]) for d in range(1, self.D + 1)}
        self.ncone = {d: int(info[22 + d]) for d in range(3, self.D + 1)}
        self.a = geom[:3].copy()
        self.H1 = float(geom[3])
        self.kappa = float(kappa)
        self.orders = tuple(int(o) for o in orders)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_plan_destroy(h)
            self._h = None

    def get(self, what: int, level: int = 0) -> np.ndarray:
        n = self._lib.orc_get(self._h, what, level, None)
        if n < 0:
            raise OracleError(f"query {what} unavailable at level {level}")
        buf = np.zeros(max(n, 1), dtype=np.int64)
        self._lib.orc_get(self._h, what, level, _ptr(buf))
        return buf[:n]

    def grid(self, level: int):
        return tuple(int(v) for v in self.get(Q_GRID, level))

    def offsets(self) -> np.ndarray:
        out = np.zeros((self.N, 3), dtype=np.float32)
        self._lib.orc_offsets(self._h, _ptr(out))
        return out

    def classify(self, level: int, v: np.ndarray) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1, 3)
        out = np.zeros(v.shape[0], dtype=np.int64)
        self._lib.orc_classify(self._h, level, v.shape[0], _ptr(v), _ptr(out))
        return out

    def has_duplicates(self) -> bool:
        return bool(self._lib.orc_has_duplicates(self._h))

    def cheb_nodes(self):
        ts = np.zeros(self.orders[0])
        tt = np.zeros(self.orders[1])
        tp = np.zeros(self.orders[2])
        self._lib.orc_cheb_nodes(self._h, _ptr(ts), _ptr(tt), _ptr(tp))
        return ts, tt, tp

    def cheb3(self, values: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(values, dtype=np.complex128).reshape(-1)
        c = np.zeros_like(f)
        self._lib.orc_cheb3(self._h, _ptr(f), _ptr(c))
        return c

    def cheb3_eval(self, coef: np.ndarray, t: np.ndarray) -> np.ndarray:
        c = np.ascontiguousarray(coef, dtype=np.complex128).reshape(-1)
        tt = np.ascontiguousarray(t, dtype=np.float64).reshape(-1, 3)
        out = np.zeros(tt.shape[0], dtype=np.complex128)
        self._lib.orc_cheb3_eval(self._h, _ptr(c), tt.shape[0], _ptr(tt), _ptr(out))
        return out

    def apply(self, dens: np.ndarray, near: bool = True, level_mask: int = -1) -> np.ndarray:
        """FP64 IFGF apply; dens (nrhs, N) or (N,) in the caller's order -> (nrhs, N)."""
        a = np.ascontiguousarray(np.atleast_2d(dens), dtype=np.complex128)
        out = np.zeros_like(a)
        st = self._lib.orc_apply(self._h, a.shape[0], _ptr(a), _ptr(out), 1 if near else 0, int(level_mask))
        if st != 0:
            raise OracleError(f"orc_apply failed with status {st}")
        return out

    def apply_stokes(self, forces: np.ndarray, near: bool = True, level_mask: int = -1) -> np.ndarray:
        """FP64 IFGF apply of the Stokeslet (kappa = 0 plans); forces (nf, 3, N) or (3, N) real in the
        caller's order -> velocities (nf, 3, N)."""
        f = np.ascontiguousarray(np.asarray(forces, dtype=np.float64).reshape(-1, 3, self.N))
        out = np.zeros_like(f)
        st = self._lib.orc_apply_stokes(self._h, f.shape[0], _ptr(f), _ptr(out), 1 if near else 0, int(level_mask))
        if st != 0:
            raise OracleError(f"orc_apply_stokes failed with status {st}")
        return out

    def apply_elastic(self, forces: np.ndarray, mu: float, nu: float, near: bool = True,
                      level_mask: int = -1) -> np.ndarray:
        """FP64 IFGF apply of Kelvin's solution (kappa = 0 plans), layouts as apply_stokes."""
        f = np.ascontiguousarray(np.asarray(forces, dtype=np.float64).reshape(-1, 3, self.N))
        out = np.zeros_like(f)
        st = self._lib.orc_apply_elastic(self._h, float(mu), float(nu), f.shape[0], _ptr(f), _ptr(out),
                                         1 if near else 0, int(level_mask))
        if st != 0:
            raise OracleError(f"orc_apply_elastic failed with status {st}")
        return out

    def shard_cones(self, level: int, points: tuple, parent_cones: tuple) -> np.ndarray:
        """M1: per level-`level` cone, bit 0 set when Interpolation(level) of the sorted points
        [points[0], points[1]) looks it up, bit 1 when Propagation(level) of the level-(level-1) cones
        [parent_cones[0], parent_cones[1]) does (the data a rank gathers from others, Sec. 3.2.3)."""
        out = np.zeros(max(self.ncone[level], 1), dtype=np.uint8)
        st = self._lib.orc_shard_cones(self._h, int(level), int(points[0]), int(points[1]), int(parent_cones[0]),
                                       int(parent_cones[1]), _ptr(out))
        if st != 0:
            raise OracleError(f"orc_shard_cones failed with status {st}")
        return out[: self.ncone[level]]

    def shard_points(self, points: tuple, leaf_cones: tuple) -> np.ndarray:
        """M1: per sorted point, bit 0 set when the near field of the sorted points [points[0],
        points[1]) reads it, bit 1 when LevelDEvaluations of the level-D cones [leaf_cones[0],
        leaf_cones[1]) does."""
        out = np.zeros(self.N, dtype=np.uint8)
        self._lib.orc_shard_points(self._h, int(points[0]), int(points[1]), int(leaf_cones[0]), int(leaf_cones[1]),
                                   _ptr(out))
        return out

    def work(self) -> dict:
        """Exact work counters of the last apply: near pairs, leaf pairs, per-level evaluations."""
        w0 = self.get(Q_WORK, self.D)
        res = {"near_pairs": int(w0[0]), "leaf_pairs": int(w0[1]), "interp": {}, "prop": {}}
        for d in range(3, self.D + 1):
            w = self.get(Q_WORK, d)
            res["interp"][d] = int(w[2])
            res["prop"][d] = int(w[3])
        return res


def partition_boxes(box_start: np.ndarray, nranks: int) -> np.ndarray:
    """Sec. 3.2.1: the Morton-ordered leaf boxes in nranks intervals whose point counts are as close
    as possible to N / nranks.  Reading: bound r is the box boundary whose point offset is nearest
    to r N / nranks (the lower one on a tie), non-decreasing in r; rank r owns boxes
    [bound r, bound r+1)."""
    box_start = np.asarray(box_start, dtype=np.int64)
    nbox = box_start.shape[0] - 1
    n = int(box_start[-1])
    bounds = [0]
    for r in range(1, nranks):
        t = n * r / nranks
        best = min(range(nbox + 1), key=lambda b: (abs(box_start[b] - t), b))
        bounds.append(max(best, bounds[-1]))
    bounds.append(nbox)
    return np.array(bounds, dtype=np.int64)


def partition_cones(nc: int, nranks: int) -> np.ndarray:
    """Sec. 3.2.1: a level's relevant cones, in cone order, in nranks contiguous intervals of
    (nearly) equal size: rank r owns [floor(r nc / nranks), floor((r + 1) nc / nranks))."""
    return np.array([nc * r // nranks for r in range(nranks + 1)], dtype=np.int64)


def rel_l2(approx: np.ndarray, exact: np.ndarray) -> float:
    """Relative L2 error of the paper's error estimator (SM, Eq. (errorcomputation))."""
    num = np.sum(np.abs(np.asarray(approx) - np.asarray(exact)) ** 2)
    den = np.sum(np.abs(np.asarray(exact)) ** 2)
    return float(np.sqrt(num / den))

"""Thin ctypes binding of libdses.so (include/dses.h), same names as the C ABI.

Argument marshalling only: every step of a registration runs in the CUDA
library. The library must have been built (paper_2502_00115_b300.build); if it
is missing, importing the binding's loader raises instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdses.so")

DSES_OK = 0
DSES_NOT_READY = 1
DSES_ERR_INVALID_ARG = -1
DSES_ERR_OOM = -2
DSES_ERR_CUDA = -3
DSES_ERR_QUEUE_FULL = -4
DSES_ERR_TIMEOUT = -5
DSES_ERR_NO_CANDIDATE = -6
DSES_ERR_UNKNOWN_TICKET = -7
DSES_ERR_EXCHANGE = -8

DSES_METRIC_INLIER, DSES_METRIC_TRUNC_L1, DSES_METRIC_TRUNC_L2, DSES_METRIC_HUBER, DSES_METRIC_LP = range(5)
DSES_GRID_HOPF, DSES_GRID_EULER_BOX, DSES_GRID_EXPLICIT = range(3)
DSES_NN_GRID, DSES_NN_BRUTE = range(2)

METRICS = {"inlier": 0, "trunc_l1": 1, "trunc_l2": 2, "huber": 3, "lp": 4}


class dses_rotation_grid(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("hopf_n", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("delta_r", ctypes.c_double),
        ("R0", ctypes.c_double * 9),
        ("explicit_R", ctypes.POINTER(ctypes.c_float)),
        ("n_explicit", ctypes.c_int64),
    ]


class dses_params(ctypes.Structure):
    _fields_ = [
        ("metric", ctypes.c_int32),
        ("epsilon", ctypes.c_float),
        ("delta_t", ctypes.c_float),
        ("tau", ctypes.c_float),
        ("huber_h", ctypes.c_float),
        ("p", ctypes.c_float),
        ("t_center", ctypes.c_float * 3),
        ("t_half", ctypes.c_float * 3),
        ("q_milli", ctypes.c_int32),
        ("top_k", ctypes.c_int32),
        ("nn_mode", ctypes.c_int32),
        ("refine_top_k", ctypes.c_int32),
        ("refine_K", ctypes.c_int32),
        ("refine_delta_r", ctypes.c_double),
    ]


class dses_result(ctypes.Structure):
    _fields_ = [
        ("R", ctypes.c_float * 9),
        ("t", ctypes.c_float * 3),
        ("rot_index", ctypes.c_int64),
        ("inliers", ctypes.c_uint32),
        ("votes", ctypes.c_uint32),
        ("cost", ctypes.c_float),
        ("status", ctypes.c_int32),
    ]


class dses_problem(ctypes.Structure):
    _fields_ = [
        ("target", ctypes.c_void_p),
        ("src", ctypes.c_void_p),
        ("n_src", ctypes.c_int64),
        ("src_is_device", ctypes.c_int32),
        ("grid", dses_rotation_grid),
        ("params", dses_params),
    ]


# int32_t (*dses_allgather_fn)(void* user, const void* send, int64_t bytes, void* recv)
ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()

# exported C symbols and their signatures
_P = ctypes.POINTER
_vp, _i32, _i64, _f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
SIGNATURES = {
    "dses_create": (_i32, [_i32, _vp, _P(_vp)]),
    "dses_destroy": (_i32, [_vp]),
    "dses_create_target": (_i32, [_vp, _vp, _i64, _i32, _f32, _i32, _P(_vp)]),
    "dses_destroy_target": (_i32, [_vp, _vp]),
    "dses_register": (_i32, [_vp, _P(dses_problem), _P(dses_result)]),
    "dses_register_batch": (_i32, [_vp, _P(dses_problem), _i32, _P(dses_result)]),
    "dses_submit": (_i32, [_vp, _P(dses_problem), _P(ctypes.c_uint64)]),
    "dses_poll": (_i32, [_vp, ctypes.c_uint64, _P(dses_result)]),
    "dses_debug_per_rotation": (_i32, [_vp, _P(dses_problem), _vp, _vp, _vp, _vp, _P(dses_result)]),
    "dses_debug_per_rotation_batch": (_i32, [_vp, _P(dses_problem), _i32, _P(_vp), _P(_vp), _P(_vp), _P(_vp),
                                             _P(dses_result)]),
    "dses_rotation_grid_build": (_i32, [_vp, _P(dses_rotation_grid), _vp, _i64, _P(_i64)]),
    "dses_target_distance_grid": (_i32, [_vp, _vp, _vp, _vp, _vp, _P(_i32), _P(_f32)]),
    "dses_set_option": (_i32, [_vp, ctypes.c_char_p, _i64]),
    "dses_get_option": (_i32, [_vp, ctypes.c_char_p, _P(_i64)]),
    "dses_vote_static": (_i32, [_i32, _vp, _vp, _i64, _vp, _i64, _vp, _i64, _P(dses_params), _vp]),
    "dses_exhaustive_search": (_i32, [_vp, _P(dses_problem), _vp, _i64, _P(dses_result)]),
    "dses_refine_translation": (_i32, [_vp, _vp, _vp, _i64, _i32, _vp, _vp, _f32, _i32, _vp, _P(ctypes.c_uint32)]),
    "dses_shard_range": (_i32, [_i64, _i32, _i32, _P(_i64), _P(_i64)]),
    "dses_register_shard": (_i32, [_vp, _P(dses_problem), _i32, _i32, _P(dses_result)]),
    "dses_combine_results": (_i32, [_P(dses_result), _i32, _P(dses_result)]),
    "dses_register_sharded": (_i32, [_vp, _P(dses_problem), _i32, _i32, ALLGATHER_FN, _vp, _P(dses_result)]),
    "dses_last_error": (ctypes.c_char_p, [_vp]),
    "dses_status_string": (ctypes.c_char_p, [_i32]),
}


def load(path: str = LIB_PATH):
    """Load libdses.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with python -m paper_2502_00115_b300.build")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class DsesError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def status_string(s: int) -> str:
    return load().dses_status_string(s).decode()


# ---------------------------------------------------------------------------
# functions with the C ABI's names (raw status returned)


def dses_create(device: int = 0, stream: int | None = None):
    h = ctypes.c_void_p()
    st = load().dses_create(device, ctypes.c_void_p(stream or 0), ctypes.byref(h))
    return st, h


def dses_destroy(ctx) -> int:
    return load().dses_destroy(ctx)


def dses_create_target(ctx, xyz_ptr: int, m: int, ptr_is_device: int, grid_cap: float, grid_res: int):
    h = ctypes.c_void_p()
    st = load().dses_create_target(ctx, ctypes.c_void_p(xyz_ptr), m, ptr_is_device, grid_cap, grid_res, ctypes.byref(h))
    return st, h


def dses_destroy_target(ctx, target) -> int:
    return load().dses_destroy_target(ctx, target)


def dses_register(ctx, problem: dses_problem):
    out = dses_result()
    st = load().dses_register(ctx, ctypes.byref(problem), ctypes.byref(out))
    return st, out


def dses_register_batch(ctx, problems):
    n = len(problems)
    arr = (dses_problem * n)(*problems)
    out = (dses_result * n)()
    st = load().dses_register_batch(ctx, arr, n, out)
    return st, list(out)


def dses_submit(ctx, problem: dses_problem):
    t = ctypes.c_uint64()
    st = load().dses_submit(ctx, ctypes.byref(problem), ctypes.byref(t))
    return st, t.value


def dses_poll(ctx, ticket: int):
    out = dses_result()
    st = load().dses_poll(ctx, ticket, ctypes.byref(out))
    return st, out


def dses_debug_per_rotation(ctx, problem: dses_problem, n_rot: int):
    k = np.zeros((n_rot, 3), dtype=np.int32)
    V = np.zeros(n_rot, dtype=np.uint32)
    M = np.zeros(n_rot, dtype=np.uint32)
    C = np.zeros(n_rot, dtype=np.float32)
    out = dses_result()
    st = load().dses_debug_per_rotation(ctx, ctypes.byref(problem), k.ctypes.data, V.ctypes.data, M.ctypes.data,
                                        C.ctypes.data, ctypes.byref(out))
    return st, k, V, M, C, out


def dses_debug_per_rotation_batch(ctx, problems, n_rots):
    """Per-problem (k*, V, M, cost) arrays of a batched run; n_rots[b] = problem b's rotations."""
    n = len(problems)
    arr = (dses_problem * n)(*problems)
    ks = [np.zeros((m, 3), dtype=np.int32) for m in n_rots]
    Vs = [np.zeros(m, dtype=np.uint32) for m in n_rots]
    Ms = [np.zeros(m, dtype=np.uint32) for m in n_rots]
    Cs = [np.zeros(m, dtype=np.float32) for m in n_rots]
    ptrs = lambda arrs: (_vp * n)(*[a.ctypes.data for a in arrs])
    out = (dses_result * n)()
    st = load().dses_debug_per_rotation_batch(ctx, arr, n, ptrs(ks), ptrs(Vs), ptrs(Ms), ptrs(Cs), out)
    return st, ks, Vs, Ms, Cs, list(out)


def dses_rotation_grid_build(ctx, grid: dses_rotation_grid):
    cnt = ctypes.c_int64()
    st = load().dses_rotation_grid_build(ctx, ctypes.byref(grid), None, 0, ctypes.byref(cnt))
    if st != DSES_OK:
        return st, None
    R = np.zeros((cnt.value, 3, 3), dtype=np.float32)
    st = load().dses_rotation_grid_build(ctx, ctypes.byref(grid), R.ctypes.data, cnt.value, ctypes.byref(cnt))
    return st, R


def dses_target_distance_grid(ctx, target):
    res = ctypes.c_int32()
    cap = ctypes.c_float()
    lo = np.zeros(3, dtype=np.float32)
    h = np.zeros(3, dtype=np.float32)
    st = load().dses_target_distance_grid(ctx, target, None, lo.ctypes.data, h.ctypes.data, ctypes.byref(res),
                                          ctypes.byref(cap))
    if st != DSES_OK:
        return st, None, lo, h, cap.value
    D = np.zeros((res.value,) * 3, dtype=np.float32)
    st = load().dses_target_distance_grid(ctx, target, D.ctypes.data, lo.ctypes.data, h.ctypes.data,
                                          ctypes.byref(res), ctypes.byref(cap))
    return st, D, lo, h, cap.value


def dses_set_option(ctx, key: str, value: int) -> int:
    return load().dses_set_option(ctx, key.encode(), int(value))


def dses_get_option(ctx, key: str):
    v = ctypes.c_int64()
    st = load().dses_get_option(ctx, key.encode(), ctypes.byref(v))
    return st, v.value


def dses_vote_static(device: int, stream: int, src_ptr: int, n_src: int, tgt_ptr: int, n_tgt: int, rot_ptr: int,
                     n_rot: int, params: dses_params, kv_ptr: int) -> int:
    return load().dses_vote_static(device, ctypes.c_void_p(stream or 0), ctypes.c_void_p(src_ptr), n_src,
                                   ctypes.c_void_p(tgt_ptr), n_tgt, ctypes.c_void_p(rot_ptr), n_rot,
                                   ctypes.byref(params), ctypes.c_void_p(kv_ptr))


def dses_refine_translation(ctx, target, src, n_src: int, src_is_device: int, R, t, epsilon: float,
                            iterations: int = 1):
    """src: a float32 (n, 3) array, or a device pointer with src_is_device = 1.
    Returns (status, t_refined float32[3], n_inliers)."""
    Rh = np.ascontiguousarray(np.asarray(R, dtype=np.float32).reshape(9))
    th = np.ascontiguousarray(np.asarray(t, dtype=np.float32).reshape(3))
    out = np.zeros(3, dtype=np.float32)
    n = ctypes.c_uint32()
    if src_is_device:
        sp = ctypes.c_void_p(src)
    else:
        src = np.ascontiguousarray(np.asarray(src, dtype=np.float32))
        sp = ctypes.c_void_p(src.ctypes.data)
    st = load().dses_refine_translation(ctx, target, sp, n_src, src_is_device, Rh.ctypes.data, th.ctypes.data,
                                        epsilon, iterations, out.ctypes.data, ctypes.byref(n))
    return st, out, n.value


def dses_exhaustive_search(ctx, problem: dses_problem, n_entries: int = 0):
    """Returns (status, result, cost array of n_entries floats or None)."""
    r = dses_result()
    cost = np.zeros(n_entries, dtype=np.float32) if n_entries else None
    st = load().dses_exhaustive_search(ctx, ctypes.byref(problem), cost.ctypes.data if cost is not None else None,
                                       n_entries, ctypes.byref(r))
    return st, r, cost


def dses_shard_range(n_rot: int, rank: int, world: int):
    b, e = ctypes.c_int64(), ctypes.c_int64()
    st = load().dses_shard_range(n_rot, rank, world, ctypes.byref(b), ctypes.byref(e))
    return st, b.value, e.value


def dses_register_shard(ctx, problem: dses_problem, rank: int, world: int):
    out = dses_result()
    st = load().dses_register_shard(ctx, ctypes.byref(problem), rank, world, ctypes.byref(out))
    return st, out


def make_allgather(gather_bytes):
    """A dses_allgather_fn from a Python function gather_bytes(bytes) -> list of
    bytes (one per shard, in rank order). Keep the returned object alive for as
    long as the library may call it."""

    def fn(user, send, nbytes, recv):
        try:
            mine = ctypes.string_at(send, nbytes)
            parts = gather_bytes(mine)
            blob = b"".join(parts)
            if any(len(q) != nbytes for q in parts):
                return 1
            ctypes.memmove(recv, blob, len(blob))
            return 0
        except Exception:  # an exception must not cross the C boundary
            return 1

    return ALLGATHER_FN(fn)


def dses_register_sharded(ctx, problem: dses_problem, rank: int, world: int, allgather):
    """allgather: an ALLGATHER_FN (see make_allgather)."""
    out = dses_result()
    st = load().dses_register_sharded(ctx, ctypes.byref(problem), rank, world, allgather, None, ctypes.byref(out))
    return st, out


def dses_combine_results(parts):
    arr = (dses_result * len(parts))(*parts)
    out = dses_result()
    st = load().dses_combine_results(arr, len(parts), ctypes.byref(out))
    return st, out


def dses_last_error(ctx) -> str:
    return load().dses_last_error(ctx).decode()


# ---------------------------------------------------------------------------
# convenience layer (still marshalling only)


def make_params(metric="trunc_l1", epsilon=0.02, delta_t=0.0, tau=0.0, huber_h=0.0, p=1.0,
                t_center=(0.0, 0.0, 0.0), t_half=(0.9, 0.9, 0.9), q_milli=0, top_k=0, nn_mode="grid",
                refine_top_k=0, refine_K=0, refine_delta_r=0.0) -> dses_params:
    P = dses_params()
    P.metric = METRICS[metric] if isinstance(metric, str) else int(metric)
    P.epsilon = epsilon
    P.delta_t = delta_t
    P.tau = tau
    P.huber_h = huber_h
    P.p = p
    P.t_center[:] = list(t_center)
    P.t_half[:] = list(t_half)
    P.q_milli = q_milli
    P.top_k = top_k
    P.nn_mode = {"grid": 0, "brute": 1}[nn_mode] if isinstance(nn_mode, str) else int(nn_mode)
    P.refine_top_k = refine_top_k
    P.refine_K = refine_K
    P.refine_delta_r = refine_delta_r
    return P


def hopf_grid(n: int) -> dses_rotation_grid:
    g = dses_rotation_grid()
    g.kind = DSES_GRID_HOPF
    g.hopf_n = n
    return g


def euler_box_grid(R0, K: int, delta_r: float) -> dses_rotation_grid:
    g = dses_rotation_grid()
    g.kind = DSES_GRID_EULER_BOX
    g.K = K
    g.delta_r = delta_r
    g.R0[:] = [float(v) for v in np.asarray(R0, dtype=np.float64).reshape(9)]
    return g


def explicit_grid(R: np.ndarray) -> tuple[dses_rotation_grid, np.ndarray]:
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float32).reshape(-1, 9))
    g = dses_rotation_grid()
    g.kind = DSES_GRID_EXPLICIT
    g.explicit_R = R.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    g.n_explicit = len(R)
    return g, R  # keep R alive while the grid is used


class Context:
    """Owns a dses_ctx; raises DsesError on a failing call."""

    def __init__(self, device: int = 0, stream: int | None = None):
        st, self.h = dses_create(device, stream)
        if st != DSES_OK:
            raise DsesError(st, "dses_create failed")
        self._keep = []

    def check(self, st: int, allow=(DSES_OK,)):
        if st not in allow:
            raise DsesError(st, dses_last_error(self.h))
        return st

    def close(self):
        if self.h:
            dses_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_option(self, key, value):
        self.check(dses_set_option(self.h, key, value))

    def get_option(self, key):
        st, v = dses_get_option(self.h, key)
        self.check(st)
        return v

    def create_target(self, Y: np.ndarray, grid_cap: float, grid_res: int = 128):
        Y = np.ascontiguousarray(np.asarray(Y, dtype=np.float32))
        st, t = dses_create_target(self.h, Y.ctypes.data, len(Y), 0, grid_cap, grid_res)
        self.check(st)
        return t

    def create_target_device(self, ptr: int, m: int, grid_cap: float, grid_res: int = 128):
        st, t = dses_create_target(self.h, ptr, m, 1, grid_cap, grid_res)
        self.check(st)
        return t

    def destroy_target(self, t):
        self.check(dses_destroy_target(self.h, t))

    def problem(self, target, X: np.ndarray | None = None, grid=None, params=None, src_ptr: int | None = None,
                n_src: int | None = None) -> dses_problem:
        pb = dses_problem()
        pb.target = target
        if src_ptr is not None:
            pb.src = src_ptr
            pb.n_src = n_src
            pb.src_is_device = 1
        else:
            X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
            self._keep.append(X)
            pb.src = X.ctypes.data
            pb.n_src = len(X)
            pb.src_is_device = 0
        pb.grid = grid
        pb.params = params
        return pb

    def register(self, pb: dses_problem) -> dses_result:
        st, r = dses_register(self.h, pb)
        self.check(st, allow=(DSES_OK, DSES_ERR_NO_CANDIDATE))
        return r

    def register_shard(self, pb: dses_problem, rank: int, world: int) -> dses_result:
        st, r = dses_register_shard(self.h, pb, rank, world)
        self.check(st, allow=(DSES_OK, DSES_ERR_NO_CANDIDATE))
        return r

    def register_sharded(self, pb: dses_problem, rank: int, world: int, allgather) -> dses_result:
        st, r = dses_register_sharded(self.h, pb, rank, world, allgather)
        self.check(st, allow=(DSES_OK, DSES_ERR_NO_CANDIDATE))
        return r

    def register_batch(self, pbs) -> list:
        st, rs = dses_register_batch(self.h, pbs)
        self.check(st, allow=(DSES_OK, DSES_ERR_NO_CANDIDATE))
        return rs

    def debug(self, pb: dses_problem, n_rot: int):
        st, k, V, M, C, r = dses_debug_per_rotation(self.h, pb, n_rot)
        self.check(st, allow=(DSES_OK, DSES_ERR_NO_CANDIDATE))
        return k, V, M, C, r

    def debug_batch(self, pbs, n_rots):
        st, k, V, M, C, r = dses_debug_per_rotation_batch(self.h, pbs, n_rots)
        self.check(st, allow=(DSES_OK, DSES_ERR_NO_CANDIDATE))
        return k, V, M, C, r

    def submit(self, pb: dses_problem) -> int:
        st, t = dses_submit(self.h, pb)
        self.check(st)
        return t

    def poll(self, ticket: int):
        st, r = dses_poll(self.h, ticket)
        return st, r

    def rotation_grid(self, grid) -> np.ndarray:
        st, R = dses_rotation_grid_build(self.h, grid)
        self.check(st)
        return R

    def distance_grid(self, target):
        st, D, lo, h, cap = dses_target_distance_grid(self.h, target)
        self.check(st)
        return D, lo, h, cap

    def exhaustive(self, pb: dses_problem, n_entries: int = 0):
        st, r, cost = dses_exhaustive_search(self.h, pb, n_entries)
        self.check(st)
        return r, cost

    def refine_translation(self, target, X, R, t, epsilon: float, iterations: int = 1):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        st, tr, n = dses_refine_translation(self.h, target, X, len(X), 0, R, t, epsilon, iterations)
        self.check(st)
        return tr, n


def shard_range(n_rot: int, rank: int, world: int) -> tuple[int, int]:
    st, b, e = dses_shard_range(n_rot, rank, world)
    if st != DSES_OK:
        raise DsesError(st, f"bad shard {rank} of {world} over {n_rot} rotations")
    return b, e


def combine_results(parts) -> dses_result:
    """The whole registration's result from its shards' results (dses_combine_results)."""
    st, r = dses_combine_results(list(parts))
    if st not in (DSES_OK, DSES_ERR_NO_CANDIDATE):
        raise DsesError(st, "shard results cannot be combined (a shard failed)")
    return r


def result_dict(r: dses_result) -> dict:
    return {
        "R": np.array(r.R[:], dtype=np.float32).reshape(3, 3),
        "t": np.array(r.t[:], dtype=np.float32),
        "rot_index": int(r.rot_index),
        "inliers": int(r.inliers),
        "votes": int(r.votes),
        "cost": float(r.cost),
        "status": int(r.status),
    }

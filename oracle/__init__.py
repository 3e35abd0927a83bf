"""FP64 CPU oracle for DSES (test infrastructure only).

Plain single-threaded C++ restatement of Algorithm 2 of arXiv 2502.00115 (see
oracle.cpp for the passages each function follows and the readings taken).
Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package; the CUDA library never does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

METRICS = {"inlier": 0, "trunc_l1": 1, "trunc_l2": 2, "huber": 3, "lp": 4}


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (plain g++ -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("metric", ctypes.c_int),
        ("epsilon", ctypes.c_double),
        ("delta_t", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("huber_h", ctypes.c_double),
        ("p", ctypes.c_double),
        ("t_center", ctypes.c_double * 3),
        ("t_half", ctypes.c_double * 3),
        ("q_milli", ctypes.c_int),
        ("top_k", ctypes.c_int),
        ("nn_mode", ctypes.c_int),
        ("grid_res", ctypes.c_int),
        ("grid_cap", ctypes.c_double),
        ("band", ctypes.c_double),
        ("refine_top_k", ctypes.c_int),
        ("refine_K", ctypes.c_int),
        ("refine_delta_r", ctypes.c_double),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("rot_index", ctypes.c_int64),
        ("R", ctypes.c_double * 9),
        ("t", ctypes.c_double * 3),
        ("votes", ctypes.c_int64),
        ("inliers", ctypes.c_int64),
        ("cost", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # test hook: DSES_ORACLE_LIB names another build of oracle.cpp (the
            # mutation test loads copies with a planted mistake)
            alt = os.environ.get("DSES_ORACLE_LIB")
            if not alt:
                build()
            lib = ctypes.CDLL(alt or _LIB)
            P = ctypes.POINTER
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            pd, pi64, pi32 = P(d), P(i64), P(i32)
            sig = {
                "orc_hopf_count": (i64, [i32]),
                "orc_healpix_centres": (None, [i32, pd, pd]),
                "orc_hopf_rotation": (None, [i32, i64, pd]),
                "orc_hopf_grid": (None, [i32, pd]),
                "orc_euler_box": (None, [pd, i32, d, pd]),
                "orc_lattice_box": (None, [pd, pd, d, pi32, pi32]),
                "orc_vote": (None, [pd, i64, pd, i64, pd, d, pi32, pi32, d, pi32, pi64, pi64]),
                "orc_vote_consistent": (i32, [pd, i64, pd, i64, pd, d, pi32, pi32, d, pi32, i64]),
                "orc_nn_dist": (None, [pd, i64, pd, i64, pd, pd, pd]),
                "orc_inliers": (None, [pd, i64, pd, i64, pd, pd, d, d, pi64, pi64]),
                "orc_refine_translation": (i64, [pd, i64, pd, i64, pd, pd, d, d, pd, pi64, pi64]),
                "orc_rho": (d, [P(Params), d]),
                "orc_exhaustive": (i64, [pd, i64, pd, i64, pd, i64, P(Params), pd, pi64, d, pi64]),
                "orc_cost_exact": (d, [pd, i64, pd, i64, pd, pd, P(Params)]),
                "orc_dist_grid_geometry": (None, [pd, i64, i32, d, pd, pd]),
                "orc_dist_grid": (None, [pd, i64, i32, d, pd]),
                "orc_dist_grid_threads": (None, [pd, i64, i32, d, pd, i32]),
                "orc_grid_lookup": (d, [pd, i32, pd, pd, d, pd]),
                "orc_cost_grid": (d, [pd, i64, pd, i32, pd, pd, d, pd, pd, P(Params)]),
                "orc_register": (i32, [pd, i64, pd, i64, pd, i64, P(Params), P(ctypes.c_int32), pi64, pi64, pd,
                                       pi64, pi64, P(Result)]),
                "orc_register_threads": (i32, [pd, i64, pd, i64, pd, i64, P(Params), i32, P(Result)]),
                "orc_register_threads_out": (i32, [pd, i64, pd, i64, pd, i64, P(Params), i32, P(ctypes.c_int32),
                                                   pi64, pi64, pd, pi64, pi64, P(Result)]),
                "orc_field_create": (ctypes.c_void_p, [pd, i64, i32, d]),
                "orc_field_free": (None, [ctypes.c_void_p]),
                "orc_field_create_threads": (ctypes.c_void_p, [pd, i64, i32, d, i32]),
                "orc_register_field_threads": (i32, [pd, i64, pd, i64, pd, i64, P(Params), ctypes.c_void_p, i32,
                                                     P(Result)]),
                "orc_eval_rotation": (None, [pd, i64, pd, i64, pd, P(Params), pi32, pi64, pi64, pi64, pi64]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_params(metric="trunc_l1", epsilon=0.02, delta_t=None, tau=None, huber_h=None, p=0.5,
                t_center=(0.0, 0.0, 0.0), t_half=(0.9, 0.9, 0.9), q_milli=0, top_k=0, nn_mode="grid",
                grid_res=128, grid_cap=None, band=1e-5, refine_top_k=0, refine_K=0, refine_delta_r=0.0) -> Params:
    P = Params()
    P.metric = METRICS[metric] if isinstance(metric, str) else int(metric)
    P.epsilon = epsilon
    P.delta_t = epsilon if delta_t is None else delta_t
    P.tau = 2 * epsilon if tau is None else tau
    P.huber_h = epsilon if huber_h is None else huber_h
    P.p = p
    P.t_center[:] = list(t_center)
    P.t_half[:] = list(t_half)
    P.q_milli = q_milli
    P.top_k = top_k
    P.nn_mode = {"grid": 0, "brute": 1}[nn_mode] if isinstance(nn_mode, str) else int(nn_mode)
    P.grid_res = grid_res
    P.grid_cap = (2 * P.tau) if grid_cap in (None, 0, 0.0) else grid_cap
    P.band = band
    P.refine_top_k = refine_top_k
    P.refine_K = refine_K
    P.refine_delta_r = refine_delta_r
    return P


def params_from_problem(prob, nn_mode="grid", **over) -> Params:
    kw = dict(metric=prob.metric, epsilon=prob.epsilon, delta_t=prob.delta_t, tau=prob.tau,
              huber_h=prob.huber_h, t_center=prob.t_center, t_half=prob.t_half, q_milli=prob.q_milli,
              top_k=prob.top_k, nn_mode=nn_mode, grid_res=prob.grid_res, grid_cap=prob.grid_cap or None,
              refine_top_k=prob.refine_top_k, refine_K=prob.refine_K, refine_delta_r=prob.refine_delta_r)
    kw.update(over)
    return make_params(**kw)


# ---------------------------------------------------------------------------
# thin numpy wrappers


def hopf_count(n: int) -> int:
    return int(_load().orc_hopf_count(n))


def healpix_centres(n: int):
    npix = 12 * n * n
    th = np.zeros(npix)
    ph = np.zeros(npix)
    _load().orc_healpix_centres(n, _pd(th), _pd(ph))
    return th, ph


def hopf_grid(n: int) -> np.ndarray:
    R = np.zeros((hopf_count(n), 3, 3))
    _load().orc_hopf_grid(n, _pd(R))
    return R


def hopf_rotation(n: int, r: int) -> np.ndarray:
    R = np.zeros((3, 3))
    _load().orc_hopf_rotation(n, int(r), _pd(R))
    return R


def euler_box(R0, K: int, delta_r: float) -> np.ndarray:
    R0 = _f64(R0)
    out = np.zeros(((2 * K + 1) ** 3, 3, 3))
    _load().orc_euler_box(_pd(R0), K, delta_r, _pd(out))
    return out


def lattice_box(t_center, t_half, delta):
    c, s = _f64(t_center), _f64(t_half)
    lo = (ctypes.c_int * 3)()
    hi = (ctypes.c_int * 3)()
    _load().orc_lattice_box(_pd(c), _pd(s), delta, lo, hi)
    return np.array(lo[:]), np.array(hi[:])


def vote(X, Y, R, delta, lo, hi, band=1e-5):
    X, Y, R = _f64(X), _f64(Y), _f64(R)
    lo = (ctypes.c_int * 3)(*map(int, lo))
    hi = (ctypes.c_int * 3)(*map(int, hi))
    k = (ctypes.c_int * 3)()
    V = ctypes.c_int64()
    nb = ctypes.c_int64()
    _load().orc_vote(_pd(X), len(X), _pd(Y), len(Y), _pd(R), delta, lo, hi, band, k, ctypes.byref(V),
                     ctypes.byref(nb))
    return np.array(k[:]), int(V.value), int(nb.value)


def vote_consistent(X, Y, R, delta, lo, hi, k_claim, V_claim, band=1e-5) -> int:
    X, Y, R = _f64(X), _f64(Y), _f64(R)
    lo = (ctypes.c_int * 3)(*map(int, lo))
    hi = (ctypes.c_int * 3)(*map(int, hi))
    kc = (ctypes.c_int * 3)(*map(int, k_claim))
    return int(_load().orc_vote_consistent(_pd(X), len(X), _pd(Y), len(Y), _pd(R), delta, lo, hi, band, kc,
                                           int(V_claim)))


def nn_dist(X, Y, R, t) -> np.ndarray:
    X, Y, R, t = _f64(X), _f64(Y), _f64(R), _f64(t)
    d = np.zeros(len(X))
    _load().orc_nn_dist(_pd(X), len(X), _pd(Y), len(Y), _pd(R), _pd(t), _pd(d))
    return d


def inliers(X, Y, R, t, eps, band=1e-5):
    X, Y, R, t = _f64(X), _f64(Y), _f64(R), _f64(t)
    c = ctypes.c_int64()
    nb = ctypes.c_int64()
    _load().orc_inliers(_pd(X), len(X), _pd(Y), len(Y), _pd(R), _pd(t), eps, band, ctypes.byref(c),
                        ctypes.byref(nb))
    return int(c.value), int(nb.value)


def refine_translation(X, Y, R, t, eps, band=1e-5):
    """Mean of the inlier translations y_nn(i) - R x_i at the pose (R, t) (the
    least-squares translation for those correspondences; t when no point is an
    inlier). Returns (t_refined, n_inliers, n_boundary, n_tie)."""
    X, Y, R, t = _f64(X), _f64(Y), _f64(R), _f64(t)
    out = np.zeros(3)
    nb = ctypes.c_int64()
    nt = ctypes.c_int64()
    n = _load().orc_refine_translation(_pd(X), len(X), _pd(Y), len(Y), _pd(R), _pd(t), eps, band, _pd(out),
                                       ctypes.byref(nb), ctypes.byref(nt))
    return out, int(n), int(nb.value), int(nt.value)


def exhaustive(X, Y, rotations, P: Params, rel_tie=1e-4):
    """Algorithm 1 over `rotations` and the lattice translations of P's box:
    returns (cost (n_rot, n_t), inlier count (n_rot, n_t), flat argmin, near_tie)."""
    X, Y = _f64(X), _f64(Y)
    Rl = _f64(np.asarray(rotations).reshape(-1, 9))
    lo, hi = lattice_box(P.t_center[:], P.t_half[:], P.delta_t)
    nt = int(np.prod(np.asarray(hi) - np.asarray(lo) + 1))
    cost = np.zeros((len(Rl), nt))
    cnt = np.zeros((len(Rl), nt), dtype=np.int64)
    tie = ctypes.c_int64()
    best = _load().orc_exhaustive(_pd(X), len(X), _pd(Y), len(Y), _pd(Rl), len(Rl), ctypes.byref(P), _pd(cost),
                                  cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rel_tie, ctypes.byref(tie))
    return cost, cnt, int(best), int(tie.value)


def rho(P: Params, d: float) -> float:
    return float(_load().orc_rho(ctypes.byref(P), d))


def cost_exact(X, Y, R, t, P: Params) -> float:
    X, Y, R, t = _f64(X), _f64(Y), _f64(R), _f64(t)
    return float(_load().orc_cost_exact(_pd(X), len(X), _pd(Y), len(Y), _pd(R), _pd(t), ctypes.byref(P)))


@dataclass
class DistGrid:
    D: np.ndarray  # (G,G,G)
    lo: np.ndarray
    h: np.ndarray
    cap: float

    @property
    def G(self):
        return self.D.shape[0]


def dist_grid(Y, G: int, cap: float, threads: int = 1) -> DistGrid:
    """The target's truncated distance grid; threads > 1 splits its x-planes
    over host threads (the same per-voxel arithmetic)."""
    Y = _f64(Y)
    lo, h = np.zeros(3), np.zeros(3)
    _load().orc_dist_grid_geometry(_pd(Y), len(Y), G, cap, _pd(lo), _pd(h))
    D = np.zeros((G, G, G))
    if threads > 1:
        _load().orc_dist_grid_threads(_pd(Y), len(Y), G, cap, _pd(D), int(threads))
    else:
        _load().orc_dist_grid(_pd(Y), len(Y), G, cap, _pd(D))
    return DistGrid(D=D, lo=lo, h=h, cap=cap)


def grid_lookup(g: DistGrid, p) -> float:
    p = _f64(p)
    return float(_load().orc_grid_lookup(_pd(g.D), g.G, _pd(g.lo), _pd(g.h), g.cap, _pd(p)))


def cost_grid(X, g: DistGrid, R, t, P: Params) -> float:
    X, R, t = _f64(X), _f64(R), _f64(t)
    return float(_load().orc_cost_grid(_pd(X), len(X), _pd(g.D), g.G, _pd(g.lo), _pd(g.h), g.cap, _pd(R), _pd(t),
                                       ctypes.byref(P)))


@dataclass
class Registration:
    status: int
    rot_index: int
    R: np.ndarray
    t: np.ndarray
    votes: int
    inliers: int
    cost: float
    k: np.ndarray | None = None  # per rotation (total, 3)
    V: np.ndarray | None = None
    M: np.ndarray | None = None
    costs: np.ndarray | None = None
    n_boundary_pairs: np.ndarray | None = None
    n_boundary_points: np.ndarray | None = None


def _result(res: Result, **extra) -> Registration:
    return Registration(status=res.status, rot_index=res.rot_index, R=np.array(res.R[:]).reshape(3, 3),
                        t=np.array(res.t[:]), votes=res.votes, inliers=res.inliers, cost=res.cost, **extra)


def register(X, Y, rotations, P: Params, threads: int = 1) -> Registration:
    """Algorithm 2 over an explicit FP64 rotation list with per-rotation outputs;
    threads > 1 fans the rotations over host threads (same arithmetic)."""
    X, Y, Rl = _f64(X), _f64(Y), _f64(rotations)
    nR = len(Rl)
    B = (2 * P.refine_K + 1) ** 3 if P.refine_top_k > 0 else 0
    total = nR + P.refine_top_k * B
    k = np.zeros((total, 3), dtype=np.int32)
    V, Mc = np.zeros(total, dtype=np.int64), np.zeros(total, dtype=np.int64)
    cost = np.zeros(total)
    nbp, nbm = np.zeros(total, dtype=np.int64), np.zeros(total, dtype=np.int64)
    res = Result()
    args = (_pd(X), len(X), _pd(Y), len(Y), _pd(Rl), nR, ctypes.byref(P))
    outs = (k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), V.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            Mc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _pd(cost),
            nbp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), nbm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            ctypes.byref(res))
    if threads > 1:
        _load().orc_register_threads_out(*args, int(threads), *outs)
    else:
        _load().orc_register(*args, *outs)
    return _result(res, k=k, V=V, M=Mc, costs=cost, n_boundary_pairs=nbp, n_boundary_points=nbm)


def register_threads(X, Y, rotations, P: Params, threads: int) -> Registration:
    """Same as register(), fanned over rotations on `threads` host threads (timing only)."""
    X, Y, Rl = _f64(X), _f64(Y), _f64(rotations)
    res = Result()
    _load().orc_register_threads(_pd(X), len(X), _pd(Y), len(Y), _pd(Rl), len(Rl), ctypes.byref(P), threads,
                                 ctypes.byref(res))
    return _result(res)


class Field:
    """A target's distance field built once (the resident-target setting)."""

    def __init__(self, Y, G: int, cap: float, threads: int = 1):
        self.Y = _f64(Y)
        if threads > 1:
            self.h = _load().orc_field_create_threads(_pd(self.Y), len(self.Y), G, cap, int(threads))
        else:
            self.h = _load().orc_field_create(_pd(self.Y), len(self.Y), G, cap)

    def close(self):
        if self.h:
            _load().orc_field_free(self.h)
            self.h = None

    def __del__(self):
        self.close()


def register_field_threads(X, Y, rotations, P: Params, field: Field | None, threads: int) -> Registration:
    """register_threads() reusing a prebuilt distance field (None: metrics that need none)."""
    X, Y, Rl = _f64(X), _f64(Y), _f64(rotations)
    res = Result()
    _load().orc_register_field_threads(_pd(X), len(X), _pd(Y), len(Y), _pd(Rl), len(Rl), ctypes.byref(P),
                                       field.h if field is not None else None, threads, ctypes.byref(res))
    return _result(res)


def eval_rotation(X, Y, R, P: Params):
    """(k*, V, M, boundary pairs, boundary points) of one rotation."""
    X, Y, R = _f64(X), _f64(Y), _f64(R)
    k = (ctypes.c_int * 3)()
    V, Mc, nbp, nbm = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _load().orc_eval_rotation(_pd(X), len(X), _pd(Y), len(Y), _pd(R), ctypes.byref(P), k, ctypes.byref(V),
                              ctypes.byref(Mc), ctypes.byref(nbp), ctypes.byref(nbm))
    return np.array(k[:]), int(V.value), int(Mc.value), int(nbp.value), int(nbm.value)

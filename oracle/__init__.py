"""ctypes front end of the plain CPU oracle (``oracle/mqo_oracle.c``).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and it never calls the CUDA
library.  It shares nothing with the product package except the seeded graph
generators in ``mqo_inputs`` (which hold none of the method's arithmetic).

Every wrapper below runs one graph and one trajectory at a time, exactly as
the C functions document.  Batched helpers simply loop over trajectories.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mqo_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmqo_oracle.so")
_lock = threading.Lock()
_lib = None

MIS, MAXCUT = 0, 1
F_B, F_L, F_P, F_A = 0, 1, 2, 3  # MaxCut relaxations
F32, BF16, F16 = 0, 1, 2
PH_DESCENT, PH_REPAIR, PH_LS, PH_WAIT = 0, 1, 2, 3
EP_DESCENT, EP_LS = 0, 1
INT64_MIN = -(1 << 63)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction of a*b+c into FMA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcGraph(C.Structure):
    _fields_ = [("n", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("w", C.c_void_p)]


class OrcParams(C.Structure):
    _fields_ = [
        ("problem", C.c_int32), ("batch", C.c_int32), ("x_dtype", C.c_int32), ("v_dtype", C.c_int32),
        ("alpha", C.c_float), ("momentum", C.c_float), ("gamma", C.c_float), ("lambda_", C.c_float),
        ("rho", C.c_double), ("sigma", C.c_float), ("t_gs", C.c_int32), ("descent_cap", C.c_int32),
        ("init_kind", C.c_int32), ("local_search", C.c_int32), ("repair", C.c_int32), ("seed", C.c_uint64),
        ("pool_k", C.c_int32), ("objective", C.c_int32),
    ]


class OrcPool(C.Structure):
    _fields_ = [("epoch", C.c_int32), ("count", C.c_int32), ("best", C.c_int64), ("merges", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OrcState(C.Structure):
    _fields_ = [
        ("phase", C.c_int32), ("s", C.c_int32), ("r", C.c_int32), ("o", C.c_int32),
        ("best", C.c_int64), ("ticks", C.c_int64), ("last_round", C.c_int32), ("last_commits", C.c_int64),
        ("ev_value", C.c_int64), ("ev_a", C.c_int64), ("ev_b", C.c_int64),
        ("accepts", C.c_int64), ("descents", C.c_int64), ("held", C.c_int64),
        ("first_value", C.c_int64), ("gain_descent", C.c_int64), ("gain_ls", C.c_int64),
        ("steps", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P = C.c_void_p
            _lib.orc_round_store.restype = C.c_float
            _lib.orc_round_store.argtypes = [C.c_float, C.c_int32]
            _lib.orc_feistel_sigma.restype = C.c_int64
            _lib.orc_feistel_sigma.argtypes = [C.c_int64, P, C.c_int64]
            _lib.orc_reset_count.restype = C.c_int64
            _lib.orc_reset_count.argtypes = [C.c_int64, C.c_double]
            _lib.orc_reset_mask.argtypes = [C.c_int64, C.c_double, C.c_uint64, C.c_int64, C.c_int64, C.c_int64, P]
            _lib.orc_reset_keys.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64, P]
            _lib.orc_philox4x64_10.argtypes = [P, P, P]
            _lib.orc_init_x.argtypes = [P, P, C.c_int64, C.c_int64, P]
            _lib.orc_eval_mis.argtypes = [P, P, P]
            _lib.orc_eval_cut.argtypes = [P, P, P]
            _lib.orc_descent_step.argtypes = [P, P, P, P, P, P, P, P]
            _lib.orc_step_rows.argtypes = [P, P, P, P, P, C.c_int64, P, P]
            for nm in ("orc_round_drop", "orc_round_complete", "orc_round_swap", "orc_round_flip1",
                       "orc_round_flip2"):
                getattr(_lib, nm).restype = C.c_int64
                getattr(_lib, nm).argtypes = [P, P]
            _lib.orc_state_init.argtypes = [P]
            _lib.orc_run_trajectory.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int32, P, P, P, P, P, P, P,
                                                C.c_int64]
            _lib.orc_ls_mis_sequential.restype = C.c_int64
            _lib.orc_ls_mis_sequential.argtypes = [P, P, P]
            _lib.orc_ls_cut_sequential.restype = C.c_int64
            _lib.orc_ls_cut_sequential.argtypes = [P, P]
            _lib.orc_pool_pick.restype = C.c_int64
            _lib.orc_pool_pick.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64, C.c_int64]
            _lib.orc_run_pool.argtypes = [P, P, C.c_int64, C.c_int32, C.c_int64, C.c_int32, P, P, P, P, P, P, P,
                                          P, P]
            _lib.orc_eval_cut_obj.argtypes = [P, P, C.c_int32, C.c_float, P]
            _lib.orc_cut_objective_f64.restype = C.c_double
            _lib.orc_cut_objective_f64.argtypes = [P, C.c_int32, C.c_double, P]
            _lib.orc_cut_gradient_f64.argtypes = [P, C.c_int32, C.c_double, P, P]
            _lib.orc_objective_f64.restype = C.c_double
            _lib.orc_objective_f64.argtypes = [P, C.c_int32, C.c_double, C.c_double, P]
            _lib.orc_gradient_f64.argtypes = [P, C.c_int32, C.c_double, C.c_double, P, P]
            _lib.orc_brute_mis.restype = C.c_int64
            _lib.orc_brute_mis.argtypes = [P]
            _lib.orc_brute_maxcut.restype = C.c_int64
            _lib.orc_brute_maxcut.argtypes = [P]
        return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Graph:
    """Holds contiguous CSR arrays alive for the C side."""

    def __init__(self, g):
        self.n = int(g.n)
        self.row_ptr = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(g.col_idx, dtype=np.int32)
        self.w = None if g.weights is None else np.ascontiguousarray(g.weights, dtype=np.int8)
        self.s = OrcGraph(self.n, _ptr(self.row_ptr).value, _ptr(self.col).value,
                          None if self.w is None else _ptr(self.w).value)

    def ref(self):
        return C.byref(self.s)


def params(problem=MIS, batch=1, x_dtype=F32, v_dtype=F32, alpha=0.8, momentum=0.3, gamma=2.0,
           lambda_=0.001, rho=0.7, sigma=0.1, t_gs=60, descent_cap=50, init_kind=0, local_search=1,
           repair=1, seed=0, pool_k=0, objective=0):
    return OrcParams(problem, batch, x_dtype, v_dtype, alpha, momentum, gamma, lambda_, rho, sigma, t_gs,
                     descent_cap, init_kind, local_search, repair, seed, pool_k, objective)


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def round_store(x: float, dtype: int) -> float:
    return lib().orc_round_store(float(x), int(dtype))


def reset_keys(seed, traj, outer, rnd):
    keys = np.zeros(6, dtype=np.uint32)
    lib().orc_reset_keys(seed, traj, outer, rnd, _ptr(keys))
    return keys


def feistel_sigma(n, keys, v):
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    return lib().orc_feistel_sigma(n, _ptr(keys), v)


def reset_mask(n, rho, seed, traj, outer, rnd):
    m = np.zeros(n, dtype=np.uint8)
    lib().orc_reset_mask(n, rho, seed, traj, outer, rnd, _ptr(m))
    return m


def init_x(g: Graph, p, traj, outer=0):
    x = np.zeros(g.n, dtype=np.float32)
    lib().orc_init_x(g.ref(), C.byref(p), traj, outer, _ptr(x))
    return x


def eval_mis(g: Graph, z):
    """(size, conflicting edges, conflicting nodes, uncovered nodes)"""
    z = np.ascontiguousarray(z, dtype=np.uint8)
    out = np.zeros(4, dtype=np.int64)
    lib().orc_eval_mis(g.ref(), _ptr(z), _ptr(out))
    return tuple(int(v) for v in out)


def eval_cut(g: Graph, z):
    """(cut, non-fixed nodes, 1-flip candidates)"""
    z = np.ascontiguousarray(z, dtype=np.uint8)
    out = np.zeros(4, dtype=np.int64)
    lib().orc_eval_cut(g.ref(), _ptr(z), _ptr(out))
    return tuple(int(v) for v in out[:3])


def eval_cut_obj(g: Graph, z, objective, lambda_):
    """(cut, nodes not fixed under the relaxation's PGA, 1-flip candidates)"""
    z = np.ascontiguousarray(z, dtype=np.uint8)
    out = np.zeros(4, dtype=np.int64)
    lib().orc_eval_cut_obj(g.ref(), _ptr(z), int(objective), float(lambda_), _ptr(out))
    return tuple(int(v) for v in out[:3])


def cut_objective_f64(g: Graph, objective, lambda_, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_cut_objective_f64(g.ref(), int(objective), float(lambda_), _ptr(x))


def cut_gradient_f64(g: Graph, objective, lambda_, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(g.n, dtype=np.float64)
    lib().orc_cut_gradient_f64(g.ref(), int(objective), float(lambda_), _ptr(x), _ptr(out))
    return out


def descent_step(g: Graph, p, x, V):
    x = np.ascontiguousarray(x, dtype=np.float32)
    V = np.ascontiguousarray(V, dtype=np.float32)
    xn = np.zeros_like(x)
    Vn = np.zeros_like(V)
    z = np.zeros(g.n, dtype=np.uint8)
    ev = np.zeros(4, dtype=np.int64)
    lib().orc_descent_step(g.ref(), C.byref(p), _ptr(x), _ptr(V), _ptr(xn), _ptr(Vn), _ptr(z), _ptr(ev))
    return xn, Vn, z, tuple(int(v) for v in ev[:3])


def step_rows(g: Graph, p, x, V, rows):
    x = np.ascontiguousarray(x, dtype=np.float32)
    V = np.ascontiguousarray(V, dtype=np.float32)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    xn = np.zeros(len(rows), dtype=np.float32)
    Vn = np.zeros(len(rows), dtype=np.float32)
    lib().orc_step_rows(g.ref(), C.byref(p), _ptr(x), _ptr(V), _ptr(rows), len(rows), _ptr(xn), _ptr(Vn))
    return xn, Vn


def _round(name, g: Graph, z):
    z = np.array(z, dtype=np.uint8, copy=True)
    k = getattr(lib(), name)(g.ref(), _ptr(z))
    return z, int(k)


def round_drop(g, z):
    return _round("orc_round_drop", g, z)


def round_complete(g, z):
    return _round("orc_round_complete", g, z)


def round_swap(g, z):
    return _round("orc_round_swap", g, z)


def round_flip1(g, z):
    return _round("orc_round_flip1", g, z)


def round_flip2(g, z):
    return _round("orc_round_flip2", g, z)


class Trajectory:
    """One trajectory of the tick machine; ``run(k)`` advances it k ticks."""

    def __init__(self, g: Graph, p, traj: int):
        self.g, self.p, self.traj = g, p, int(traj)
        n = g.n
        self.st = OrcState()
        self.x = np.zeros(n, dtype=np.float32)
        self.V = np.zeros(n, dtype=np.float32)
        self.zbest = np.zeros(n, dtype=np.uint8)
        self.zwork = np.zeros(n, dtype=np.uint8)
        self.zx_prev = np.zeros(n, dtype=np.uint8)
        self.started = False

    def run(self, nticks: int, trace_ticks: int = 0):
        tr = np.zeros((trace_ticks, self.g.n), dtype=np.float32) if trace_ticks else None
        lib().orc_run_trajectory(self.g.ref(), C.byref(self.p), self.traj, int(nticks), int(self.started),
                                 C.byref(self.st), _ptr(self.x), _ptr(self.V), _ptr(self.zbest),
                                 _ptr(self.zwork), _ptr(self.zx_prev), _ptr(tr), int(trace_ticks))
        self.started = True
        return tr

    @property
    def state(self):
        return self.st.as_dict()


def ls_mis_sequential(g: Graph, z):
    """OneTwoSwap in the paper's scan order; returns (z, swaps, adds)."""
    z = np.ascontiguousarray(z, dtype=np.uint8).copy()
    adds = C.c_int64()
    k = lib().orc_ls_mis_sequential(g.ref(), _ptr(z), C.byref(adds))
    return z, int(k), adds.value


def ls_cut_sequential(g: Graph, z):
    """OneTwoFlip in the paper's scan order; returns (z, moves)."""
    z = np.ascontiguousarray(z, dtype=np.uint8).copy()
    k = lib().orc_ls_cut_sequential(g.ref(), _ptr(z))
    return z, int(k)


def pool_pick(seed, traj, outer, rnd, count):
    return int(lib().orc_pool_pick(seed, traj, outer, rnd, count))


class PoolGraph:
    """The B trajectories of one graph in pool mode (pmQO, Alg. 3/4);
    trajectory ids traj0 .. traj0+B-1; ``run(k)`` advances them k ticks."""

    def __init__(self, g: Graph, p, traj0: int, B: int):
        self.g, self.p, self.traj0, self.B = g, p, int(traj0), int(B)
        n, K = g.n, max(1, int(p.pool_k))
        self.st = (OrcState * B)()
        self.x = np.zeros((B, n), dtype=np.float32)
        self.V = np.zeros((B, n), dtype=np.float32)
        self.zbest = np.zeros((B, n), dtype=np.uint8)
        self.zwork = np.zeros((B, n), dtype=np.uint8)
        self.zx_prev = np.zeros((B, n), dtype=np.uint8)
        self.pool = OrcPool()
        self.pool_bits = np.zeros((K, n), dtype=np.uint8)
        self.pool_vals = np.zeros(K, dtype=np.int64)
        self.started = False

    def run(self, nticks: int):
        lib().orc_run_pool(self.g.ref(), C.byref(self.p), self.traj0, self.B, int(nticks), int(self.started),
                           self.st, _ptr(self.x), _ptr(self.V), _ptr(self.zbest), _ptr(self.zwork),
                           _ptr(self.zx_prev), C.byref(self.pool), _ptr(self.pool_bits), _ptr(self.pool_vals))
        self.started = True

    def state(self, b):
        return self.st[b].as_dict()

    def members(self):
        """(values, bits) of the pool members, best first"""
        c = self.pool.count
        return self.pool_vals[:c].copy(), self.pool_bits[:c].copy()


def objective_f64(g: Graph, problem, gamma, lambda_, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_objective_f64(g.ref(), problem, gamma, lambda_, _ptr(x))


def gradient_f64(g: Graph, problem, gamma, lambda_, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(g.n, dtype=np.float64)
    lib().orc_gradient_f64(g.ref(), problem, gamma, lambda_, _ptr(x), _ptr(out))
    return out


def brute_mis(g: Graph) -> int:
    assert g.n <= 26
    return int(lib().orc_brute_mis(g.ref()))


def brute_maxcut(g: Graph) -> int:
    assert g.n <= 26
    return int(lib().orc_brute_maxcut(g.ref()))

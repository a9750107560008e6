"""Python binding of the mQO GB300 library (``_build/libmqo.so``, C ABI in include/mqo.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  PyTorch provides device memory (tensors) and the current CUDA
stream.  Importing this package loads the compiled library and raises
``ImportError`` if it is missing and cannot be built; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "MqoError", "Params", "TrajInfo", "Graph", "Solver", "params", "lib", "fb_forward", "spmm_grad",
    "pga_momentum_step", "pga_adam_step", "FbObjective", "PGAMomentum", "PGAAdam",
    "MIS", "MAXCUT", "F32", "BF16", "F16", "OBJ_FB", "OBJ_FL", "OBJ_FP", "OBJ_FA",
]

MIS, MAXCUT = 0, 1
F32, BF16, F16 = 0, 1, 2
OBJ_FB, OBJ_FL, OBJ_FP, OBJ_FA = 0, 1, 2, 3
INT64_MIN = -(1 << 63)
_STATUS = {0: "MQO_OK", -1: "MQO_EINVAL", -2: "MQO_EGRAPH", -3: "MQO_ENOMEM", -4: "MQO_ECUDA",
           -5: "MQO_ETIMEOUT", -6: "MQO_ESTATE"}


class MqoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("problem", C.c_int32), ("batch", C.c_int32), ("x_dtype", C.c_int32), ("v_dtype", C.c_int32),
        ("alpha", C.c_float), ("momentum", C.c_float), ("gamma", C.c_float), ("lambda_", C.c_float),
        ("rho", C.c_double), ("sigma", C.c_float), ("t_gs", C.c_int32), ("descent_cap", C.c_int32),
        ("init_kind", C.c_int32), ("local_search", C.c_int32), ("repair", C.c_int32), ("seed", C.c_uint64),
        ("objective", C.c_int32), ("pool_k", C.c_int32),
    ]


def _plan(p):
    """Decode the plan word of mqo_solver_info / mqo_autotune."""
    if p & 1:
        kern = "smem_wide" if p & 4 else "smem"
    else:
        kern = "staged" if p & 8 else "global"
    return {"step_kernel": kern, "discrete_kernel": "graph" if p & 2 else "pairs", "lanes_vec": (p >> 4) & 15,
            "slice_kb": (p >> 8) & 255, "col16": bool(p & (1 << 16)), "ell": bool(p & (1 << 17))}


class TrajInfo(C.Structure):
    _fields_ = [
        ("phase", C.c_int32), ("s", C.c_int32), ("r", C.c_int32), ("o", C.c_int32),
        ("best", C.c_int64), ("ticks", C.c_int64), ("last_round", C.c_int32), ("pad0", C.c_int32),
        ("last_commits", C.c_int64), ("ev_value", C.c_int64), ("ev_a", C.c_int64), ("ev_b", C.c_int64),
        ("accepts", C.c_int64), ("descents", C.c_int64), ("held", C.c_int64),
        ("first_value", C.c_int64), ("gain_descent", C.c_int64), ("gain_ls", C.c_int64),
        ("steps", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad0"}


def params(problem=MIS, batch=1, x_dtype=F32, v_dtype=None, alpha=0.8, momentum=0.3, gamma=2.0, lambda_=0.001,
           rho=0.7, sigma=0.1, t_gs=60, descent_cap=50, init_kind=0, local_search=1, repair=1, seed=0,
           objective=0, pool_k=0) -> Params:
    if v_dtype is None:
        v_dtype = x_dtype
    return Params(problem, batch, x_dtype, v_dtype, alpha, momentum, gamma, lambda_, rho, sigma, t_gs,
                  descent_cap, init_kind, local_search, repair, seed, objective, pool_k)


_lib = None

# (name, argtypes) of every entry point declared in include/mqo.h
_P = C.c_void_p
_SIGS = {
    "mqo_graph_create_csr": [C.c_int64, C.c_int64, _P, _P, _P, C.c_int32, _P, _P],
    "mqo_graph_create_packed": [C.c_int32, _P, C.c_int64, _P, _P, _P, C.c_int32, _P, _P],
    "mqo_graph_destroy": [_P],
    "mqo_graph_info": [_P, _P, _P, _P],
    "mqo_solver_create": [_P, _P, _P, _P],
    "mqo_solver_destroy": [_P],
    "mqo_init": [_P],
    "mqo_step": [_P, C.c_int32],
    "mqo_step_stats": [_P, _P, _P, _P],
    "mqo_run": [_P, C.c_int64],
    "mqo_reset": [_P, _P],
    "mqo_round": [_P, _P],
    "mqo_evaluate": [_P, _P, _P, _P, _P],
    "mqo_local_search": [_P, C.c_int32],
    "mqo_solve": [_P, C.c_int64],
    "mqo_run_timed": [_P, C.c_int64, _P, _P],
    "mqo_best": [_P, _P, _P],
    "mqo_traj_state": [_P, _P],
    "mqo_pool_state": [_P, _P, _P, _P, _P],
    "mqo_solver_info": [_P, _P, _P, _P, _P],
    "mqo_autotune": [_P, C.c_int32, _P, _P],
    "mqo_get_x": [_P, _P],
    "mqo_set_x": [_P, _P],
    "mqo_get_v": [_P, _P],
    "mqo_objective_f64": [_P, _P],
    "mqo_fb_forward": [_P, _P, C.c_int32, C.c_float, _P, _P],
    "mqo_spmm_grad": [_P, _P, _P, _P, C.c_int32, C.c_float, _P],
    "mqo_spmm_grad_static": [_P, _P, _P, _P, C.c_int32, C.c_float, _P],
    "mqo_pga_momentum_step": [_P, _P, _P, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float, _P],
    "mqo_pga_adam_step": [_P, _P, _P, _P, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int64,
                          C.c_float, C.c_float, _P],
    "mqo_measure_smem_gbs": [C.c_int32, _P],
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if needed) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            try:
                path = _build.build()
            except Exception as e:  # no silent fallback: the library is the product
                raise ImportError(f"mQO CUDA library missing and could not be built: {e}") from e
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.mqo_last_error.restype = C.c_char_p
        L.mqo_last_error.argtypes = []
        L.mqo_version.restype = C.c_char_p
        L.mqo_version.argtypes = []
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise MqoError(status, lib().mqo_last_error().decode())


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _hptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Graph:
    """Device copy of a symmetric CSR graph (or a packed batch of graphs).

    ``g`` is any object with ``n``, ``row_ptr``, ``col_idx``, ``weights`` and
    ``node_offsets`` (e.g. ``mqo_inputs.Graph``); host arrays are validated by
    the library and deep-copied.
    """

    def __init__(self, g, stream=None):
        self.handle = C.c_void_p()
        rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(g.col_idx, dtype=np.int32)
        w = None if g.weights is None else np.ascontiguousarray(g.weights, dtype=np.int8)
        offs = getattr(g, "node_offsets", None)
        s = _stream(stream)
        if offs is not None and len(offs) > 2:
            offs = np.ascontiguousarray(offs, dtype=np.int64)
            _check(lib().mqo_graph_create_packed(len(offs) - 1, _hptr(offs), int(rp[-1]), _hptr(rp), _hptr(col),
                                                 _hptr(w), 0, s, C.byref(self.handle)))
        else:
            _check(lib().mqo_graph_create_csr(int(g.n), int(rp[-1]), _hptr(rp), _hptr(col), _hptr(w), 0, s,
                                              C.byref(self.handle)))
        n, nnz, ng = C.c_int64(), C.c_int64(), C.c_int32()
        _check(lib().mqo_graph_info(self.handle, C.byref(n), C.byref(nnz), C.byref(ng)))
        self.n, self.nnz, self.num_graphs = n.value, nnz.value, ng.value

    def close(self):
        if self.handle:
            _check(lib().mqo_graph_destroy(self.handle))
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_TORCH_DT = {F32: "float32", BF16: "bfloat16", F16: "float16"}


class Solver:
    """B trajectories per member graph of the mQO machine on one GPU."""

    def __init__(self, graph: Graph, p: Params, stream=None):
        import torch
        self.graph = graph
        self.p = p
        self.B = p.batch
        self.T = graph.num_graphs * p.batch
        self.Bw = (p.batch + 31) // 32
        self.handle = C.c_void_p()
        self._torch = torch
        _check(lib().mqo_solver_create(graph.handle, C.byref(p), _stream(stream), C.byref(self.handle)))

    def close(self):
        if self.handle:
            _check(lib().mqo_solver_destroy(self.handle))
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- thin wrappers
    def init(self):
        _check(lib().mqo_init(self.handle))

    def step(self, nsteps=1):
        _check(lib().mqo_step(self.handle, int(nsteps)))

    def run(self, nticks):
        _check(lib().mqo_run(self.handle, int(nticks)))

    PHASES = ("ctrl", "apply", "step", "disc_a", "disc_b", "disc_c", "tick_end")

    def run_timed(self, nticks):
        """Run nticks ticks kernel by kernel; returns ({phase: summed ms}, kernel launches)."""
        ms = (C.c_double * 7)()
        k = C.c_int64()
        _check(lib().mqo_run_timed(self.handle, int(nticks), ms, C.byref(k)))
        return dict(zip(self.PHASES, list(ms))), k.value

    def solve(self, nticks):
        _check(lib().mqo_solve(self.handle, int(nticks)))

    def reset(self, mask=None):
        _check(lib().mqo_reset(self.handle, _dptr(mask)))

    def local_search(self, max_rounds=1 << 20):
        _check(lib().mqo_local_search(self.handle, int(max_rounds)))

    def _i64(self):
        return self._torch.empty(self.T, dtype=self._torch.int64, device="cuda")

    def step_stats(self):
        v, a, b = self._i64(), self._i64(), self._i64()
        _check(lib().mqo_step_stats(self.handle, _dptr(v), _dptr(a), _dptr(b)))
        return v, a, b

    def bits_tensor(self):
        return self._torch.zeros(self.graph.n * self.Bw, dtype=self._torch.int32, device="cuda")

    def round(self, out=None):
        out = self.bits_tensor() if out is None else out
        _check(lib().mqo_round(self.handle, _dptr(out)))
        return out

    def evaluate(self, bits):
        v, a, b = self._i64(), self._i64(), self._i64()
        _check(lib().mqo_evaluate(self.handle, _dptr(bits), _dptr(v), _dptr(a), _dptr(b)))
        return v, a, b

    def best(self, want_bits=True):
        vals = np.zeros(self.T, dtype=np.int64)
        bits = self.bits_tensor() if want_bits else None
        _check(lib().mqo_best(self.handle, _hptr(vals), _dptr(bits)))
        return vals, bits

    def info(self):
        """Execution plan: step kernel (smem, smem_wide, staged or global), discrete kernel, trajectories per
        lane, KB of gathered rows per staged slice, smem bytes, items, counter replicas."""
        k, sm, it, r = C.c_int32(), C.c_int64(), C.c_int32(), C.c_int32()
        _check(lib().mqo_solver_info(self.handle, C.byref(k), C.byref(sm), C.byref(it), C.byref(r)))
        return dict(_plan(k.value), smem_bytes=sm.value, items=it.value, replicas=r.value)

    def autotune(self, ticks=10):
        """Time every launch plan over `ticks` ticks (state restored after each) and keep the fastest."""
        plan, ms = C.c_int32(), C.c_double()
        _check(lib().mqo_autotune(self.handle, int(ticks), C.byref(plan), C.byref(ms)))
        return dict(_plan(plan.value), ms_per_tick=ms.value)

    def pool_state(self):
        """Pool mode: (counts [G], values [G, K], merges [G]) on the host and the
        members' bits (device words, n * ceil(K/32))."""
        K = self.p.pool_k
        G = self.graph.num_graphs
        counts = np.zeros(G, dtype=np.int32)
        values = np.zeros(G * K, dtype=np.int64)
        merges = np.zeros(G, dtype=np.int64)
        bits = self._torch.zeros(self.graph.n * ((K + 31) // 32), dtype=self._torch.int32, device="cuda")
        _check(lib().mqo_pool_state(self.handle, _hptr(counts), _hptr(values), _hptr(merges), _dptr(bits)))
        return counts, values.reshape(G, K), merges, bits

    def traj_state(self):
        arr = (TrajInfo * self.T)()
        _check(lib().mqo_traj_state(self.handle, arr))
        return [a.as_dict() for a in arr]

    def steps_taken(self):
        """Descent steps taken so far by every trajectory (int64 array [T])."""
        arr = (TrajInfo * self.T)()
        _check(lib().mqo_traj_state(self.handle, arr))
        return np.array([a.steps for a in arr], dtype=np.int64)

    def get_x(self):
        t = self._torch.empty(self.graph.n * self.B, dtype=getattr(self._torch, _TORCH_DT[self.p.x_dtype]),
                              device="cuda")
        _check(lib().mqo_get_x(self.handle, _dptr(t)))
        return t.view(self.graph.n, self.B)

    def get_v(self):
        t = self._torch.empty(self.graph.n * self.B, dtype=getattr(self._torch, _TORCH_DT[self.p.v_dtype]),
                              device="cuda")
        _check(lib().mqo_get_v(self.handle, _dptr(t)))
        return t.view(self.graph.n, self.B)

    def set_x(self, x):
        x = x.contiguous()
        _check(lib().mqo_set_x(self.handle, _dptr(x)))

    def objective_f64(self):
        out = self._torch.empty(self.T, dtype=self._torch.float64, device="cuda")
        _check(lib().mqo_objective_f64(self.handle, _dptr(out)))
        return out


def unpack_bits(bits, n: int, B: int):
    """Node-major bit words -> (n, B) uint8 numpy array (host helper)."""
    w = np.asarray(bits.cpu().numpy() if hasattr(bits, "cpu") else bits).view(np.uint32)
    Bw = (B + 31) // 32
    w = w.reshape(n, Bw)
    b = np.arange(B)
    return ((w[:, b // 32] >> (b % 32).astype(np.uint32)) & 1).astype(np.uint8)


def pack_bits(z, B: int):
    """(n, B) 0/1 array -> node-major uint32 words as int32 numpy array."""
    z = np.asarray(z, dtype=np.uint32)
    n = z.shape[0]
    Bw = (B + 31) // 32
    out = np.zeros((n, Bw), dtype=np.uint32)
    for b in range(B):
        out[:, b // 32] |= z[:, b] << np.uint32(b % 32)
    return out.reshape(-1).view(np.int32)


# ---------------------------------------------------------------- graph-level kernels
def fb_forward(graph: Graph, X, lambda_: float):
    """f_B per column of a float32 (n, B) CUDA tensor, as a float64 tensor [B]."""
    import torch
    X = X.contiguous()
    B = X.shape[1]
    out = torch.empty(B, dtype=torch.float64, device=X.device)
    _check(lib().mqo_fb_forward(graph.handle, _dptr(X), B, float(lambda_), _dptr(out), _stream()))
    return out


def spmm_grad(graph: Graph, X, lambda_: float, gout=None):
    """gout[b] * (-lambda - 2 A X) as a float32 (n, B) tensor."""
    import torch
    X = X.contiguous()
    B = X.shape[1]
    G = torch.empty_like(X)
    g = None if gout is None else gout.to(torch.float32).contiguous()
    _check(lib().mqo_spmm_grad(graph.handle, _dptr(X), _dptr(g), _dptr(G), B, float(lambda_), _stream()))
    return G


def spmm_grad_static(graph: Graph, X, lambda_: float, gout=None, out=None):
    """As spmm_grad, through the allocation-free entry point: the library
    allocates nothing (partial sums go to its static scratch array), and the
    output tensor may be passed in by a caller that manages its own memory."""
    import torch
    X = X.contiguous()
    B = X.shape[1]
    G = torch.empty_like(X) if out is None else out
    g = None if gout is None else gout.to(torch.float32).contiguous()
    _check(lib().mqo_spmm_grad_static(graph.handle, _dptr(X), _dptr(g), _dptr(G), B, float(lambda_), _stream()))
    return G


def measure_smem_gbs(iters: int = 4096) -> float:
    """Measured shared-memory load bandwidth of the current device, GB/s."""
    out = C.c_double(0.0)
    _check(lib().mqo_measure_smem_gbs(int(iters), C.byref(out)))
    return out.value


def pga_momentum_step(x, v, grad, lr, mu, lo, hi):
    _check(lib().mqo_pga_momentum_step(_dptr(x), _dptr(v), _dptr(grad), x.numel(), float(lr), float(mu), float(lo),
                                       float(hi), _stream()))


def pga_adam_step(x, m, u, grad, lr, b1, b2, eps, t, lo, hi):
    _check(lib().mqo_pga_adam_step(_dptr(x), _dptr(m), _dptr(u), _dptr(grad), x.numel(), float(lr), float(b1),
                                   float(b2), float(eps), int(t), float(lo), float(hi), _stream()))


def _autograd():
    import torch

    class FbObjective(torch.autograd.Function):
        """f_B(X) per column (Eq. 7) with the fused SpMM gradient as backward."""

        @staticmethod
        def forward(ctx, X, graph, lambda_):
            ctx.graph, ctx.lambda_ = graph, lambda_
            ctx.save_for_backward(X)
            return fb_forward(graph, X.detach(), lambda_)

        @staticmethod
        def backward(ctx, gout):
            (X,) = ctx.saved_tensors
            return spmm_grad(ctx.graph, X.detach(), ctx.lambda_, gout), None, None

    class PGAMomentum(torch.optim.Optimizer):
        """Projected momentum ascent on p.grad: v <- mu v + g, p <- Pi(p + lr v)."""

        def __init__(self, params, lr, momentum, lo=-1.0, hi=1.0):
            super().__init__(params, dict(lr=lr, momentum=momentum, lo=lo, hi=hi))

        @torch.no_grad()
        def step(self, closure=None):
            for grp in self.param_groups:
                for p in grp["params"]:
                    if p.grad is None:
                        continue
                    st = self.state[p]
                    if "v" not in st:
                        st["v"] = torch.zeros_like(p)
                    pga_momentum_step(p, st["v"], p.grad.contiguous(), grp["lr"], grp["momentum"], grp["lo"],
                                      grp["hi"])

    class PGAAdam(torch.optim.Optimizer):
        """Projected Adam ascent on p.grad (bias-corrected moments)."""

        def __init__(self, params, lr, betas=(0.9, 0.999), eps=1e-8, lo=-1.0, hi=1.0):
            super().__init__(params, dict(lr=lr, betas=betas, eps=eps, lo=lo, hi=hi))

        @torch.no_grad()
        def step(self, closure=None):
            for grp in self.param_groups:
                for p in grp["params"]:
                    if p.grad is None:
                        continue
                    st = self.state[p]
                    if "m" not in st:
                        st["m"] = torch.zeros_like(p)
                        st["u"] = torch.zeros_like(p)
                        st["t"] = 0
                    st["t"] += 1
                    b1, b2 = grp["betas"]
                    pga_adam_step(p, st["m"], st["u"], p.grad.contiguous(), grp["lr"], b1, b2, grp["eps"], st["t"],
                                  grp["lo"], grp["hi"])

    return FbObjective, PGAMomentum, PGAAdam


def __getattr__(name):
    if name in ("FbObjective", "PGAMomentum", "PGAAdam"):
        fo, pm, pa = _autograd()
        globals().update(FbObjective=fo, PGAMomentum=pm, PGAAdam=pa)
        return globals()[name]
    raise AttributeError(name)


lib()

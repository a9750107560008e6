"""The allocation-free gradient entry point (mqo_spmm_grad_static).

Some callers cannot allocate device memory during a call: applications whose
device memory is held by their own pool or caching allocator, and loops that
must not pay for cudaMalloc / cudaFree (which can synchronise the device).
They use mqo_spmm_grad_static, whose scratch is a static 4 MiB device array
inside the library.  Its output must equal mqo_spmm_grad's bit for bit (both
add every row in CSR order and the partial sums of rows longer than 512
entries in chunk order), on two calls in a row (the array keeps the previous
call's contents), through the C ABI, unweighted and with +-1 edge weights,
and agree with the oracle's float64 gradient.  This file is collected last
so a stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import mqo_inputs as mi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mq():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2605_06921_gb300 as m
    return m


def graph_with_long_rows(signed):
    cl = mi.chung_lu(30000, 2.5, 8.0, 3)
    hub = mi.from_edges(2501, np.zeros(2500, int), np.arange(1, 2501))
    G = mi.pack([cl, hub])
    if not signed:
        return mi.Graph(G.n, G.row_ptr, G.col_idx, None)
    rows, cols = G.edges_directed()
    up = rows < cols
    w = np.random.default_rng(7).choice(np.array([-1, 1], dtype=np.int8), size=int(up.sum()))
    return mi.from_edges(G.n, rows[up], cols[up], w)


def call_static(mq, g, X, gout, lam, out):
    lib = mq.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mqo_spmm_grad_static(g.handle, ctypes.c_void_p(X.data_ptr()),
                                  None if gout is None else ctypes.c_void_p(gout.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), X.shape[1], ctypes.c_float(lam), stream)
    assert st == 0, lib.mqo_last_error()


@pytest.mark.parametrize("B,signed", [(8, False), (64, False), (32, True)])
def test_static_matches_allocating_entry_point_twice(mq, B, signed):
    G = graph_with_long_rows(signed)
    assert (np.diff(G.row_ptr) > 512).sum() >= 2
    g = mq.Graph(G)
    rng = np.random.default_rng(B)
    lam = 0.001
    for call in range(2):
        X = torch.from_numpy((rng.random((G.n, B)) * 2 - 1).astype(np.float32)).cuda()
        gout = torch.linspace(0.5, 1.5, B, device="cuda") if call else None
        want = mq.spmm_grad(g, X, lam, gout)
        out = torch.full_like(X, float("nan"))
        call_static(mq, g, X, gout, lam, out)
        torch.cuda.synchronize()
        assert torch.equal(out, want), call


def test_static_matches_the_oracle_gradient(mq):
    """-lambda - 2 A x per column against the oracle's float64 gradient, within
    the float32 rounding of a sum in CSR order: |err| <= 1e-5 (lambda + 2 sum |x_u|)."""
    import oracle
    G = graph_with_long_rows(True)
    g = mq.Graph(G)
    og = oracle.Graph(G)
    B, lam = 8, 0.001
    Xh = (np.random.default_rng(3).random((G.n, B)) * 2 - 1).astype(np.float32)
    out = torch.empty((G.n, B), device="cuda")
    call_static(mq, g, torch.from_numpy(Xh).cuda(), None, lam, out)
    got = out.cpu().numpy().astype(np.float64)
    deg = np.diff(G.row_ptr)
    rows = np.repeat(np.arange(G.n), deg)
    for b in range(B):
        want = oracle.gradient_f64(og, oracle.MAXCUT, 2.0, lam, Xh[:, b].astype(np.float64))
        absum = np.bincount(rows, weights=np.abs(Xh[G.col_idx, b].astype(np.float64)), minlength=G.n)
        assert np.all(np.abs(got[:, b] - want) <= 1e-5 * (lam + 2 * absum) + 1e-7), b


def test_static_rejects_oversized_requests(mq):
    """More long-row chunks than the static array holds: a clear error, no launch."""
    stars = [mi.from_edges(300001, np.zeros(300000, int), np.arange(1, 300001)) for _ in range(8)]
    P = mi.pack(stars)
    G = mi.Graph(P.n, P.row_ptr, P.col_idx, None)
    g = mq.Graph(G)
    B = 256
    X = torch.zeros((1, B), device="cuda")  # never read: the size check fails first
    lib = mq.lib()
    st = lib.mqo_spmm_grad_static(g.handle, ctypes.c_void_p(X.data_ptr()), None, ctypes.c_void_p(X.data_ptr()), B,
                                  ctypes.c_float(0.001), None)
    assert st == -1
    assert b"static scratch holds" in lib.mqo_last_error()

"""The allocation-free gradient entry point (mqo_spmm_grad_static).

Callers that cannot allocate device memory during a call (work issued while
a stream is captured into a CUDA graph, memory held by the caller's own
pool, allocation-free loops) use mqo_spmm_grad_static, whose scratch is a
static 4 MiB device array.  Its output must match mqo_spmm_grad's, on two
calls in a row (the array keeps the previous call's contents), through the
C ABI.  This file is collected last so a stop-at-first-failure run has
already run every other test.
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


def graph_with_long_rows():
    cl = mi.chung_lu(30000, 2.5, 8.0, 3)
    hub = mi.from_edges(2501, np.zeros(2500, int), np.arange(1, 2501))
    G = mi.pack([cl, hub])
    return mi.Graph(G.n, G.row_ptr, G.col_idx, None)


@pytest.mark.parametrize("B", [8, 64])
def test_static_matches_allocating_entry_point_twice(mq, B):
    G = graph_with_long_rows()
    assert (np.diff(G.row_ptr) > 512).sum() >= 2
    g = mq.Graph(G)
    rng = np.random.default_rng(B)
    lib = mq.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lam = 0.001
    for call in range(2):
        X = torch.from_numpy((rng.random((G.n, B)) * 2 - 1).astype(np.float32)).cuda()
        gout = torch.linspace(0.5, 1.5, B, device="cuda") if call else None
        want = mq.spmm_grad(g, X, lam, gout)
        out = torch.full_like(X, float("nan"))
        st = lib.mqo_spmm_grad_static(g.handle, ctypes.c_void_p(X.data_ptr()),
                                      None if gout is None else ctypes.c_void_p(gout.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), B, ctypes.c_float(lam), stream)
        assert st == 0, lib.mqo_last_error()
        torch.cuda.synchronize()
        assert torch.allclose(out, want, rtol=1e-5, atol=1e-4), call


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

"""Graph creation on a GPU machine: the entry checks run on the device and report
the same errors as the host checks (mqo_graph_create_csr / _packed), from
host or device arrays; valid graphs pass."""
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


def _create(mq, rp, col, w=None, offs=None, device=False):
    lib = mq.lib()
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.int8)
    keep = []
    if device:
        ts = [torch.from_numpy(a).cuda() for a in (rp, col) + ((w,) if w is not None else ())]
        keep += ts
        prp, pcol = ctypes.c_void_p(ts[0].data_ptr()), ctypes.c_void_p(ts[1].data_ptr())
        pw = ctypes.c_void_p(ts[2].data_ptr()) if w is not None else None
    else:
        prp, pcol = rp.ctypes.data_as(ctypes.c_void_p), col.ctypes.data_as(ctypes.c_void_p)
        pw = None if w is None else w.ctypes.data_as(ctypes.c_void_p)
    n = len(rp) - 1
    if offs is None:
        st = lib.mqo_graph_create_csr(n, len(col), prp, pcol, pw, int(device), None, ctypes.byref(h))
    else:
        o = np.ascontiguousarray(offs, dtype=np.int64)
        st = lib.mqo_graph_create_packed(len(o) - 1, o.ctypes.data_as(ctypes.c_void_p), len(col), prp, pcol, pw,
                                         int(device), None, ctypes.byref(h))
    msg = lib.mqo_last_error()
    if st == 0:
        lib.mqo_graph_destroy(h)
    return st, msg


@pytest.mark.parametrize("device", [False, True])
def test_device_checks_report_the_host_messages(mq, device):
    cases = [
        (([0, 1, 1], [1]), b"reverse"),                        # 0->1 without 1->0
        (([0, 1, 2], [0, 0]), b"self loop"),
        (([0, 2, 3, 4], [2, 1, 0, 0]), b"not strictly ascending"),
        (([0, 1, 2], [5, 0]), b"out of range"),
    ]
    for (rp, col), want in cases:
        st, msg = _create(mq, rp, col, device=device)
        assert st == -2 and want in msg, (rp, col, msg)
    st, msg = _create(mq, [0, 1, 2], [1, 0], w=[1, -1], device=device)   # asymmetric weight
    assert st == -2 and b"not symmetric" in msg
    st, msg = _create(mq, [0, 1, 2], [1, 0], w=[3, 3], device=device)    # weight outside {-1,+1}
    assert st == -2 and b"not in {-1,+1}" in msg
    st, msg = _create(mq, [0, 1, 2, 2], [1, 0], offs=[0, 1, 3], device=device)  # edge across member graphs
    assert st == -2 and b"joins two member graphs" in msg


@pytest.mark.parametrize("device", [False, True])
def test_smallest_bad_row_is_reported(mq, device):
    """Delete the reverse entries (b, a) of two edges (a, b), a < b: rows a
    are then the only bad rows, and the smaller one is reported."""
    G = mi.erdos_renyi(3000, 0.01, 1)
    rp, col = G.row_ptr, G.col_idx
    edges = []
    for a in (2100, 1700):
        b = int(next(u for u in col[rp[a]:rp[a + 1]] if u > a))
        edges.append((a, b))
    drop = np.zeros(len(col), dtype=bool)
    for a, b in edges:
        row = col[rp[b]:rp[b + 1]]
        drop[rp[b] + int(np.searchsorted(row, a))] = True
    keep = ~drop
    counts = np.diff(rp) - np.add.reduceat(drop.astype(np.int64), rp[:-1])
    new_rp = np.concatenate([[0], np.cumsum(counts)])
    st, msg = _create(mq, new_rp, col[keep], device=device)
    a, b = min(edges)
    assert st == -2 and f"edge ({a},{b}) has no reverse entry".encode() in msg, msg


@pytest.mark.parametrize("device", [False, True])
def test_valid_graphs_pass(mq, device):
    for G in (mi.erdos_renyi(500, 0.05, 2), mi.random_regular(300, 3, 3),
              mi.pack([mi.erdos_renyi(100, 0.1, 4), mi.erdos_renyi(80, 0.2, 5)])):
        offs = G.node_offsets if G.node_offsets is not None and len(G.node_offsets) > 2 else None
        st, msg = _create(mq, G.row_ptr, G.col_idx, offs=offs, device=device)
        assert st == 0, msg

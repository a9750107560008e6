"""Row partition of one graph over several ranks and its halo exchange (CPU).

The plan must cover every row exactly once, map every local entry back to
its global neighbour in the global CSR order, and pair every rank's ghost
rows with the rows their owners send; float32 row sums over the local CSR
(own rows plus ghosts) must equal the global ones bit for bit.  The halo
exchange runs on two gloo ranks.
"""
import os
import socket

import numpy as np
import pytest

import mqo_inputs as mi
from paper_2605_06921_gb300 import partition as pt

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def graphs():
    yield mi.erdos_renyi(300, 0.04, 1)
    yield mi.chung_lu(2000, 2.5, 6.0, 2)
    G = mi.random_regular(500, 3, 3, signed_weights=True)
    yield G
    yield mi.from_edges(50, np.zeros(49, int), np.arange(1, 50))  # one hub row


def global_of(part, j):
    u = part.col_local[j]
    return u + part.row0 if u < part.n_own else part.halo[u - part.n_own]


@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_plan_covers_rows_and_maps_entries_back(P):
    for G in graphs():
        parts = pt.plan(G, P)
        assert parts[0].row0 == 0 and parts[-1].row1 == G.n
        for a, b in zip(parts, parts[1:]):
            assert a.row1 == b.row0
        nnz = [int(p.row_ptr[-1]) for p in parts]
        assert sum(nnz) == G.nnz
        if P > 1 and G.nnz > 100 * P:
            assert max(nnz) <= 1.6 * G.nnz / P + np.diff(G.row_ptr).max()
        for p in parts:
            for v in range(p.row0, p.row1):
                lo, hi = p.row_ptr[v - p.row0], p.row_ptr[v - p.row0 + 1]
                got = np.array([global_of(p, j) for j in range(lo, hi)], dtype=np.int64)
                want = G.col_idx[G.row_ptr[v]:G.row_ptr[v + 1]]
                assert np.array_equal(got, want)  # same neighbours, same (global CSR) order
                if G.weights is not None:
                    assert np.array_equal(p.weights[lo:hi], G.weights[G.row_ptr[v]:G.row_ptr[v + 1]])
            # the halo is exactly the neighbours owned elsewhere, ascending
            nb = G.col_idx[G.row_ptr[p.row0]:G.row_ptr[p.row1]]
            outside = np.unique(nb[(nb < p.row0) | (nb >= p.row1)])
            assert np.array_equal(p.halo, outside)
        # what q sends to r is what r's ghost slots from q hold, in that order
        for r, pr in enumerate(parts):
            for q, pq in enumerate(parts):
                assert np.array_equal(pq.send[r] + pq.row0, pr.halo[pr.recv[q]])
            assert sum(len(x) for x in pr.recv) == pr.n_halo


def rowsum_f32(row_ptr, col, w, x, rows):
    """float32 sums over CSR rows, one rounding per addition, in row order."""
    out = np.zeros((len(rows), x.shape[1]), np.float32)
    for i, v in enumerate(rows):
        acc = np.zeros(x.shape[1], np.float32)
        for j in range(row_ptr[v], row_ptr[v + 1]):
            f = x[col[j]]
            acc = acc + f if (w is None or w[j] >= 0) else acc - f
        out[i] = acc
    return out


@pytest.mark.parametrize("P", [2, 3])
def test_local_row_sums_equal_the_global_ones(P):
    for G in graphs():
        x = np.random.default_rng(P).random((G.n, 4)).astype(np.float32) * 2 - 1
        want = rowsum_f32(G.row_ptr, G.col_idx, G.weights, x, range(G.n))
        for p in pt.plan(G, P):
            xl = np.concatenate([x[p.row0:p.row1], x[p.halo]])
            got = rowsum_f32(p.row_ptr, p.col_local, p.weights, xl, range(p.n_own))
            assert np.array_equal(got, want[p.row0:p.row1])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import mqo_inputs as mi_
    from paper_2605_06921_gb300 import partition as pt_
    dist.init_process_group("gloo", rank=rank, world_size=world)
    G = mi_.chung_lu(3000, 2.5, 8.0, 7)
    part = pt_.plan(G, world)[rank]
    x = np.random.default_rng(5).random((G.n, 8)).astype(np.float32)
    xl = torch.full((part.n_own + part.n_halo, 8), float("nan"))
    xl[:part.n_own] = torch.from_numpy(x[part.row0:part.row1])  # only the own rows are known here
    pt_.exchange_halo(xl, part)
    ok_halo = bool(torch.equal(xl[part.n_own:], torch.from_numpy(x[part.halo])))
    got = rowsum_f32(part.row_ptr, part.col_local, part.weights, xl.numpy(), range(part.n_own))
    want = rowsum_f32(G.row_ptr, G.col_idx, G.weights, x, range(part.row0, part.row1))
    out[rank] = (ok_halo, bool(np.array_equal(got, want)), part.n_halo)
    dist.barrier()
    dist.destroy_process_group()


def test_halo_exchange_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ok_halo, ok_sums, n_halo = out[r]
        assert n_halo > 0 and ok_halo and ok_sums

"""The seeded synthetic inputs: every generator returns a symmetric CSR with
sorted rows and no self loops, and has the shape its workload states (ER edge
probability, exact regular degrees, packed member graphs, power-law degree
skew), deterministically per seed."""
import numpy as np
import pytest

import mqo_inputs as mi


def assert_valid(G):
    rp, col = G.row_ptr, G.col_idx
    assert rp[0] == 0 and rp[-1] == len(col) and np.all(np.diff(rp) >= 0)
    rows = np.repeat(np.arange(G.n), np.diff(rp))
    assert np.all(col != rows), "self loop"
    for v in range(G.n):
        r = col[rp[v]:rp[v + 1]]
        assert np.all(np.diff(r) > 0), f"row {v} not strictly ascending"
    fwd = set(zip(rows.tolist(), col.tolist()))
    assert all((u, v) in fwd for v, u in fwd), "not symmetric"
    if G.weights is not None:
        w = dict(zip(zip(rows.tolist(), col.tolist()), G.weights.tolist()))
        assert all(w[(v, u)] == w[(u, v)] and w[(v, u)] in (-1, 1) for v, u in fwd)


@pytest.mark.parametrize("n,p,seed", [(200, 0.05, 0), (150, 0.3, 3), (60, 0.9, 7), (10, 0.0, 1)])
def test_erdos_renyi(n, p, seed):
    G = mi.erdos_renyi(n, p, seed)
    assert_valid(G)
    m = G.nnz // 2
    mean, sd = p * n * (n - 1) / 2, np.sqrt(p * (1 - p) * n * (n - 1) / 2)
    assert abs(m - mean) <= 5 * sd + 1e-9
    H = mi.erdos_renyi(n, p, seed)
    assert np.array_equal(G.row_ptr, H.row_ptr) and np.array_equal(G.col_idx, H.col_idx)


def test_random_regular_exact_degree():
    for n, d, seed in [(100, 3, 0), (1000, 3, 5), (64, 4, 2)]:
        G = mi.random_regular(n, d, seed)
        assert_valid(G)
        assert np.all(np.diff(G.row_ptr) == d)


def test_pack_and_subgraph_round_trip():
    gs = [mi.erdos_renyi(30, 0.2, 1), mi.random_regular(40, 3, 2), mi.erdos_renyi(25, 0.4, 3)]
    P = mi.pack(gs)
    assert_valid(P)
    assert P.num_graphs == 3 and list(P.node_offsets) == [0, 30, 70, 95]
    for k, g in enumerate(gs):
        s = P.subgraph(k)
        assert np.array_equal(s.row_ptr, g.row_ptr) and np.array_equal(s.col_idx, g.col_idx)
    # no edge crosses member graphs
    rows = np.repeat(np.arange(P.n), np.diff(P.row_ptr))
    gid = np.searchsorted(P.node_offsets, np.arange(P.n), side="right") - 1
    assert np.all(gid[rows] == gid[P.col_idx])


def test_chung_lu_power_law_skew():
    G = mi.chung_lu(20000, 2.5, 8.0, 0)
    assert_valid(G)
    deg = np.diff(G.row_ptr)
    assert 6.0 < deg.mean() < 8.5            # self loops and duplicates removed
    assert deg[:20].mean() > 20 * deg[-1000:].mean()  # expected degrees fall as (i+1)^(-2/3)
    assert deg.max() > 100                    # hubs at the low node ids


def test_er_table_workload_density():
    G = mi.workload_er_table(1000, 100.0, num_graphs=2)
    assert G.num_graphs == 2 and G.n == 2000
    for k in range(2):
        s = G.subgraph(k)
        assert abs(np.diff(s.row_ptr).mean() - 100 * 999 / 1000) < 3.0   # p = d/n


def test_signed_weights_are_symmetric():
    G = mi.erdos_renyi(80, 0.1, 4)
    rows, cols = G.edges_directed()
    keep = rows < cols
    rng = np.random.default_rng(0)
    w = np.where(rng.random(int(keep.sum())) < 0.5, -1, 1)
    H = mi.from_edges(G.n, rows[keep], cols[keep], w)
    assert_valid(H)


def test_random_regular_rejects_odd_stub_count_and_signs_edges():
    with pytest.raises(ValueError):
        mi.random_regular(11, 3, 0)
    G = mi.random_regular(200, 3, 4, signed_weights=True)
    assert_valid(G)
    w = G.weights
    assert set(np.unique(w).tolist()) == {-1, 1}
    assert 0.35 < (w == 1).mean() < 0.65

"""pmQO pool machine (Alg. 3 for MIS, Alg. 4 for MaxCut) on the CUDA path
against the oracle's pool machine, element by element: every trajectory's
state (held sets included), the best sets, and the pool members (count,
values, bits) of every member graph, at several points of a run."""
import numpy as np
import pytest

import mqo_inputs as mi
import oracle
from test_gpu_parity import close, host, okw, oracle_graphs, signed, small_batch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KEYS = ("phase", "s", "r", "o", "best", "ticks", "last_round", "last_commits", "ev_value", "ev_a", "ev_b",
        "accepts", "descents", "held", "first_value", "gain_descent", "gain_ls", "steps")


@pytest.fixture(scope="module")
def mq():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2605_06921_gb300 as m
    return m


def _pool_machine(mq, G, p, checkpoints, trace=0):
    s = mq.Solver(mq.Graph(G), p)
    po = okw(p)
    B, K = p.batch, p.pool_k
    ogs = oracle_graphs(G)
    pgs = [oracle.PoolGraph(og, po, g * B, B) for g, og in enumerate(ogs)]
    for k in range(trace):  # x of every descending trajectory, tick by tick
        s.run(1)
        gx = host(s.get_x())
        for g, pg in enumerate(pgs):
            pg.run(1)
            lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
            for b in range(B):
                st = pg.state(b)
                if st["phase"] == oracle.PH_DESCENT and st["last_round"] == -1:
                    assert close(gx[lo:hi, b], pg.x[b]), (k, g, b)
    done = trace
    merges_total = 0
    for upto in checkpoints:
        s.run(upto - done)
        for pg in pgs:
            pg.run(upto - done)
        done = upto
        states = s.traj_state()
        vals, bits = s.best()
        z = mq.unpack_bits(bits, G.n, B)
        counts, pvals, merges, pbits = s.pool_state()
        pz = mq.unpack_bits(pbits, G.n, K)
        for g, pg in enumerate(pgs):
            lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
            for b in range(B):
                t = g * B + b
                want = pg.state(b)
                for key in KEYS:
                    assert states[t][key] == want[key], (upto, g, b, key, states[t][key], want[key])
                assert vals[t] == want["best"]
                assert np.array_equal(z[lo:hi, b], pg.zbest[b]), (upto, g, b)
            wv, wb = pg.members()
            assert counts[g] == len(wv) and merges[g] == pg.pool.merges, (upto, g)
            assert np.array_equal(pvals[g, :counts[g]], wv), (upto, g)
            for k in range(counts[g]):
                assert np.array_equal(pz[lo:hi, k], wb[k]), (upto, g, k)
            merges_total += int(merges[g])
    assert merges_total > 0
    return s, pgs


def mis_params(mq, B, K, **kw):
    d = dict(problem=0, batch=B, alpha=0.8, momentum=0.45, rho=0.6, t_gs=4, descent_cap=25, init_kind=1, sigma=0.2,
             seed=5, pool_k=K)
    d.update(kw)
    return mq.params(**d)


def cut_params(mq, B, K, **kw):
    d = dict(problem=1, batch=B, alpha=0.05, momentum=0.8, lambda_=0.001, rho=0.8, t_gs=3, descent_cap=40,
             init_kind=1, sigma=0.2, seed=5, pool_k=K)
    d.update(kw)
    return mq.params(**d)


@pytest.mark.parametrize("B,K", [(4, 1), (8, 3), (32, 8), (16, 40)])
def test_pool_mis(mq, monkeypatch, B, K):
    monkeypatch.setenv("MQO_DISC_KERNEL", "graph" if B >= 32 else "pairs")
    G = small_batch(3, 30, 70, 0.15, seed=K)
    _pool_machine(mq, G, mis_params(mq, B, K, seed=B + K), [120, 300, 500], trace=20)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("B,K", [(4, 2), (8, 8), (64, 33)])
def test_pool_maxcut(mq, weighted, B, K):
    G = mi.pack([mi.random_regular(80, 3, 5 + K), mi.erdos_renyi(60, 0.1, 6 + B)])
    if weighted:
        G = signed(G, 7)
    _pool_machine(mq, G, cut_params(mq, B, K, seed=K), [150, 400, 700], trace=20)


@pytest.mark.parametrize("problem", [0, 1])
def test_pool_without_local_search_or_repair(mq, problem):
    G = small_batch(2, 30, 50, 0.2, seed=9)
    if problem == 0:
        p = mis_params(mq, 8, 4, t_gs=2, descent_cap=8, local_search=0, repair=0, seed=2)
    else:
        p = cut_params(mq, 8, 4, t_gs=2, descent_cap=15, local_search=0, seed=2)
    _pool_machine(mq, G, p, [100, 300])


@pytest.mark.parametrize("problem", [0, 1])
def test_pool_generic_kernels(mq, monkeypatch, problem):
    """the pool machine over the global-memory step kernel and the
    node-parallel discrete passes"""
    monkeypatch.setenv("MQO_STEP_KERNEL", "generic")
    monkeypatch.setenv("MQO_DISC_KERNEL", "pairs")
    G = small_batch(2, 30, 60, 0.15, seed=4)
    p = mis_params(mq, 32, 5, seed=4) if problem == 0 else cut_params(mq, 32, 5, seed=4)
    _pool_machine(mq, G, p, [200, 400])


def test_pool_autotune_keeps_results(mq):
    G = small_batch(3, 60, 120, 0.1, seed=11)
    p = mis_params(mq, 32, 6, seed=3)
    s = mq.Solver(mq.Graph(G), p)
    s.run(60)
    s.autotune(ticks=5)
    s.run(140)
    vals, bits = s.best()
    counts, pvals, merges, pbits = s.pool_state()
    po = okw(p)
    for g, og in enumerate(oracle_graphs(G)):
        pg = oracle.PoolGraph(og, po, g * 32, 32)
        pg.run(200)
        wv, _ = pg.members()
        assert np.array_equal(pvals[g, :counts[g]], wv) and merges[g] == pg.pool.merges
        assert all(vals[g * 32 + b] == pg.state(b)["best"] for b in range(32))


def test_pool_rejects_standalone_reset_and_search(mq):
    G = small_batch(2, seed=1)
    s = mq.Solver(mq.Graph(G), mis_params(mq, 8, 2))
    with pytest.raises(mq.MqoError):
        s.reset()
    with pytest.raises(mq.MqoError):
        s.local_search()
    s2 = mq.Solver(mq.Graph(G), mis_params(mq, 8, 0))
    with pytest.raises(mq.MqoError):
        s2.pool_state()

"""Pins of the oracle's pool machine (pmQO, Alg. 3 / Alg. 4) against facts
that do not come from the oracle itself: integer definitions, uniformity,
invariants of the pool, brute-force optima, and the special case in which
pmQO and the per-trajectory machine (Alg. 1 / 2, pinned elsewhere) take the
same steps."""
import numpy as np
import pytest

import mqo_inputs as mi
import oracle


def og(G):
    return oracle.Graph(G)


def test_pool_pick_is_the_high_word_of_u_times_count():
    # Alg. 3/4 step 7 draws a pool member uniformly: index = floor(u * count / 2^64)
    for traj, outer, rnd, count in [(0, 0, 1, 1), (5, 2, 3, 7), (123, 9, 60, 32), (7, 1, 2, 3)]:
        u = int(oracle.philox4x64_10([3, outer, rnd, 0], [11, traj])[0])
        assert oracle.pool_pick(11, traj, outer, rnd, count) == (u * count) >> 64
    assert oracle.pool_pick(11, 0, 0, 1, 0) == -1


def test_pool_pick_uniform():
    count, n = 5, 20000
    hits = np.bincount([oracle.pool_pick(3, t, 0, 1, count) for t in range(n)], minlength=count)
    assert hits.min() >= 0 and len(hits) == count
    chi2 = float(((hits - n / count) ** 2 / (n / count)).sum())
    assert chi2 < 20.5  # 4 degrees of freedom, p ~ 4e-4


def _pool_params(problem, K, B, t_gs=4, ls=1, seed=5):
    if problem == 0:
        return oracle.params(problem=0, batch=B, alpha=0.8, momentum=0.45, rho=0.6, t_gs=t_gs, descent_cap=25,
                             init_kind=1, sigma=0.2, local_search=ls, seed=seed, pool_k=K)
    return oracle.params(problem=1, batch=B, alpha=0.05, momentum=0.8, lambda_=0.001, rho=0.8, t_gs=t_gs,
                         descent_cap=40, init_kind=1, sigma=0.2, local_search=ls, seed=seed, pool_k=K)


@pytest.mark.parametrize("problem", [0, 1])
@pytest.mark.parametrize("K,B", [(1, 4), (3, 8), (8, 4)])
def test_pool_invariants(problem, K, B):
    G = mi.erdos_renyi(50, 0.12, 7 + K)
    g = og(G)
    pg = oracle.PoolGraph(g, _pool_params(problem, K, B), 0, B)
    best_seen = oracle.INT64_MIN
    for _ in range(12):
        pg.run(40)
        vals, bits = pg.members()
        assert len(vals) <= K
        assert all(vals[i] >= vals[i + 1] for i in range(len(vals) - 1))
        for v, z in zip(vals, bits):
            if problem == 0:
                size, conf_e, conf_n, unc = oracle.eval_mis(g, z)
                assert (conf_e, conf_n, unc) == (0, 0, 0)  # members are maximal independent sets
                assert size == v
            else:
                assert oracle.eval_cut(g, z)[0] == v
        best = pg.pool.best
        assert best >= best_seen  # the best set only improves
        best_seen = best
        if len(vals):
            assert best >= vals[0]
        for b in range(B):
            st = pg.state(b)
            assert st["best"] == best
            ev = oracle.eval_mis(g, pg.zbest[b]) if problem == 0 else oracle.eval_cut(g, pg.zbest[b])
            if best != oracle.INT64_MIN:
                assert ev[0] == best
        # trajectories of a graph move in lock step
        assert len({pg.state(b)["o"] for b in range(B)}) == 1
        assert len({pg.state(b)["r"] for b in range(B)}) == 1


@pytest.mark.parametrize("problem", [0, 1])
def test_pool_never_beats_brute_force(problem):
    G = mi.erdos_renyi(16, 0.3, 4)
    g = og(G)
    opt = oracle.brute_mis(g) if problem == 0 else oracle.brute_maxcut(g)
    pg = oracle.PoolGraph(g, _pool_params(problem, 4, 8, t_gs=3), 0, 8)
    pg.run(600)
    assert pg.pool.best <= opt
    assert pg.pool.best == opt  # a 16-node graph is solved by 600 ticks of 8 trajectories


@pytest.mark.parametrize("problem", [0, 1])
def test_pool_of_one_is_the_single_trajectory_machine(problem):
    """B = 1, K = 1, no local search: the pool holds the best descent result
    (ties keep the older set) and every reset starts from it, exactly as
    Alg. 1/2 reset from the best set.  The pool machine waits one tick at
    each round barrier, so the two are compared round by round."""
    G = mi.erdos_renyi(70, 0.08, 2)
    g = og(G)
    p = _pool_params(problem, 1, 1, t_gs=6, ls=0, seed=9)
    single = oracle.Trajectory(g, p, 0)
    pool = oracle.PoolGraph(g, p, 0, 1)

    def by_round(step, state, n):
        seen = {}
        for _ in range(n):
            step()
            st = state()
            seen.setdefault((st["o"], st["r"]), (st["best"], st["descents"]))
        return seen

    a = by_round(lambda: single.run(1), lambda: single.state, 1500)
    b = by_round(lambda: pool.run(1), lambda: pool.state(0), 1500)
    common = sorted(set(a) & set(b))
    assert len(common) > 20
    for key in common:  # the best set when round (o, r) starts, and the descents before it
        assert a[key] == b[key], (key, a[key], b[key])


@pytest.mark.parametrize("problem", [0, 1])
def test_pool_without_reset_rounds_goes_straight_to_local_search(problem):
    """T_gs = 0: after the first merge the graph runs local search (step 13)
    and then fresh initialisations; the pool invariants still hold and the
    best value never decreases."""
    G = mi.erdos_renyi(40, 0.15, 3)
    g = og(G)
    pg = oracle.PoolGraph(g, _pool_params(problem, 3, 4, t_gs=0), 0, 4)
    last = oracle.INT64_MIN
    for _ in range(10):
        pg.run(30)
        vals, bits = pg.members()
        assert all(vals[i] >= vals[i + 1] for i in range(len(vals) - 1))
        best = pg.pool.best
        assert best >= last
        last = best
        for b in range(4):
            assert pg.state(b)["r"] == 0          # no reset round is ever started
    assert pg.pool.merges > 0

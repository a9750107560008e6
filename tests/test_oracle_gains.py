"""Pins of the oracle's gains breakdown (the appendix on mQO's gains: the
value at the end of the first descent's gradient updates, then the increases
from global resets and from local search): every strict improvement of the
best value is booked exactly once, local search books nothing when it is
off, and the first booked value is the first descent's own evaluation."""
import numpy as np
import pytest

import mqo_inputs as mi
import oracle


def _params(problem, ls=1, pool_k=0, seed=3):
    if problem == 0:
        return oracle.params(problem=0, batch=4, alpha=0.8, momentum=0.45, rho=0.6, t_gs=3, descent_cap=25,
                             init_kind=1, sigma=0.2, local_search=ls, seed=seed, pool_k=pool_k)
    return oracle.params(problem=1, batch=4, alpha=0.05, momentum=0.8, lambda_=0.001, rho=0.8, t_gs=3,
                         descent_cap=40, init_kind=1, sigma=0.2, local_search=ls, seed=seed, pool_k=pool_k)


@pytest.mark.parametrize("problem", [0, 1])
@pytest.mark.parametrize("ls", [0, 1])
def test_breakdown_sums_to_best(problem, ls):
    G = mi.erdos_renyi(60, 0.1, 4)
    g = oracle.Graph(G)
    for traj in range(4):
        tr = oracle.Trajectory(g, _params(problem, ls), traj)
        for _ in range(6):
            tr.run(80)
            st = tr.state
            if st["best"] == oracle.INT64_MIN:
                assert st["first_value"] == oracle.INT64_MIN
                continue
            assert st["first_value"] + st["gain_descent"] + st["gain_ls"] == st["best"]
            assert st["gain_descent"] >= 0 and st["gain_ls"] >= 0
            if not ls:
                assert st["gain_ls"] == 0


@pytest.mark.parametrize("problem", [0, 1])
def test_first_value_is_the_first_descent(problem):
    """Run tick by tick until the first acceptance: the booked first value is
    the exact value of the set accepted then (MIS: size of an independent
    set; MaxCut: its cut), evaluated independently."""
    G = mi.erdos_renyi(50, 0.12, 9)
    g = oracle.Graph(G)
    tr = oracle.Trajectory(g, _params(problem), 0)
    for _ in range(400):
        tr.run(1)
        if tr.state["best"] != oracle.INT64_MIN:
            break
    st = tr.state
    assert st["accepts"] == 1 and st["first_value"] == st["best"]
    if problem == 0:
        size, ce, cn, unc = oracle.eval_mis(g, tr.zbest)
        assert ce == 0 and size == st["first_value"]
    else:
        assert oracle.eval_cut(g, tr.zbest)[0] == st["first_value"]


@pytest.mark.parametrize("problem", [0, 1])
def test_breakdown_in_pool_mode(problem):
    G = mi.erdos_renyi(50, 0.12, 7)
    g = oracle.Graph(G)
    pg = oracle.PoolGraph(g, _params(problem, pool_k=3), 0, 4)
    for _ in range(8):
        pg.run(60)
        for b in range(4):
            st = pg.state(b)
            if st["best"] != oracle.INT64_MIN:
                assert st["first_value"] + st["gain_descent"] + st["gain_ls"] == st["best"]

"""Pins of the oracle's machine rules that the brute-force bounds cannot see.

* the degree-based initialisation of Alg. 1 step 2 (MIS) and Alg. 2 step 2
  (MaxCut): centre 1 - d(v)/Delta, resp. 2(1 - d(v)/Delta) - 1, plus noise of
  standard deviation sigma, projected onto the box;
* the global reset of Alg. 1 / Alg. 2 steps 6-8: x from the best set
  (1 / 0 for MIS, +1 / -1 for MaxCut), 0 on the reset set R, momentum 0;
  checked through the machine: the first step after a reset must start from
  that point;
* strict acceptance (Alg. 1 / Alg. 2 steps 4, 10, 11): a candidate whose
  value only equals the best value leaves the best set and the acceptance
  count unchanged.

Each test is written so that a plausible mistake in the oracle (a dropped
affine map, a wrong sign, -1 instead of 0 on R, a momentum that survives the
reset, >= instead of >) fails it.
"""
import numpy as np

import mqo_inputs as mi
import oracle


def dense_adj(g):
    A = np.zeros((g.n, g.n))
    for v in range(g.n):
        for j in range(g.row_ptr[v], g.row_ptr[v + 1]):
            A[v, g.col[j]] = 1.0 if g.w is None else float(g.w[j])
    return A


# ---------------------------------------------------------------- initialisation
def test_degree_init_centres_without_noise():
    """sigma = 0: x_v is exactly the projected centre of Alg. 1 / Alg. 2 step 2."""
    G = mi.erdos_renyi(300, 0.03, 5)
    g = oracle.Graph(G)
    d = G.degrees().astype(np.float64)
    q = d / d.max()
    for problem, centre, lo in ((oracle.MIS, 1.0 - q, 0.0), (oracle.MAXCUT, 2.0 * (1.0 - q) - 1.0, -1.0)):
        x = oracle.init_x(g, oracle.params(problem=problem, init_kind=1, sigma=0.0), 0).astype(np.float64)
        np.testing.assert_allclose(x, np.clip(centre, lo, 1.0), rtol=0, atol=2e-7)
        # a node of maximum degree starts at the lower end of the box
        assert np.all(x[d == d.max()] == lo)


def test_maxcut_degree_init_centre_and_noise():
    """MaxCut: mean of x_v - (2(1 - d/Delta) - 1) is 0 and its spread is sigma
    over the nodes whose centre lies well inside [-1, 1]; the MIS centre
    1 - d/Delta (no affine map) is rejected by the same data."""
    G = mi.erdos_renyi(6000, 0.0015, 2)
    g = oracle.Graph(G)
    d = G.degrees().astype(np.float64)
    q = d / d.max()
    sigma = 0.05
    centre = 2.0 * (1.0 - q) - 1.0
    inner = np.abs(centre) < 1.0 - 6 * sigma
    assert inner.sum() > 3000
    res = []
    for traj in range(3):
        x = oracle.init_x(g, oracle.params(problem=oracle.MAXCUT, init_kind=1, sigma=sigma), traj)
        assert x.min() >= -1.0 and x.max() <= 1.0
        res.append((x.astype(np.float64) - centre)[inner])
    r = np.concatenate(res)
    assert abs(r.mean()) < 0.003
    assert abs(r.std() - sigma) < 0.05 * sigma
    # the dropped affine map (centre 1 - d/Delta) or the reversed sign
    # (2(1 + d/Delta) - 1) would leave an offset of more than 0.1 on average
    for wrong in (1.0 - q, 2.0 * (1.0 + q) - 1.0):
        assert abs(float(np.mean((centre - wrong)[inner]))) > 0.1


def test_init_noise_differs_per_trajectory_and_outer_iteration():
    """Each trajectory and each outer iteration draws its own noise."""
    G = mi.erdos_renyi(500, 0.02, 3)
    g = oracle.Graph(G)
    p = oracle.params(problem=oracle.MAXCUT, init_kind=1, sigma=0.1)
    a = oracle.init_x(g, p, 0, 0)
    assert not np.array_equal(a, oracle.init_x(g, p, 1, 0))
    assert not np.array_equal(a, oracle.init_x(g, p, 0, 1))
    assert np.array_equal(a, oracle.init_x(g, p, 0, 0))


# ---------------------------------------------------------------- reset through the machine
def _step_f64(A, problem, p, x, V):
    """One projected momentum step in float64 from (x, V) (Sec. 3, Sec. 5)."""
    Ax = A @ x
    if problem == oracle.MIS:
        grad, lo = 1.0 - float(p.gamma) * Ax, 0.0
    else:
        grad, lo = -float(p.lambda_) - 2.0 * Ax, -1.0
    Vn = float(p.momentum) * V + float(p.alpha) * grad
    return np.clip(x + Vn, lo, 1.0)


def _reset_point(problem, zbest, in_r):
    """Alg. 1 steps 6-8 (MIS) / Alg. 2 steps 6-8 (MaxCut)."""
    if problem == oracle.MIS:
        x = zbest.astype(np.float64)
    else:
        x = np.where(zbest != 0, 1.0, -1.0)
    x[in_r != 0] = 0.0
    return x


def _run_reset_pin(problem, graphs, params_for):
    checked = 0
    base_not_last = 0
    for k, G in enumerate(graphs):
        g = oracle.Graph(G)
        A = dense_adj(g)
        p = params_for(k)
        tr = oracle.Trajectory(g, p, 0)
        last = None
        for _ in range(400):
            before = tr.state
            zx_before = tr.zx_prev.copy()
            tr.run(1)
            st = tr.state
            if st["r"] == before["r"] + 1 and st["o"] == before["o"]:
                in_r = oracle.reset_mask(g.n, p.rho, p.seed, 0, st["o"], st["r"])
                assert int(in_r.sum()) == int(np.floor(p.rho * g.n))
                x0 = _reset_point(problem, tr.zbest, in_r)
                want = _step_f64(A, problem, p, x0, np.zeros(g.n))
                np.testing.assert_allclose(tr.x.astype(np.float64), want, rtol=0, atol=5e-6)
                checked += 1
                if before["phase"] == oracle.PH_DESCENT and not np.array_equal(zx_before, tr.zbest):
                    base_not_last += 1
            last = st
        assert last is not None
    return checked, base_not_last


def test_mis_reset_rule_through_the_machine():
    """MIS: after a reset the first step starts from x = 1(v in I_sol) off R,
    0 on R, V = 0 (momentum 0.6, so a surviving V would show)."""
    graphs = [mi.erdos_renyi(40, 0.15, s) for s in range(6)]
    checked, base_not_last = _run_reset_pin(
        oracle.MIS, graphs,
        lambda k: oracle.params(alpha=0.3, momentum=0.6, rho=0.4, t_gs=8, descent_cap=25, seed=10 + k))
    assert checked >= 30
    # some resets start from a best set that is not the last descent's set
    assert base_not_last >= 3


def test_maxcut_reset_rule_through_the_machine():
    """MaxCut: after a reset the first step starts from x = +1 on S_sol, -1
    off it, 0 on R, V = 0."""
    graphs = [mi.erdos_renyi(30, 0.2, s) for s in range(4)]
    graphs.append(mi.random_regular(30, 3, 1, signed_weights=True))
    checked, _ = _run_reset_pin(
        oracle.MAXCUT, graphs,
        lambda k: oracle.params(problem=oracle.MAXCUT, alpha=0.05, momentum=0.8, rho=0.5, t_gs=8,
                                descent_cap=30, init_kind=1, sigma=0.2, seed=20 + k))
    assert checked >= 20


# ---------------------------------------------------------------- strict acceptance
def _acceptance_events(problem, graphs, params_for, nticks):
    """Replays the machine tick by tick; for every tick that ends a descent
    (or a repair, or a local search) returns (candidate value, candidate set,
    best and best set and acceptance count before and after)."""
    events = []
    for k, G in enumerate(graphs):
        g = oracle.Graph(G)
        p = params_for(k)
        tr = oracle.Trajectory(g, p, 0)
        tr.run(1)
        for _ in range(nticks):
            b = tr.state
            zx, zw, zb = tr.zx_prev.copy(), tr.zwork.copy(), tr.zbest.copy()
            tr.run(1)
            a = tr.state
            cand = None
            if b["phase"] == oracle.PH_DESCENT and a["descents"] == b["descents"] + 1:
                passed = (b["ev_a"] == 0 and b["ev_b"] == 0) if problem == oracle.MIS else True
                if passed:
                    cand = zx
            elif b["phase"] == oracle.PH_REPAIR and b["ev_a"] == 0 and b["ev_b"] == 0:
                cand = zw
            elif b["phase"] == oracle.PH_LS and a["o"] == b["o"] + 1:
                cand = zw
            if cand is not None:
                events.append((b["ev_value"], cand, b["best"], zb, b["accepts"], a["best"], tr.zbest.copy(),
                               a["accepts"]))
    return events


def _check_strict(events):
    ties = 0
    for value, cand, best0, zb0, acc0, best1, zb1, acc1 in events:
        if value > best0:
            assert best1 == value and np.array_equal(zb1, cand) and acc1 == acc0 + 1
        else:
            assert best1 == best0 and np.array_equal(zb1, zb0) and acc1 == acc0
            if value == best0 and not np.array_equal(cand, zb0):
                ties += 1
    return ties


def test_mis_acceptance_is_strict():
    graphs = [mi.erdos_renyi(36, 0.15, s) for s in range(4)]
    events = _acceptance_events(
        oracle.MIS, graphs,
        lambda k: oracle.params(alpha=0.3, momentum=0.3, rho=0.5, t_gs=6, descent_cap=25, seed=40 + k), 500)
    # equal-valued candidates with a different set must have occurred
    assert _check_strict(events) >= 5


def test_maxcut_acceptance_is_strict():
    graphs = [mi.erdos_renyi(24, 0.25, s) for s in range(4)]
    events = _acceptance_events(
        oracle.MAXCUT, graphs,
        lambda k: oracle.params(problem=oracle.MAXCUT, alpha=0.05, momentum=0.8, rho=0.5, t_gs=6,
                                descent_cap=40, init_kind=1, sigma=0.2, seed=60 + k), 600)
    assert _check_strict(events) >= 5


# ---------------------------------------------------------------- step count
def test_steps_count_the_ticks_that_ran_a_gradient_step():
    """`steps` grows by one exactly on the ticks whose round is a descent step
    (last_round == -1); with repair and local search off every tick steps."""
    G = mi.erdos_renyi(40, 0.15, 1)
    g = oracle.Graph(G)
    tr = oracle.Trajectory(g, oracle.params(t_gs=3, descent_cap=20, seed=5), 0)
    for _ in range(400):
        before = tr.state["steps"]
        tr.run(1)
        st = tr.state
        assert st["steps"] - before == (1 if st["last_round"] == -1 else 0)
    assert 0 < st["steps"] < st["ticks"]
    tr = oracle.Trajectory(g, oracle.params(t_gs=3, descent_cap=20, seed=5, local_search=0, repair=0), 0)
    tr.run(300)
    assert tr.state["steps"] == tr.state["ticks"] == 300

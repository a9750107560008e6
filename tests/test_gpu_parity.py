"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bars: integer evaluation and every machine decision bit-exact; float32
iterates within 1e-5 relative (they are expected to be bit-exact: both sides
accumulate (Ax)_v in CSR order with one rounding per operation).
"""
import numpy as np
import pytest

import mqo_inputs as mi
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-5


@pytest.fixture(scope="module")
def mq():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2605_06921_gb300 as m
    return m


def host(t):
    if t.dtype in (torch.bfloat16, torch.float16):
        t = t.float()
    return t.cpu().numpy()


def close(a, b, rtol=RTOL):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.all(np.abs(a - b) <= rtol * np.maximum(np.abs(b), 1e-30) + 1e-30)


def small_batch(num=5, lo=40, hi=90, p=0.12, seed=0):
    sizes = mi.er_batch_sizes(num, lo, hi, 77 + seed)
    return mi.pack([mi.erdos_renyi(int(sizes[k]), p, 1000 * seed + k) for k in range(num)])


def signed(G, seed=0):
    rng = np.random.default_rng(seed)
    rows, cols = G.edges_directed()
    keep = rows < cols
    w = np.where(rng.random(int(keep.sum())) < 0.5, -1, 1)
    H = mi.from_edges(G.n, rows[keep], cols[keep], w)
    H.node_offsets = G.node_offsets
    return H


def okw(p):
    """oracle params matching a library Params struct"""
    return oracle.params(problem=p.problem, batch=p.batch, x_dtype=p.x_dtype, v_dtype=p.v_dtype, alpha=p.alpha,
                         momentum=p.momentum, gamma=p.gamma, lambda_=p.lambda_, rho=p.rho, sigma=p.sigma,
                         t_gs=p.t_gs, descent_cap=p.descent_cap, init_kind=p.init_kind,
                         local_search=p.local_search, repair=p.repair, seed=p.seed, objective=p.objective,
                         pool_k=p.pool_k)


def oracle_graphs(G):
    return [oracle.Graph(G.subgraph(g)) for g in range(G.num_graphs)]


# ------------------------------------------------------------------ init + plain steps
@pytest.mark.parametrize("problem", [0, 1])
@pytest.mark.parametrize("init_kind", [0, 1])
@pytest.mark.parametrize("dt", [0, 1, 2])
def test_init_matches_oracle(mq, problem, init_kind, dt):
    G = small_batch(3)
    B = 8
    p = mq.params(problem=problem, batch=B, x_dtype=dt, init_kind=init_kind, sigma=0.2, seed=11)
    s = mq.Solver(mq.Graph(G), p)
    x = host(s.get_x())
    po = okw(p)
    for g, og in enumerate(oracle_graphs(G)):
        lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
        for b in range(B):
            want = oracle.init_x(og, po, g * B + b, 0)
            assert np.array_equal(x[lo:hi, b], want), (g, b)


def _plain_steps(mq, G, p, nsteps):
    s = mq.Solver(mq.Graph(G), p)
    po = okw(p)
    B = p.batch
    ogs = oracle_graphs(G)
    xs = [[oracle.init_x(og, po, g * B + b, 0) for b in range(B)] for g, og in enumerate(ogs)]
    vs = [[np.zeros(og.n, np.float32) for b in range(B)] for og in ogs]
    for k in range(nsteps):
        s.step(1)
        gx = host(s.get_x())
        gv = host(s.get_v())
        sv, sa, sb = (host(t) for t in s.step_stats())
        for g, og in enumerate(ogs):
            lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
            for b in range(B):
                xn, vn, z, ev = oracle.descent_step(og, po, xs[g][b], vs[g][b])
                xs[g][b], vs[g][b] = xn, vn
                t = g * B + b
                assert (sv[t], sa[t], sb[t]) == ev, (k, g, b)
                assert close(gx[lo:hi, b], xn), (k, g, b)
                assert close(gv[lo:hi, b], vn), (k, g, b)
    return s


def test_plain_steps_config1_200_steps_bitexact(mq):
    G = mi.workload_mis_plain()
    p = mq.params(batch=1, alpha=0.8, momentum=0.3, gamma=2.0, seed=0)
    s = mq.Solver(mq.Graph(G), p)
    og = oracle.Graph(G)
    po = okw(p)
    x = oracle.init_x(og, po, 0, 0)
    V = np.zeros(G.n, np.float32)
    worst = 0.0
    for k in range(200):
        s.step(1)
        x, V, z, ev = oracle.descent_step(og, po, x, V)
        gx = host(s.get_x())[:, 0]
        worst = max(worst, float(np.max(np.abs(gx - x) / np.maximum(np.abs(x), 1e-30))))
        assert np.array_equal(gx, x), k
        assert tuple(int(t[0]) for t in (host(u) for u in s.step_stats())) == ev, k
    assert worst <= RTOL


@pytest.mark.parametrize("B", [1, 2, 4, 8, 16, 32, 64, 128])
def test_plain_steps_batch_sizes_mis(mq, B):
    _plain_steps(mq, small_batch(3, seed=B), mq.params(batch=B, alpha=0.8, momentum=0.45, seed=B), 12)


@pytest.mark.parametrize("problem", [0, 1])
@pytest.mark.parametrize("B,xd", [(32, 0), (32, 1), (64, 0), (128, 1)])
def test_generic_step_kernel_on_small_graphs(mq, monkeypatch, problem, B, xd):
    """the global-memory step kernel and the node-parallel discrete passes
    (used for large graphs) on graphs that would otherwise take the
    shared-memory kernels"""
    monkeypatch.setenv("MQO_STEP_KERNEL", "generic")
    monkeypatch.setenv("MQO_DISC_KERNEL", "pairs")
    p = mq.params(problem=problem, batch=B, x_dtype=xd, alpha=0.8 if problem == 0 else 0.05, momentum=0.5, seed=B)
    _plain_steps(mq, small_batch(2, seed=B + 1), p, 8)
    G = small_batch(2, 30, 60, 0.15, seed=B)
    _machine(mq, G, mq.params(problem=problem, batch=B, x_dtype=xd, t_gs=3, descent_cap=20, seed=3), 150)


@pytest.mark.parametrize("problem", [0, 1])
@pytest.mark.parametrize("B,xd,vd", [(32, 1, 1), (32, 2, 0), (32, 0, 0), (64, 1, 1), (64, 0, 0), (128, 2, 2)])
def test_wide_lane_step_kernel(mq, monkeypatch, problem, B, xd, vd):
    """the shared-memory step kernel with 16-byte lanes (an autotuner plan)"""
    monkeypatch.setenv("MQO_STEP_KERNEL", "wide")
    p = mq.params(problem=problem, batch=B, x_dtype=xd, v_dtype=vd, alpha=0.8 if problem == 0 else 0.05,
                  momentum=0.5, seed=B + 7)
    _plain_steps(mq, small_batch(3, seed=B + 2), p, 8)
    G = small_batch(2, 30, 60, 0.15, seed=B + 5)
    s, _ = _machine(mq, G, mq.params(problem=problem, batch=B, x_dtype=xd, v_dtype=vd, t_gs=3, descent_cap=20,
                                     seed=5), 150)
    assert s.info()["step_kernel"] == "smem_wide"


@pytest.mark.parametrize("problem,weighted", [(0, False), (1, False), (1, True)])
@pytest.mark.parametrize("B,xd,vd", [(8, 2, 2), (16, 2, 2), (16, 2, 0), (32, 1, 1), (8, 0, 0), (64, 0, 0),
                                     (128, 1, 1), (128, 1, 0)])
def test_staged_step_kernel(mq, monkeypatch, problem, weighted, B, xd, vd):
    """the staged-gather step kernel (the default for graphs too large for
    shared memory) on small graphs; with 256-byte rows of x (B = 128 in
    16-bit, B = 64 in float32) every work item spans many slices"""
    mode = "staged"
    monkeypatch.setenv("MQO_STEP_KERNEL", mode)
    monkeypatch.setenv("MQO_DISC_KERNEL", "pairs")
    G = small_batch(3, 60, 300, 0.05, seed=B + xd)
    if weighted:
        G = signed(G, B)
    p = mq.params(problem=problem, batch=B, x_dtype=xd, v_dtype=vd, alpha=0.8 if problem == 0 else 0.05,
                  momentum=0.5, seed=B + 11)
    s = _plain_steps(mq, G, p, 8)
    assert s.info()["step_kernel"] == mode and s.info()["slice_kb"] == 32
    G = small_batch(2, 30, 60, 0.15, seed=B + 9)
    if weighted:
        G = signed(G, B + 1)
    s, _ = _machine(mq, G, mq.params(problem=problem, batch=B, x_dtype=xd, v_dtype=vd, t_gs=3, descent_cap=20,
                                     seed=9), 150)
    assert s.info()["step_kernel"] == mode


def test_staged_step_kernel_grows_the_slice_for_long_rows(mq, monkeypatch):
    """a star of 200 leaves with 256-byte rows of x (50 KB of neighbour rows):
    the staged kernel takes 64 KB slices"""
    monkeypatch.setenv("MQO_STEP_KERNEL", "staged")
    star = mi.from_edges(201, np.zeros(200, int), np.arange(1, 201))
    G = mi.pack([star, mi.erdos_renyi(80, 0.1, 5)])
    p = mq.params(problem=1, batch=128, x_dtype=1, alpha=0.05, momentum=0.5, seed=6)
    s = _plain_steps(mq, G, p, 6)
    assert s.info()["step_kernel"] == "staged" and s.info()["slice_kb"] == 64


def test_staged_step_kernel_falls_back_on_long_rows(mq, monkeypatch):
    """a row whose neighbour rows of x exceed the largest slice (a star of 600
    leaves, 256-byte rows: 150 KB against 128 KB): the plain global-memory
    kernel takes the step"""
    monkeypatch.setenv("MQO_STEP_KERNEL", "staged")
    star = mi.from_edges(601, np.zeros(600, int), np.arange(1, 601))
    G = mi.pack([star, mi.erdos_renyi(80, 0.1, 4)])
    p = mq.params(problem=1, batch=128, x_dtype=1, alpha=0.05, momentum=0.5, seed=4)
    s = _plain_steps(mq, G, p, 6)
    assert s.info()["step_kernel"] == "global"


@pytest.mark.parametrize("xd,vd", [(1, 1), (1, 0), (2, 2), (2, 0)])
@pytest.mark.parametrize("B", [16, 32, 128])
def test_plain_steps_low_precision_mis(mq, xd, vd, B):
    _plain_steps(mq, small_batch(2, seed=3), mq.params(batch=B, x_dtype=xd, v_dtype=vd, seed=5), 10)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("B,xd", [(4, 0), (32, 0), (64, 1), (128, 1), (16, 2)])
def test_plain_steps_maxcut(mq, weighted, B, xd):
    G = mi.pack([mi.random_regular(60, 3, 1), mi.random_regular(90, 3, 2), mi.erdos_renyi(70, 0.1, 3)])
    if weighted:
        G = signed(G, 4)
    p = mq.params(problem=1, batch=B, x_dtype=xd, alpha=0.05, momentum=0.8, lambda_=0.001, init_kind=0, seed=9)
    _plain_steps(mq, G, p, 15)


# ------------------------------------------------------------------ exact evaluation
@pytest.mark.parametrize("problem,weighted", [(0, False), (1, False), (1, True)])
@pytest.mark.parametrize("B", [1, 8, 32, 64])
def test_evaluate_bitexact(mq, problem, weighted, B):
    G = small_batch(4, seed=B)
    if weighted:
        G = signed(G, B)
    p = mq.params(problem=problem, batch=B, seed=1)
    s = mq.Solver(mq.Graph(G), p)
    rng = np.random.default_rng(B)
    for density in (0.05, 0.3, 0.7):
        z = (rng.random((G.n, B)) < density).astype(np.uint8)
        bits = torch.from_numpy(mq.pack_bits(z, B)).cuda()
        v, a, c = (host(t) for t in s.evaluate(bits))
        for g, og in enumerate(oracle_graphs(G)):
            lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
            for b in range(B):
                t = g * B + b
                if problem == 0:
                    size, ce, cn, unc = oracle.eval_mis(og, z[lo:hi, b])
                    assert (v[t], a[t], c[t]) == (size, ce, unc)
                else:
                    cut, nf, cand = oracle.eval_cut(og, z[lo:hi, b])
                    assert (v[t], a[t], c[t]) == (cut, nf, cand)
        # round trip of the rounding kernel
    r = s.round()
    x = host(s.get_x())
    thr = 0.5 if problem == 0 else 0.0
    assert np.array_equal(mq.unpack_bits(r, G.n, B), (x > thr).astype(np.uint8))


# ------------------------------------------------------------------ the machine
def _machine(mq, G, p, nticks, trace=0, tune_at=None):
    s = mq.Solver(mq.Graph(G), p)
    po = okw(p)
    B = p.batch
    ogs = oracle_graphs(G)
    trs = [[oracle.Trajectory(og, po, g * B + b) for b in range(B)] for g, og in enumerate(ogs)]
    for k in range(trace):
        s.run(1)
        gx = host(s.get_x())
        for g, og in enumerate(ogs):
            lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
            for b in range(B):
                tr = trs[g][b]
                tr.run(1)
                if tr.state["phase"] == oracle.PH_DESCENT and tr.state["last_round"] == -1:
                    assert close(gx[lo:hi, b], tr.x), (k, g, b)
    if tune_at is None:
        s.run(nticks - trace)
    else:
        s.run(tune_at - trace)
        plan = s.autotune(ticks=5)
        assert plan["ms_per_tick"] > 0
        assert plan["step_kernel"].startswith("smem") == (plan["lanes_vec"] == 0)
        s.run(nticks - tune_at)
    vals, bits = s.best()
    z = mq.unpack_bits(bits, G.n, B)
    states = s.traj_state()
    for g, og in enumerate(ogs):
        lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
        for b in range(B):
            tr = trs[g][b]
            tr.run(nticks - trace)
            t = g * B + b
            want = tr.state
            got = states[t]
            for key in ("phase", "s", "r", "o", "best", "ticks", "last_round", "last_commits", "ev_value", "ev_a",
                        "ev_b", "accepts", "descents", "first_value", "gain_descent", "gain_ls", "steps"):
                assert got[key] == want[key], (g, b, key, got[key], want[key])
            assert vals[t] == want["best"]
            assert np.array_equal(z[lo:hi, b], tr.zbest), (g, b)
    return s, trs


def test_machine_config1_2000_ticks(mq):
    """MIS on ER(200, 0.05) seed 0, one trajectory, 2000 ticks, x traced for 200."""
    G = mi.workload_mis_plain()
    p = mq.params(batch=1, alpha=0.8, momentum=0.3, gamma=2.0, rho=0.7, t_gs=60, descent_cap=50, seed=0)
    s, trs = _machine(mq, G, p, 2000, trace=200)
    og = oracle.Graph(G)
    assert oracle.eval_mis(og, trs[0][0].zbest)[1:] == (0, 0, 0)


@pytest.mark.parametrize("disc", ["graph", "pairs"])
@pytest.mark.parametrize("B", [1, 8, 32])
def test_machine_packed_mis(mq, monkeypatch, B, disc):
    """both discrete-kernel plans: the fused per-graph kernel (forced here; by
    default it serves batches of many member graphs) and the node-parallel
    passes"""
    monkeypatch.setenv("MQO_DISC_KERNEL", disc)
    G = small_batch(4, 30, 70, 0.15, seed=B)
    p = mq.params(batch=B, alpha=0.8, momentum=0.45, rho=0.6, t_gs=4, descent_cap=25, seed=B)
    _machine(mq, G, p, 400, trace=30)


@pytest.mark.parametrize("disc", ["graph", "pairs"])
@pytest.mark.parametrize("serial", ["0", "1"])
def test_step_and_discrete_branches_take_the_same_ticks(mq, monkeypatch, serial, disc):
    """The step and the discrete kernels (fused, or the node-parallel passes)
    run as two branches of a tick (default) or one after the other
    (MQO_SERIAL_TICK=1): the machine takes the oracle's ticks either way."""
    monkeypatch.setenv("MQO_DISC_KERNEL", disc)
    monkeypatch.setenv("MQO_SERIAL_TICK", serial)
    G = small_batch(6, 40, 90, 0.15, seed=31)
    p = mq.params(batch=32, x_dtype=1, v_dtype=1, alpha=0.8, momentum=0.45, rho=0.6, t_gs=3, descent_cap=20,
                  seed=13)
    s, _ = _machine(mq, G, p, 300)
    assert s.info()["discrete_kernel"] == disc


@pytest.mark.parametrize("stream", ["csr32", "csr16", "ell"])
def test_shared_memory_step_kernel_index_streams(mq, monkeypatch, stream):
    """the shared-memory step kernel with 32-bit global and with 16-bit
    member-local CSR column indices, and with the sliced-ELL stream, takes
    the same ticks"""
    monkeypatch.setenv("MQO_COL16", "1" if stream == "csr16" else "0")
    monkeypatch.setenv("MQO_STEP_ELL", "1" if stream == "ell" else "0")
    G = small_batch(4, 60, 120, 0.1, seed=21)
    p = mq.params(batch=32, x_dtype=1, v_dtype=1, alpha=0.8, momentum=0.45, rho=0.6, t_gs=3, descent_cap=25,
                  seed=7)
    s, _ = _machine(mq, G, p, 150)
    info = s.info()
    assert info["step_kernel"] == "smem" and info["col16"] == (stream == "csr16") and info["ell"] == (stream == "ell")


def star_batch(leaves=150, seed=0):
    """a star (one row of `leaves` entries among rows of one entry: its warp
    group is padded to the hub's length) packed with two ER graphs"""
    star = mi.from_edges(leaves + 1, np.zeros(leaves, int), np.arange(1, leaves + 1))
    return mi.pack([mi.erdos_renyi(70, 0.12, seed), star, mi.erdos_renyi(45, 0.2, seed + 1)])


@pytest.mark.parametrize("problem", [0, 1])
@pytest.mark.parametrize("B,xd,vd,wide", [(32, 1, 1, False), (32, 1, 0, False), (64, 1, 1, False),
                                          (128, 1, 1, False), (32, 1, 1, True), (64, 1, 0, True),
                                          (128, 1, 1, True), (32, 2, 2, False), (64, 2, 0, True)])
def test_ell_step_kernel(mq, monkeypatch, problem, B, xd, vd, wide):
    """the shared-memory step kernel with the sliced-ELL stream for every
    lane layout (rows per warp 1 to 8), element by element against the
    oracle's steps and through the machine; MIS with float16 x has no ELL
    form (its checker reads rounding words) and keeps the CSR indices"""
    monkeypatch.setenv("MQO_STEP_ELL", "1")
    if wide:
        monkeypatch.setenv("MQO_STEP_KERNEL", "wide")
    p = mq.params(problem=problem, batch=B, x_dtype=xd, v_dtype=vd, alpha=0.8 if problem == 0 else 0.05,
                  momentum=0.5, seed=B + 13)
    s = _plain_steps(mq, star_batch(seed=B), p, 10)
    info = s.info()
    assert info["step_kernel"] == ("smem_wide" if wide else "smem")
    assert info["ell"] == (problem == 1 or xd == 1)
    G = small_batch(3, 30, 70, 0.15, seed=B + 3)
    s, _ = _machine(mq, G, mq.params(problem=problem, batch=B, x_dtype=xd, v_dtype=vd, t_gs=3, descent_cap=20,
                                     seed=B), 150)
    assert s.info()["ell"] == (problem == 1 or xd == 1)


@pytest.mark.parametrize("problem", [0, 1])
@pytest.mark.parametrize("wide", [False, True])
def test_ell_step_kernel_isolated_nodes(mq, monkeypatch, problem, wide):
    """member graphs whose last rows (in decreasing-degree order) have no
    neighbours: their lockstep groups hold no vectors at all"""
    monkeypatch.setenv("MQO_STEP_ELL", "1")
    if wide:
        monkeypatch.setenv("MQO_STEP_KERNEL", "wide")
    rng = np.random.default_rng(5)
    parts = []
    for k in range(3):
        n, m = 70 + 9 * k, 40
        u = rng.integers(0, m, 120)
        v = rng.integers(0, m, 120)
        keep = u != v
        parts.append(mi.from_edges(n, u[keep], v[keep]))  # nodes m .. n-1 isolated
    G = mi.pack(parts)
    assert (np.diff(G.row_ptr) == 0).sum() >= 90
    p = mq.params(problem=problem, batch=32, x_dtype=1, alpha=0.8 if problem == 0 else 0.05, momentum=0.5, seed=4)
    s = _plain_steps(mq, G, p, 8)
    assert s.info()["ell"] and s.info()["step_kernel"] == ("smem_wide" if wide else "smem")
    _machine(mq, G, mq.params(problem=problem, batch=32, x_dtype=1, t_gs=3, descent_cap=20, seed=6), 120)


def test_ell_step_kernel_not_for_weighted_maxcut(mq, monkeypatch):
    """the ELL stream carries no edge weights: signed MaxCut keeps the CSR
    indices"""
    monkeypatch.setenv("MQO_STEP_ELL", "1")
    G = signed(small_batch(3, 40, 80, 0.1, seed=4), 4)
    p = mq.params(problem=1, batch=32, x_dtype=1, alpha=0.05, momentum=0.8, seed=2)
    s = _plain_steps(mq, G, p, 6)
    assert s.info()["step_kernel"] == "smem" and not s.info()["ell"]


@pytest.mark.parametrize("xd", [0, 1])
@pytest.mark.parametrize("problem", [0, 1])
def test_autotune_keeps_results(mq, monkeypatch, problem, xd):
    """Autotuning mid-run (every plan tried, state restored) changes no tick
    of the machine; with bfloat16 x the candidates include the wide lanes,
    both CSR index widths and the sliced-ELL stream."""
    monkeypatch.setenv("MQO_DISC_KERNEL", "graph")  # make the fused discrete plan one of the candidates
    G = small_batch(4, 60, 120, 0.1, seed=11)
    if problem == 0:
        p = mq.params(batch=32, x_dtype=xd, alpha=0.8, momentum=0.45, rho=0.6, t_gs=4, descent_cap=25, seed=3)
    else:
        p = mq.params(problem=1, batch=32, x_dtype=xd, alpha=0.05, momentum=0.8, lambda_=0.001, rho=0.8, t_gs=3,
                      descent_cap=40, init_kind=1, sigma=0.2, seed=3)
    _machine(mq, G, p, 200, trace=0, tune_at=60)


def test_machine_mis_low_precision(mq):
    G = small_batch(3, 40, 60, 0.15, seed=2)
    p = mq.params(batch=16, x_dtype=1, v_dtype=1, alpha=0.8, momentum=0.45, rho=0.6, t_gs=3, descent_cap=25, seed=4)
    _machine(mq, G, p, 300)


@pytest.mark.parametrize("disc", ["graph", "pairs"])
@pytest.mark.parametrize("weighted", [False, True])
def test_machine_maxcut(mq, monkeypatch, weighted, disc):
    monkeypatch.setenv("MQO_DISC_KERNEL", disc)
    G = mi.pack([mi.random_regular(80, 3, 5), mi.erdos_renyi(60, 0.1, 6)])
    if weighted:
        G = signed(G, 7)
    p = mq.params(problem=1, batch=8, alpha=0.05, momentum=0.8, lambda_=0.001, rho=0.8, t_gs=3, descent_cap=60,
                  init_kind=1, sigma=0.2, seed=8)
    _machine(mq, G, p, 600, trace=40)


def test_machine_no_local_search_no_repair(mq):
    G = small_batch(2, 30, 50, 0.2, seed=9)
    p = mq.params(batch=4, t_gs=2, descent_cap=8, local_search=0, repair=0, seed=2)
    _machine(mq, G, p, 200)


def test_machine_edge_cases(mq):
    """isolated nodes, an edgeless graph, a star, a clique, a node of degree >> mean"""
    star = mi.from_edges(40, np.zeros(39, int), np.arange(1, 40))
    clique = mi.from_edges(12, *np.triu_indices(12, 1))
    empty = mi.from_edges(7, [], [])
    iso = mi.erdos_renyi(50, 0.03, 1)
    G = mi.pack([star, clique, empty, iso])
    p = mq.params(batch=4, t_gs=3, descent_cap=20, seed=5)
    _machine(mq, G, p, 250)
    p = mq.params(problem=1, batch=4, alpha=0.05, momentum=0.8, t_gs=3, descent_cap=40, seed=5)
    _machine(mq, G, p, 250)


# ------------------------------------------------------------------ reset, local search, objective
def test_forced_reset(mq):
    G = small_batch(3, seed=5)
    B = 8
    p = mq.params(batch=B, rho=0.6, t_gs=5, descent_cap=20, seed=3)
    s = mq.Solver(mq.Graph(G), p)
    s.run(57)
    st = s.traj_state()
    _, bits = s.best()
    zb = mq.unpack_bits(bits, G.n, B)
    mask = torch.zeros(G.num_graphs * B, dtype=torch.uint8, device="cuda")
    mask[1::3] = 1
    x_before = host(s.get_x())
    s.reset(mask)
    x = host(s.get_x())
    st2 = s.traj_state()
    for g in range(G.num_graphs):
        lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
        for b in range(B):
            t = g * B + b
            if t % 3 != 1:
                assert np.array_equal(x[lo:hi, b], x_before[lo:hi, b])
                continue
            inr = oracle.reset_mask(hi - lo, 0.6, 3, t, st[t]["o"], st[t]["r"] + 1)
            want = np.where(inr == 1, 0.0, zb[lo:hi, b].astype(np.float32))
            assert np.array_equal(x[lo:hi, b], want)
            assert st2[t]["r"] == st[t]["r"] + 1 and st2[t]["s"] == 0 and st2[t]["phase"] == 0


@pytest.mark.parametrize("problem", [0, 1])
def test_standalone_local_search(mq, problem):
    G = small_batch(3, 40, 80, 0.12, seed=6)
    B = 8
    p = mq.params(problem=problem, batch=B, alpha=0.8 if problem == 0 else 0.05, momentum=0.4, t_gs=2,
                  descent_cap=15, local_search=0, seed=6)
    s = mq.Solver(mq.Graph(G), p)
    s.run(40)
    st0 = s.traj_state()
    v0, b0 = s.best()
    z0 = mq.unpack_bits(b0, G.n, B)
    s.local_search()
    v1, b1 = s.best()
    z1 = mq.unpack_bits(b1, G.n, B)
    st1 = s.traj_state()
    rnd = (oracle.round_complete, oracle.round_swap) if problem == 0 else (oracle.round_flip1, oracle.round_flip2)
    for g, og in enumerate(oracle_graphs(G)):
        lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
        for b in range(B):
            t = g * B + b
            z = z0[lo:hi, b].copy()
            last = None
            while True:  # the LS round policy of the machine
                if problem == 0:
                    free = oracle.eval_mis(og, z)[3]
                    if free > 0:
                        z, k = rnd[0](og, z); last = ("c", k)
                    elif last is None or last != ("s", 0):
                        z, k = rnd[1](og, z); last = ("s", k)
                    else:
                        break
                else:
                    cand = oracle.eval_cut(og, z)[2]
                    if cand > 0:
                        z, k = rnd[0](og, z); last = ("1", k)
                    elif last is None or last != ("2", 0):
                        z, k = rnd[1](og, z); last = ("2", k)
                    else:
                        break
            val = oracle.eval_mis(og, z)[0] if problem == 0 else oracle.eval_cut(og, z)[0]
            if val > v0[t]:
                assert v1[t] == val and np.array_equal(z1[lo:hi, b], z)
            else:
                assert v1[t] == v0[t] and np.array_equal(z1[lo:hi, b], z0[lo:hi, b])
            for key in ("phase", "s", "r", "o", "ev_a", "ev_b"):
                assert st1[t][key] == st0[t][key]


@pytest.mark.parametrize("problem", [0, 1])
def test_objective_f64(mq, problem):
    G = small_batch(3, seed=7)
    B = 8
    p = mq.params(problem=problem, batch=B, gamma=1.7, lambda_=0.01, seed=7)
    s = mq.Solver(mq.Graph(G), p)
    s.step(3)
    obj = host(s.objective_f64())
    x = host(s.get_x())
    for g, og in enumerate(oracle_graphs(G)):
        lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
        for b in range(B):
            xb = x[lo:hi, b].astype(np.float64)
            want = oracle.objective_f64(og, problem, 1.7, 0.01, xb)
            # (Ax)_v is accumulated in float32 (relative error <= d(v) 2^-24),
            # products and sums in double: bound by the size of the terms
            dmax = int(np.diff(og.row_ptr).max())
            scale = np.abs(xb).sum() * (1.0 + 1.7 * dmax * np.abs(xb).max())
            assert abs(obj[g * B + b] - want) <= 1e-7 * dmax * scale + 1e-12

"""MaxCut relaxations f_L, f_P, f_A (Sec. 3) beside f_B on the CUDA path,
against the oracle element by element: the plain fused step (gradient of
the selected relaxation, its fixed-point count), the whole machine, and the
float64 relaxed objective."""
import numpy as np
import pytest

import mqo_inputs as mi
import oracle
from test_gpu_parity import _machine, _plain_steps, host, oracle_graphs, signed

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OBJS = {"f_L": 1, "f_P": 2, "f_A": 3, "f_B": 0}


@pytest.fixture(scope="module")
def mq():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2605_06921_gb300 as m
    return m


def cut_batch(seed):
    return mi.pack([mi.random_regular(60, 3, seed), mi.erdos_renyi(90, 0.08, seed + 1),
                    mi.erdos_renyi(45, 0.3, seed + 2)])


@pytest.mark.parametrize("obj", sorted(OBJS))
@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("B,xd,kernel", [(8, 0, None), (32, 0, None), (32, 1, "generic"), (64, 2, "wide"),
                                         (128, 1, None)])
def test_plain_steps_objective(mq, monkeypatch, obj, weighted, B, xd, kernel):
    if kernel:
        monkeypatch.setenv("MQO_STEP_KERNEL", kernel)
    G = cut_batch(B + OBJS[obj])
    if weighted:
        G = signed(G, B)
    p = mq.params(problem=1, batch=B, x_dtype=xd, alpha=0.02, momentum=0.7, lambda_=0.05, init_kind=0,
                  objective=OBJS[obj], seed=B + 3)
    _plain_steps(mq, G, p, 12)


@pytest.mark.parametrize("obj", sorted(OBJS))
@pytest.mark.parametrize("weighted", [False, True])
def test_machine_objective(mq, obj, weighted):
    G = mi.pack([mi.random_regular(80, 3, 5), mi.erdos_renyi(60, 0.1, 6)])
    if weighted:
        G = signed(G, 7)
    p = mq.params(problem=1, batch=8, alpha=0.05, momentum=0.8, lambda_=0.001, rho=0.8, t_gs=3, descent_cap=60,
                  init_kind=1, sigma=0.2, objective=OBJS[obj], seed=8)
    _machine(mq, G, p, 500, trace=30)


@pytest.mark.parametrize("obj", sorted(OBJS))
def test_objective_f64_relaxations(mq, obj):
    G = signed(cut_batch(4), 4)
    B = 8
    lam = 0.01
    p = mq.params(problem=1, batch=B, lambda_=lam, alpha=0.05, momentum=0.5, objective=OBJS[obj], seed=7)
    s = mq.Solver(mq.Graph(G), p)
    s.step(3)
    got = host(s.objective_f64())
    x = host(s.get_x())
    for g, og in enumerate(oracle_graphs(G)):
        lo, hi = int(G.node_offsets[g]), int(G.node_offsets[g + 1])
        deg = np.diff(og.row_ptr)
        dmax = int(deg.max())
        for b in range(B):
            xb = x[lo:hi, b].astype(np.float64)
            want = oracle.cut_objective_f64(og, OBJS[obj], lam, xb)
            # (Ax)_v in float32 (relative error <= d(v) 2^-24), the rest in double
            scale = float(np.abs(xb).sum() * (dmax + 1) * (1 + np.abs(xb).max()) + (deg * xb * xb).sum())
            assert abs(got[g * B + b] - want) <= 1e-7 * dmax * scale + 1e-12, (g, b)


def test_fl_interior_point_stays(mq):
    """Prop. 3.2: x = c 1 is a stationary point of f_L (its gradient 1/2 Lx
    vanishes); from there the fused step leaves x exactly in place and the
    rounded point (all in S for c > 0) has cut 0."""
    G = mi.pack([mi.random_regular(60, 3, 1), mi.erdos_renyi(50, 0.2, 2)])
    B = 8
    p = mq.params(problem=1, batch=B, alpha=0.3, momentum=0.5, objective=OBJS["f_L"], seed=1)
    s = mq.Solver(mq.Graph(G), p)
    x0 = torch.full((G.n, B), 0.25, dtype=torch.float32, device="cuda")
    s.set_x(x0)
    for _ in range(5):
        s.step(1)
        assert torch.equal(s.get_x(), x0)
    v, a, c = (host(t) for t in s.step_stats())
    assert (v == 0).all()

"""f_B as a differentiable objective: forward, fused-SpMM backward, optimisers.

The backward (grad f_B = -lambda 1 - 2 A x, proof of Thm 3.6) is checked
against the oracle's float64 gradient, against central finite differences
(h = 1e-3) and through torch.autograd; the projected momentum / Adam kernels
against torch.optim's SGD(momentum) / Adam followed by a clamp.
"""
import numpy as np
import pytest

import mqo_inputs as mi
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mq():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2605_06921_gb300 as m
    return m


def power_law_with_hub(n=20000, hub=3000, seed=0):
    """Chung–Lu graph plus a star whose centre has degree > the chunk split."""
    cl = mi.chung_lu(n, 2.5, 8.0, seed)
    star = mi.from_edges(hub + 1, np.zeros(hub, int), np.arange(1, hub + 1))
    G = mi.pack([cl, star])
    return mi.Graph(G.n, G.row_ptr, G.col_idx, None)  # one graph (block diagonal)


@pytest.fixture(scope="module")
def graph_and_x():
    G = power_law_with_hub()
    rng = np.random.default_rng(0)
    B = 8
    X = (rng.random((G.n, B)) * 2 - 1).astype(np.float32)
    return G, X, B


def test_forward_matches_oracle(mq, graph_and_x):
    G, X, B = graph_and_x
    assert G.degrees().max() > 512  # chunked rows are exercised
    g = mq.Graph(G)
    lam = 0.001
    obj = mq.fb_forward(g, torch.from_numpy(X).cuda(), lam).cpu().numpy()
    og = oracle.Graph(G)
    for b in range(B):
        want = oracle.objective_f64(og, oracle.MAXCUT, 0.0, lam, X[:, b].astype(np.float64))
        assert obj[b] == pytest.approx(want, rel=2e-6, abs=1e-3)


def test_backward_matches_oracle_gradient(mq, graph_and_x):
    G, X, B = graph_and_x
    g = mq.Graph(G)
    lam = 0.001
    gout = torch.linspace(0.5, 2.0, B, device="cuda")
    Gr = mq.spmm_grad(g, torch.from_numpy(X).cuda(), lam, gout).cpu().numpy()
    og = oracle.Graph(G)
    go = gout.cpu().numpy().astype(np.float64)
    for b in range(B):
        want = go[b] * oracle.gradient_f64(og, oracle.MAXCUT, 0.0, lam, X[:, b].astype(np.float64))
        assert np.allclose(Gr[:, b], want, rtol=1e-5, atol=1e-4)


def test_backward_central_differences(mq, graph_and_x):
    G, X, B = graph_and_x
    g = mq.Graph(G)
    lam = 0.001
    rng = np.random.default_rng(1)
    Xt = torch.from_numpy(X).cuda()
    Gr = mq.spmm_grad(g, Xt, lam).double()
    og = oracle.Graph(G)
    h = 1e-3
    for _ in range(3):
        D = torch.from_numpy(rng.standard_normal(X.shape).astype(np.float32)).cuda()
        want = (Gr * D.double()).sum(dim=0).cpu().numpy()
        Xp = (Xt.double() + h * D.double()).cpu().numpy()
        Xm = (Xt.double() - h * D.double()).cpu().numpy()
        for b in range(B):
            fd = (oracle.objective_f64(og, 1, 0.0, lam, Xp[:, b]) - oracle.objective_f64(og, 1, 0.0, lam, Xm[:, b])) / (2 * h)
            assert fd == pytest.approx(want[b], rel=1e-5, abs=1e-3)
        # the GPU forward's own finite differences (float32 terms, double sums)
        fp = mq.fb_forward(g, (Xt + h * D).contiguous(), lam).cpu().numpy()
        fm = mq.fb_forward(g, (Xt - h * D).contiguous(), lam).cpu().numpy()
        assert np.allclose((fp - fm) / (2 * h), want, rtol=2e-2, atol=1.0)


def test_autograd_function(mq, graph_and_x):
    G, X, B = graph_and_x
    g = mq.Graph(G)
    lam = 0.002
    Xt = torch.from_numpy(X).cuda().requires_grad_(True)
    w = torch.arange(1, B + 1, device="cuda", dtype=torch.float64)
    loss = (mq.FbObjective.apply(Xt, g, lam) * w).sum()
    loss.backward()
    want = mq.spmm_grad(g, Xt.detach(), lam, w.float())
    assert torch.equal(Xt.grad, want)


def test_momentum_and_adam_match_torch(mq, graph_and_x):
    G, X, B = graph_and_x
    g = mq.Graph(G)
    lam = 0.001
    x0 = torch.from_numpy(X).cuda()
    for kind in ("momentum", "adam"):
        xa = x0.clone().requires_grad_(True)
        xb = x0.clone().requires_grad_(True)
        if kind == "momentum":
            oa = mq.PGAMomentum([xa], lr=0.003, momentum=0.8)
            ob = torch.optim.SGD([xb], lr=0.003, momentum=0.8)
        else:
            oa = mq.PGAAdam([xa], lr=0.01)
            ob = torch.optim.Adam([xb], lr=0.01)
        for _ in range(5):
            oa.zero_grad()
            mq.FbObjective.apply(xa, g, lam).sum().backward()
            oa.step()
            ob.zero_grad()
            xb.grad = -mq.spmm_grad(g, xb.detach(), lam)  # torch minimises -f
            ob.step()
            with torch.no_grad():
                xb.clamp_(-1.0, 1.0)
        assert torch.allclose(xa, xb, rtol=1e-5, atol=1e-5), kind


@pytest.mark.parametrize("B,signed", [(32, False), (64, False), (64, True), (128, False), (256, True)])
def test_pipelined_kernel_equals_unit_kernel_and_oracle(mq, monkeypatch, B, signed):
    """B >= 32 takes the warp-pipelined kernel (neighbour rows staged through
    shared memory a batch ahead): its gradient equals the unit kernel's bit
    for bit (same CSR-order sums per row and per 512-entry chunk) and the
    oracle's float64 gradient within the float32 rounding of the sums; its
    objective matches the oracle's."""
    G = power_law_with_hub(6000, 1500, seed=B)
    if signed:
        rows, cols = G.edges_directed()
        up = rows < cols
        w = np.random.default_rng(B).choice(np.array([-1, 1], dtype=np.int8), size=int(up.sum()))
        G = mi.from_edges(G.n, rows[up], cols[up], w)
    assert G.degrees().max() > 512
    g = mq.Graph(G)
    lam = 0.001
    Xh = (np.random.default_rng(B + 1).random((G.n, B)) * 2 - 1).astype(np.float32)
    X = torch.from_numpy(Xh).cuda()
    gout = torch.linspace(0.5, 2.0, B, device="cuda")
    got = mq.spmm_grad(g, X, lam, gout)
    obj = mq.fb_forward(g, X, lam).cpu().numpy()
    monkeypatch.setenv("MQO_FB_KERNEL", "units")
    want_units = mq.spmm_grad(g, X, lam, gout)
    monkeypatch.delenv("MQO_FB_KERNEL")
    torch.cuda.synchronize()
    assert torch.equal(got, want_units)
    og = oracle.Graph(G)
    gh = got.cpu().numpy().astype(np.float64)
    deg = np.diff(G.row_ptr)
    rows = np.repeat(np.arange(G.n), deg)
    go = gout.cpu().numpy().astype(np.float64)
    for b in range(0, B, max(1, B // 8)):
        xb = Xh[:, b].astype(np.float64)
        want = oracle.gradient_f64(og, oracle.MAXCUT, 0.0, lam, xb) * go[b]
        absum = np.bincount(rows, weights=np.abs(Xh[G.col_idx, b].astype(np.float64)), minlength=G.n)
        assert np.all(np.abs(gh[:, b] - want) <= 1e-5 * go[b] * (lam + 2 * absum) + 1e-7), b
        wobj = oracle.objective_f64(og, oracle.MAXCUT, 0.0, lam, xb)
        assert obj[b] == pytest.approx(wobj, rel=2e-6, abs=1e-3), b


def test_misaligned_block_is_rejected(mq):
    """B >= 32 reads rows of X in 16-byte pieces: a pointer off that
    boundary is an argument error (nothing launched), not a fault."""
    G = power_law_with_hub(2000, 600, seed=3)
    g = mq.Graph(G)
    buf = torch.zeros(G.n * 32 + 1, device="cuda")
    X = buf[1:].view(G.n, 32)
    with pytest.raises(Exception, match="16-byte aligned"):
        mq.fb_forward(g, X, 0.001)
    with pytest.raises(Exception, match="16-byte aligned"):
        mq.spmm_grad(g, X, 0.001)

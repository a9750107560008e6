"""Pins of the oracle's four MaxCut relaxations (Sec. 3: f_L of Eq. 4,
f_P of Eq. 5, f_A of Eq. 6, f_B of
Eq. 7) against their definitions and the paper's statements
about their fixed points (Prop. 3.2, Thm 3.3, Prop. 3.4, Thm 3.6)."""
import itertools

import numpy as np
import pytest

import mqo_inputs as mi
import oracle

OBJ = {"f_B": oracle.F_B, "f_L": oracle.F_L, "f_P": oracle.F_P, "f_A": oracle.F_A}
LAM = 0.001


def signed(G, seed):
    rng = np.random.default_rng(seed)
    rows, cols = G.edges_directed()
    keep = rows < cols
    return mi.from_edges(G.n, rows[keep], cols[keep], np.where(rng.random(int(keep.sum())) < 0.5, -1, 1))


@pytest.mark.parametrize("name", list(OBJ))
@pytest.mark.parametrize("weighted", [False, True])
def test_gradient_matches_central_differences(name, weighted):
    G = mi.erdos_renyi(40, 0.2, 3)
    if weighted:
        G = signed(G, 4)
    g = oracle.Graph(G)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, G.n)
    grad = oracle.cut_gradient_f64(g, OBJ[name], LAM, x)
    h = 1e-3
    for v in range(0, G.n, 3):
        e = np.zeros(G.n)
        e[v] = h
        fd = (oracle.cut_objective_f64(g, OBJ[name], LAM, x + e) - oracle.cut_objective_f64(g, OBJ[name], LAM, x - e)) / (2 * h)
        assert abs(fd - grad[v]) <= 1e-8 * max(1.0, abs(grad[v]))  # quadratic: exact up to rounding


@pytest.mark.parametrize("weighted", [False, True])
def test_binary_values_are_affine_in_the_cut(weighted):
    # on s in {-1,1}^n: f_L = cut, f_P = 4 cut + lambda n, f_A = 4 cut - 2 W
    G = mi.erdos_renyi(30, 0.25, 8)
    if weighted:
        G = signed(G, 9)
    g = oracle.Graph(G)
    W = int(np.asarray(G.weights if G.weights is not None else np.ones(G.nnz)).sum()) // 2
    rng = np.random.default_rng(1)
    for _ in range(20):
        z = rng.integers(0, 2, G.n).astype(np.uint8)
        s = np.where(z == 1, 1.0, -1.0)
        cut = oracle.eval_cut(g, z)[0]
        assert oracle.cut_objective_f64(g, oracle.F_L, LAM, s) == pytest.approx(cut, abs=1e-9)
        assert oracle.cut_objective_f64(g, oracle.F_P, LAM, s) == pytest.approx(4 * cut + LAM * G.n, abs=1e-9)
        assert oracle.cut_objective_f64(g, oracle.F_A, LAM, s) == pytest.approx(4 * cut - 2 * W, abs=1e-9)


@pytest.mark.parametrize("name", list(OBJ))
@pytest.mark.parametrize("weighted", [False, True])
def test_fixed_point_rule_is_the_projection_test(name, weighted):
    """For every binary point of small graphs: the integer rule of the
    evaluation counts exactly the coordinates that a PGA step moves."""
    for seed in range(3):
        G = mi.erdos_renyi(9, 0.4, seed)
        if weighted:
            G = signed(G, seed + 20)
        g = oracle.Graph(G)
        for bits in itertools.product([0, 1], repeat=G.n):
            z = np.array(bits, dtype=np.uint8)
            s = np.where(z == 1, 1.0, -1.0)
            grad = oracle.cut_gradient_f64(g, OBJ[name], LAM, s)
            moved = int(np.count_nonzero(np.clip(s + 0.1 * grad, -1, 1) != s))
            assert oracle.eval_cut_obj(g, z, OBJ[name], LAM)[1] == moved


@pytest.mark.parametrize("name", ["f_L", "f_P"])
def test_every_binary_point_is_fixed(name):
    # f_P: Thm 3.3; f_L: boundary fixed points of Prop. 3.2 -- PGA cannot
    # leave a binary point, not even a 1-flip repairable one
    G = mi.erdos_renyi(10, 0.5, 2)
    g = oracle.Graph(G)
    for bits in itertools.product([0, 1], repeat=G.n):
        assert oracle.eval_cut_obj(g, np.array(bits, dtype=np.uint8), OBJ[name], LAM)[1] == 0
    p = oracle.params(problem=1, alpha=0.1, momentum=0.0, lambda_=LAM, objective=OBJ[name])
    rng = np.random.default_rng(0)
    x = np.where(rng.integers(0, 2, G.n) == 1, 1.0, -1.0).astype(np.float32)
    xn, Vn, _, _ = oracle.descent_step(g, p, x, np.zeros(G.n, np.float32))
    assert np.array_equal(xn, x)


@pytest.mark.parametrize("name", ["f_A", "f_B"])
def test_one_flip_repairable_points_are_not_fixed(name):
    # Prop. 3.4 (f_A) and Thm 3.6 (f_B): a binary point with a positive
    # 1-flip gain is not a PGA fixed point
    G = mi.erdos_renyi(10, 0.5, 6)
    g = oracle.Graph(G)
    n_rep = 0
    for bits in itertools.product([0, 1], repeat=G.n):
        cut, nonfixed, cand = oracle.eval_cut_obj(g, np.array(bits, dtype=np.uint8), OBJ[name], LAM)
        if cand > 0:
            n_rep += 1
            assert nonfixed > 0
    assert n_rep > 0


def test_laplacian_interior_stationary_point_keeps_cut_zero():
    # Prop. 3.2 (ii): x = c 1 is stationary for f_L (L 1 = 0).  With a dyadic
    # c every sum is exact in float32, so PGA does not move at all.
    G = mi.erdos_renyi(100, 0.66, 1)
    g = oracle.Graph(G)
    p = oracle.params(problem=1, alpha=0.1, momentum=0.0, lambda_=LAM, objective=oracle.F_L)
    for c in (0.25, -0.375, 0.5):
        x = np.full(G.n, c, dtype=np.float32)
        V = np.zeros(G.n, np.float32)
        for _ in range(50):
            x, V, z, ev = oracle.descent_step(g, p, x, V)
            assert ev[0] == 0
        assert np.all(x == np.float32(c))


def test_perturbed_laplacian_leaves_the_interior_point():
    # f_P's gradient at c 1 is 2 lambda c 1 != 0: PGA moves towards the box corner
    G = mi.erdos_renyi(100, 0.66, 1)
    g = oracle.Graph(G)
    p = oracle.params(problem=1, alpha=0.1, momentum=0.0, lambda_=LAM, objective=oracle.F_P)
    x = np.full(G.n, 0.25, dtype=np.float32)
    V = np.zeros(G.n, np.float32)
    xn, _, _, _ = oracle.descent_step(g, p, x, V)
    assert np.all(xn > x)


@pytest.mark.parametrize("name", list(OBJ))
def test_float_step_follows_the_f64_gradient(name):
    G = signed(mi.erdos_renyi(60, 0.1, 12), 13)
    g = oracle.Graph(G)
    p = oracle.params(problem=1, alpha=0.05, momentum=0.0, lambda_=LAM, objective=OBJ[name])
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, G.n).astype(np.float32)
    xn, _, _, _ = oracle.descent_step(g, p, x, np.zeros(G.n, np.float32))
    want = np.clip(x.astype(np.float64) + 0.05 * oracle.cut_gradient_f64(g, OBJ[name], LAM, x.astype(np.float64)), -1, 1)
    assert np.allclose(xn, want, rtol=0, atol=2e-5)

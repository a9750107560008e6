"""Local search in the paper's scan order (restart after each move) beside
the round-based variant the machine runs: both end at points with the
defining properties of OneTwoSwap / OneTwoFlip (Defs. 2.3-2.5), checked here
from the definitions: independent, maximal and free of (1,2)-swaps; free of
improving 1-flips and 2-flips; every swap adds exactly one node; every move
raises the cut; never above the brute-force optimum."""
import itertools

import numpy as np
import pytest

import mqo_inputs as mi
import oracle


def nbrs(G):
    return [set(G.col_idx[G.row_ptr[v]:G.row_ptr[v + 1]].tolist()) for v in range(G.n)]


def swap_free(N, z):
    S = {v for v in range(len(z)) if z[v]}
    for v in S:
        tight = [u for u in N[v] if u not in S and len(N[u] & S) == 1]
        for a, b in itertools.combinations(tight, 2):
            if b not in N[a]:
                return False
    return True


def random_independent(G, rng, keep=0.5):
    z = np.zeros(G.n, dtype=np.uint8)
    for v in rng.permutation(G.n):
        nb = G.col_idx[G.row_ptr[v]:G.row_ptr[v + 1]]
        if rng.random() < keep and not z[nb].any():
            z[v] = 1
    return z


@pytest.mark.parametrize("seed", range(6))
def test_mis_sequential_end_state(seed):
    G = mi.erdos_renyi(70, 0.08 + 0.02 * seed, seed)
    g = oracle.Graph(G)
    N = nbrs(G)
    rng = np.random.default_rng(seed)
    z0 = random_independent(G, rng)
    z, swaps, adds = oracle.ls_mis_sequential(g, z0)
    size, conf_e, conf_n, unc = oracle.eval_mis(g, z)
    assert conf_e == 0 and unc == 0            # independent and maximal
    assert swap_free(N, z)
    assert size == int(z0.sum()) + adds + swaps  # each swap adds exactly one node
    # the round-based variant (completion, then swap rounds until one applies nothing)
    zr = z0.copy()
    while True:
        while oracle.eval_mis(g, zr)[3] > 0:
            zr, _ = oracle.round_complete(g, zr)
        zr, k = oracle.round_swap(g, zr)
        if k == 0 and oracle.eval_mis(g, zr)[3] == 0:
            break
    assert oracle.eval_mis(g, zr)[1:] == (0, 0, 0) and swap_free(N, zr)


@pytest.mark.parametrize("seed", range(4))
def test_mis_sequential_never_beats_brute_force(seed):
    G = mi.erdos_renyi(18, 0.25, 100 + seed)
    g = oracle.Graph(G)
    z, _, _ = oracle.ls_mis_sequential(g, np.zeros(G.n, dtype=np.uint8))
    assert oracle.eval_mis(g, z)[0] <= oracle.brute_mis(g)


def cut_and_gains(G, z):
    s = np.where(z == 1, 1, -1)
    w = np.ones(G.nnz, dtype=np.int64) if G.weights is None else G.weights.astype(np.int64)
    rows = np.repeat(np.arange(G.n), np.diff(G.row_ptr))
    As = np.bincount(rows, weights=w * s[G.col_idx], minlength=G.n).astype(np.int64)
    return s, As, w, rows


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_cut_sequential_end_state(weighted, seed):
    G = mi.erdos_renyi(60, 0.1, 10 + seed)
    if weighted:
        r, c = G.edges_directed()
        k = r < c
        w = np.where(np.random.default_rng(seed).random(int(k.sum())) < 0.5, -1, 1)
        G = mi.from_edges(G.n, r[k], c[k], w)
    g = oracle.Graph(G)
    z0 = (np.random.default_rng(seed).random(G.n) < 0.5).astype(np.uint8)
    z, moves = oracle.ls_cut_sequential(g, z0)
    cut0, cut1 = oracle.eval_cut(g, z0)[0], oracle.eval_cut(g, z)[0]
    assert cut1 - cut0 >= moves                 # integer weights: every move gains at least 1
    s, As, w, rows = cut_and_gains(G, z)
    gain = s * As
    assert np.all(gain <= 0)                    # no improving 1-flip
    pair = gain[rows] + gain[G.col_idx] + 2 * w  # 2-flip of edge (rows, col) across the cut
    across = z[rows] != z[G.col_idx]
    assert not np.any(pair[across] > 0)         # no improving 2-flip


@pytest.mark.parametrize("seed", range(3))
def test_cut_sequential_never_beats_brute_force(seed):
    G = mi.erdos_renyi(16, 0.3, 200 + seed)
    g = oracle.Graph(G)
    z, _ = oracle.ls_cut_sequential(g, np.zeros(G.n, dtype=np.uint8))
    assert oracle.eval_cut(g, z)[0] <= oracle.brute_maxcut(g)

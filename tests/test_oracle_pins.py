"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test ties one oracle function to a library routine, a closed form, the
paper's literal definition, a theorem of the paper, or brute force, chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails.
"""
import itertools
import math
import os

import numpy as np
import pytest

import mqo_inputs as mi
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_graph(n, p, seed):
    return oracle.Graph(mi.erdos_renyi(n, p, seed))


def dense_adj(g):
    A = np.zeros((g.n, g.n))
    for v in range(g.n):
        for j in range(g.row_ptr[v], g.row_ptr[v + 1]):
            A[v, g.col[j]] = 1.0 if g.w is None else float(g.w[j])
    return A


# ---------------------------------------------------------------- Philox
def test_philox_matches_numpy_philox4x64():
    """numpy.random.Philox is Philox4x64-10; it increments its 256-bit
    counter before each block, so counter c-1 there yields block c here."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        key = rng.integers(0, 2**63, size=2, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
        ctr = rng.integers(1, 2**63, size=4, dtype=np.uint64)
        bg = np.random.Philox(key=key, counter=ctr - np.array([1, 0, 0, 0], dtype=np.uint64))
        want = bg.random_raw(4)
        got = oracle.philox4x64_10(ctr, key)
        assert np.array_equal(got, want)


# ---------------------------------------------------------------- storage rounding
def _special_floats(rng, k):
    bits = rng.integers(0, 2**32, size=k, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    f = f[np.isfinite(f)]
    small = (rng.random(k) * 2.0 - 1.0).astype(np.float32) * np.float32(2.0 ** -20)  # fp16 subnormals
    mid = (rng.random(k) * 4.0 - 2.0).astype(np.float32)
    return np.concatenate([f, small, mid, np.float32([0.5, 1.0, -1.0, 65504.0, 65519.0, 65520.0, 2.0 ** -24,
                                                      2.0 ** -25, 3 * 2.0 ** -25, 1.0 + 2.0 ** -11])])


def test_round_store_f16_matches_numpy():
    rng = np.random.default_rng(1)
    xs = _special_floats(rng, 4000)
    want = xs.astype(np.float16).astype(np.float32)
    got = np.array([oracle.round_store(float(x), oracle.F16) for x in xs], dtype=np.float32)
    assert np.array_equal(got, want, equal_nan=True)


def test_round_store_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    xs = _special_floats(rng, 4000)
    want = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.round_store(float(x), oracle.BF16) for x in xs], dtype=np.float32)
    assert np.array_equal(got, want, equal_nan=True)


# ---------------------------------------------------------------- evaluation
def _indep_maximal(A, z):
    zs = np.asarray(z, dtype=bool)
    indep = not np.any(A[np.ix_(zs, zs)])
    cov = A[:, zs].sum(axis=1) > 0
    maximal = bool(np.all(zs | cov))
    return indep, maximal


def test_mis_checker_is_maximal_independent_set_exhaustive():
    """Checker of Eq. 8 <=> maximal independent set, over all
    2^n binary points of small graphs (Prop. 3.1 and its derivation)."""
    for seed in range(6):
        g = small_graph(9, 0.35, seed)
        A = dense_adj(g)
        for bits in range(1 << g.n):
            z = np.array([(bits >> i) & 1 for i in range(g.n)], dtype=np.uint8)
            size, conf_e, conf_n, unc = oracle.eval_mis(g, z)
            indep, maximal = _indep_maximal(A, z)
            assert size == int(z.sum())
            assert conf_e == int(z @ A @ z) // 2
            assert (conf_n == 0) == indep
            assert (conf_n == 0 and unc == 0) == (indep and maximal)


def test_mis_checker_equals_literal_pga_fixed_point():
    """1{z == Pi_[0,1](z + alpha grad h(z))} computed literally in float64."""
    rng = np.random.default_rng(3)
    for seed in range(4):
        g = small_graph(10, 0.3, 100 + seed)
        A = dense_adj(g)
        for _ in range(200):
            z = (rng.random(g.n) < 0.3).astype(np.uint8)
            gamma = 1.0 + rng.random() * 3.0 + 1e-3
            alpha = 0.05 + rng.random()
            grad = 1.0 - gamma * (A @ z)
            lit = np.array_equal(np.clip(z + alpha * grad, 0.0, 1.0), z.astype(float))
            _, _, conf_n, unc = oracle.eval_mis(g, z)
            assert lit == (conf_n == 0 and unc == 0)


def test_cut_value_two_ways_and_fb_fixed_point_literal():
    """cut = #crossing edges = f_L(s) = 1/4 s^T L s (Eq. 4); non-fixed
    count = #coordinates moved by Pi(s + alpha grad f_B(s)) (Thm 3.6)."""
    rng = np.random.default_rng(4)
    for seed in range(4):
        for signed in (False, True):
            base = mi.erdos_renyi(12, 0.4, 200 + seed)
            if signed:
                rows, cols = base.edges_directed()
                keep = rows < cols
                w = np.where(rng.random(int(keep.sum())) < 0.5, -1, 1)
                base = mi.from_edges(12, rows[keep], cols[keep], w)
            g = oracle.Graph(base)
            A = dense_adj(g)
            L = np.diag(A.sum(axis=1)) - A
            for _ in range(100):
                z = (rng.random(g.n) < 0.5).astype(np.uint8)
                s = np.where(z == 1, 1.0, -1.0)
                cut, nonfixed, cand = oracle.eval_cut(g, z)
                crossing = sum(A[u, v] for u in range(g.n) for v in range(u + 1, g.n) if z[u] != z[v])
                assert cut == int(crossing)
                assert cut == int(round(0.25 * s @ L @ s))
                lam = 0.001 + rng.random() * 1.9
                alpha = 0.01 + rng.random()
                grad = -lam - 2.0 * (A @ s)
                moved = np.clip(s + alpha * grad, -1, 1) != s
                assert nonfixed == int(moved.sum())
                gains = s * (A @ s)
                assert cand == int((gains > 0).sum())


def test_one_flip_gain_identity():
    """f_A(x^(i)) - f_A(x) = 4 x_i (Ax)_i (proof of Prop. 3.4); the cut
    change of flipping i equals x_i (Ax)_i."""
    rng = np.random.default_rng(5)
    g = small_graph(15, 0.3, 9)
    A = dense_adj(g)
    for _ in range(50):
        z = (rng.random(g.n) < 0.5).astype(np.uint8)
        s = np.where(z == 1, 1.0, -1.0)
        i = int(rng.integers(g.n))
        s2 = s.copy(); s2[i] = -s2[i]
        fa = oracle.objective_f64(g, oracle.MAXCUT, 0.0, 0.0, s)
        fa2 = oracle.objective_f64(g, oracle.MAXCUT, 0.0, 0.0, s2)
        assert fa2 - fa == pytest.approx(4 * s[i] * (A @ s)[i], abs=1e-9)
        z2 = z.copy(); z2[i] ^= 1
        assert oracle.eval_cut(g, z2)[0] - oracle.eval_cut(g, z)[0] == int(s[i] * (A @ s)[i])


def _golden_k3():
    edges, s = [], None
    vals = {}
    with open(os.path.join(GOLDEN, "k3_fa_plateau.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            t = line.split()
            if t[0] == "n":
                n = int(t[1])
            elif t[0] == "e":
                edges.append((int(t[1]), int(t[2])))
            elif t[0] == "s":
                s = np.array([float(v) for v in t[1:]])
            else:
                vals[t[0]] = float(t[1])
    u, v = zip(*edges)
    return n, mi.from_edges(n, u, v), s, vals


def test_k3_worked_example_fa_plateau():
    n, G, s, vals = _golden_k3()
    g = oracle.Graph(G)
    for t in np.linspace(-1, 1, 11):
        x = s.copy(); x[0] = t
        assert oracle.objective_f64(g, oracle.MAXCUT, 0.0, 0.0, x) == pytest.approx(vals["fa"], abs=1e-12)
    z = (s > 0).astype(np.uint8)
    assert oracle.eval_cut(g, z)[0] == int(vals["cut"])


# ---------------------------------------------------------------- brute force
def _closed_form_graph(kind, n):
    if kind == "cycle":
        return mi.from_edges(n, np.arange(n), (np.arange(n) + 1) % n)
    if kind == "complete":
        u, v = np.triu_indices(n, 1)
        return mi.from_edges(n, u, v)
    if kind == "empty":
        return mi.from_edges(n, [], [])
    if kind == "petersen":
        outer = [(i, (i + 1) % 5) for i in range(5)]
        inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
        spokes = [(i, i + 5) for i in range(5)]
        u, v = zip(*(outer + inner + spokes))
        return mi.from_edges(10, u, v)
    if kind == "bipartite34":
        u, v = zip(*[(a, 3 + b) for a in range(3) for b in range(4)])
        return mi.from_edges(7, u, v)
    raise ValueError(kind)


def test_brute_force_closed_forms():
    with open(os.path.join(GOLDEN, "closed_forms.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for kind, n, a, mc in rows:
        g = oracle.Graph(_closed_form_graph(kind, int(n)))
        assert oracle.brute_mis(g) == int(a), kind
        assert oracle.brute_maxcut(g) == int(mc), kind


# ---------------------------------------------------------------- gradients / step
def test_gradients_match_central_differences():
    """Objectives are quadratic, so central differences are exact up to
    rounding: (f(x+h d) - f(x-h d)) / 2h = grad . d, h = 1e-3."""
    rng = np.random.default_rng(6)
    for problem, lo in ((oracle.MIS, 0.0), (oracle.MAXCUT, -1.0)):
        for signed in (False, True):
            base = mi.erdos_renyi(40, 0.2, 11)
            if signed:
                rows, cols = base.edges_directed()
                keep = rows < cols
                base = mi.from_edges(40, rows[keep], cols[keep],
                                     np.where(rng.random(int(keep.sum())) < 0.5, -1, 1))
            g = oracle.Graph(base)
            for _ in range(10):
                x = lo + (1 - lo) * rng.random(g.n)
                d = rng.standard_normal(g.n)
                gamma, lam = 1.7, 0.001
                h = 1e-3
                fp = oracle.objective_f64(g, problem, gamma, lam, x + h * d)
                fm = oracle.objective_f64(g, problem, gamma, lam, x - h * d)
                grad = oracle.gradient_f64(g, problem, gamma, lam, x)
                assert (fp - fm) / (2 * h) == pytest.approx(grad @ d, rel=1e-9, abs=1e-9)


def test_descent_step_closed_form_float64():
    """x' = Pi(x + mu V + alpha grad) with grad h = 1 - gamma A x or grad f_B =
    -lambda - 2 A x, computed in float64; the float32 oracle agrees to 1e-6."""
    rng = np.random.default_rng(8)
    G = mi.erdos_renyi(60, 0.15, 12)
    g = oracle.Graph(G)
    A = dense_adj(g)
    for problem, lo in ((oracle.MIS, 0.0), (oracle.MAXCUT, -1.0)):
        p = oracle.params(problem=problem, alpha=0.3, momentum=0.6, gamma=2.5, lambda_=0.01)
        x = (lo + (1 - lo) * rng.random(g.n)).astype(np.float32)
        V = (0.1 * rng.standard_normal(g.n)).astype(np.float32)
        xn, Vn, z, ev = oracle.descent_step(g, p, x, V)
        x64, V64 = x.astype(np.float64), V.astype(np.float64)
        grad = 1.0 - 2.5 * (A @ x64) if problem == oracle.MIS else -0.01 - 2.0 * (A @ x64)
        Vw = 0.6 * V64 + 0.3 * grad
        xw = np.clip(x64 + Vw, lo, 1.0)
        assert np.allclose(Vn, Vw, rtol=1e-5, atol=1e-6)
        assert np.allclose(xn, xw, rtol=1e-5, atol=1e-6)
        thr = 0.5 if problem == oracle.MIS else 0.0
        assert np.array_equal(z, (x > thr).astype(np.uint8))


def test_prop31_maximal_sets_are_pga_fixed():
    """Prop. 3.1: every maximal independent set (incl. (1,2)-swap repairable
    ones) is a fixed point of projected gradient ascent on h."""
    rng = np.random.default_rng(9)
    for seed in range(5):
        G = mi.erdos_renyi(30, 0.15, 300 + seed)
        g = oracle.Graph(G)
        z = np.zeros(g.n, dtype=np.uint8)
        for v in rng.permutation(g.n):   # random greedy maximal IS
            if not any(z[g.col[j]] for j in range(g.row_ptr[v], g.row_ptr[v + 1])):
                z[v] = 1
        p = oracle.params(alpha=float(0.1 + rng.random()), momentum=0.0, gamma=float(1.01 + rng.random()))
        x = z.astype(np.float32)
        xn, _, _, ev = oracle.descent_step(g, p, x, np.zeros(g.n, np.float32))
        assert np.array_equal(xn, x)
        assert ev[1] == 0 and ev[2] == 0


def test_thm36_one_flip_repairable_points_move_under_fb():
    """Thm 3.6(i): a 1-flip repairable binary point is not PGA-fixed for f_B."""
    rng = np.random.default_rng(10)
    G = mi.erdos_renyi(30, 0.2, 13)
    g = oracle.Graph(G)
    A = dense_adj(g)
    checked = 0
    for _ in range(100):
        z = (rng.random(g.n) < 0.5).astype(np.uint8)
        s = np.where(z == 1, 1.0, -1.0)
        if not np.any(s * (A @ s) > 0):
            continue
        p = oracle.params(problem=oracle.MAXCUT, alpha=0.01, momentum=0.0, lambda_=0.001)
        xn, _, _, ev = oracle.descent_step(g, p, s.astype(np.float32), np.zeros(g.n, np.float32))
        assert not np.array_equal(xn, s.astype(np.float32))
        assert ev[1] > 0
        checked += 1
    assert checked > 50


# ---------------------------------------------------------------- reset set
def test_feistel_is_a_bijection_and_reset_size_exact():
    rng = np.random.default_rng(11)
    for n in list(range(1, 70)) + [127, 128, 129, 200, 750, 1000, 1025]:
        keys = rng.integers(0, 2**32, size=6, dtype=np.uint64).astype(np.uint32)
        sig = [oracle.feistel_sigma(n, keys, v) for v in range(n)]
        assert sorted(sig) == list(range(n))
        for rho in (0.0, 0.3, 0.5, 0.7, 0.8, 0.999):
            m = oracle.reset_mask(n, rho, 5, 3, 1, 2)
            assert int(m.sum()) == math.floor(rho * n)


def test_reset_set_uniform_chi_square():
    """|R| = 3 of n = 7: all C(7,3) = 35 subsets equally likely."""
    counts = {}
    trials = 7000
    for t in range(trials):
        m = oracle.reset_mask(7, 3.5 / 7, 2024, t, 0, 1)
        key = tuple(np.nonzero(m)[0])
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 35
    exp = trials / 35
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 80.0  # 34 d.o.f.: P(chi2 > 80) < 1e-5
    # every node has inclusion frequency 3/7
    inc = np.zeros(7)
    for key, c in counts.items():
        inc[list(key)] += c
    assert np.allclose(inc / trials, 3 / 7, atol=0.03)


# ---------------------------------------------------------------- discrete rounds
def _tight_pairs_exist(g, z):
    n = g.n
    c = np.array([sum(z[g.col[j]] for j in range(g.row_ptr[v], g.row_ptr[v + 1])) for v in range(n)])
    for v in range(n):
        if not z[v]:
            continue
        t = [g.col[j] for j in range(g.row_ptr[v], g.row_ptr[v + 1]) if not z[g.col[j]] and c[g.col[j]] == 1]
        for a, b in itertools.combinations(t, 2):
            if b not in set(g.col[g.row_ptr[a]:g.row_ptr[a + 1]]):
                return True
    return False


def test_repair_and_swap_rounds_invariants():
    rng = np.random.default_rng(12)
    for seed in range(8):
        G = mi.erdos_renyi(40, 0.12, 400 + seed)
        g = oracle.Graph(G)
        A = dense_adj(g)
        z = (rng.random(g.n) < 0.5).astype(np.uint8)
        z1, k = oracle.round_drop(g, z)
        assert _indep_maximal(A, z1)[0]
        assert np.all(z1 <= z) and k == int(z.sum() - z1.sum())
        for _ in range(100):
            size0 = int(z1.sum())
            z2, k = oracle.round_complete(g, z1)
            assert _indep_maximal(A, z2)[0] and int(z2.sum()) == size0 + k
            z1 = z2
            if k == 0:
                break
        assert _indep_maximal(A, z1) == (True, True)
        for _ in range(200):
            size0 = int(z1.sum())
            z2, k = oracle.round_swap(g, z1)
            assert _indep_maximal(A, z2)[0]
            assert int(z2.sum()) == size0 + k    # each swap adds exactly one (Def. 2.3)
            z1 = z2
            while True:
                z1, kc = oracle.round_complete(g, z1)
                if kc == 0:
                    break
            if k == 0:
                break
        assert not _tight_pairs_exist(g, z1)
        assert int(z1.sum()) <= oracle.brute_mis(oracle.Graph(G.induced(g.n))) if g.n <= 26 else True


def test_flip_rounds_invariants():
    rng = np.random.default_rng(13)
    for seed in range(6):
        for signed in (False, True):
            G = mi.erdos_renyi(40, 0.15, 500 + seed)
            if signed:
                rows, cols = G.edges_directed()
                keep = rows < cols
                G = mi.from_edges(40, rows[keep], cols[keep], np.where(rng.random(int(keep.sum())) < .5, -1, 1))
            g = oracle.Graph(G)
            A = dense_adj(g)
            z = (rng.random(g.n) < 0.5).astype(np.uint8)
            last = None
            for _ in range(500):
                s = np.where(z == 1, 1.0, -1.0)
                gains = s * (A @ s)
                cut0 = oracle.eval_cut(g, z)[0]
                if np.any(gains > 0):
                    z2, k = oracle.round_flip1(g, z)
                    flipped = np.nonzero(z2 != z)[0]
                    assert len(flipped) == k > 0
                    assert not np.any(A[np.ix_(flipped, flipped)])
                    assert oracle.eval_cut(g, z2)[0] - cut0 == int(gains[flipped].sum())
                    last = 1
                else:
                    z2, k = oracle.round_flip2(g, z)
                    assert oracle.eval_cut(g, z2)[0] >= cut0 + k
                    if k == 0:
                        break
                z = z2
            s = np.where(z == 1, 1.0, -1.0)
            gains = s * (A @ s)
            assert not np.any(gains > 0)
            for u in range(g.n):
                for v in range(u + 1, g.n):
                    if A[u, v] != 0 and z[u] != z[v]:
                        assert gains[u] + gains[v] + 2 * A[u, v] <= 0


# ---------------------------------------------------------------- whole trajectory
def test_trajectory_on_n20_never_beats_brute_force():
    """mQO value <= optimum always; equal on most seeds (statistical)."""
    graphs = [mi.workload_mis_plain().induced(20)] + [mi.erdos_renyi(20, 0.3, s) for s in range(40)]
    equal = 0
    for k, G in enumerate(graphs):
        g = oracle.Graph(G)
        A = dense_adj(g)
        opt = oracle.brute_mis(g)
        p = oracle.params(t_gs=10, descent_cap=30, seed=k)
        tr = oracle.Trajectory(g, p, 0)
        tr.run(600)
        best = tr.state["best"]
        assert best <= opt
        assert best == int(tr.zbest.sum())
        assert _indep_maximal(A, tr.zbest) == (True, True)
        equal += best == opt
    assert equal >= 0.8 * len(graphs)


def test_trajectory_maxcut_never_beats_brute_force():
    equal = 0
    graphs = [mi.erdos_renyi(16, 0.35, s) for s in range(20)]
    for k, G in enumerate(graphs):
        g = oracle.Graph(G)
        opt = oracle.brute_maxcut(g)
        p = oracle.params(problem=oracle.MAXCUT, alpha=0.05, momentum=0.8, rho=0.8, t_gs=10, descent_cap=100,
                          seed=k, init_kind=1, sigma=0.2)
        tr = oracle.Trajectory(g, p, 0)
        tr.run(1500)
        best = tr.state["best"]
        assert best <= opt and best == oracle.eval_cut(g, tr.zbest)[0]
        equal += best == opt
    assert equal >= 0.7 * len(graphs)


def test_init_distributions():
    G = mi.erdos_renyi(4000, 0.002, 1)
    g = oracle.Graph(G)
    x = oracle.init_x(g, oracle.params(init_kind=0), 0)
    assert x.min() >= 0 and x.max() < 1 and abs(x.mean() - 0.5) < 0.02
    xc = oracle.init_x(g, oracle.params(problem=oracle.MAXCUT, init_kind=0), 3)
    assert xc.min() >= -1 and xc.max() < 1 and abs(xc.mean()) < 0.04
    p = oracle.params(init_kind=1, sigma=0.05)
    xd = oracle.init_x(g, p, 0)
    d = G.degrees()
    base = 1 - d / d.max()
    assert abs(float(np.mean(xd - base))) < 0.01
    assert abs(float(np.std(xd - base)) - 0.05) < 0.01


def test_oracle_struct_layouts_match_the_c_source(tmp_path):
    """The oracle binding's ctypes structures have the sizes and field offsets
    of the C structures of oracle/mqo_oracle.c."""
    import ctypes
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pairs = {"orc_params": oracle.OrcParams, "orc_state": oracle.OrcState, "orc_pool": oracle.OrcPool,
             "orc_graph": oracle.OrcGraph}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{root}/oracle/mqo_oracle.c"', "int main(void) {"]
    for st, cls in pairs.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-o", str(exe), str(src), "-lm"], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if ln:
            st, name, val = ln.split()
            got[(st, name)] = int(val)
    for st, cls in pairs.items():
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)

"""Seeded synthetic graph generators shared by the tests, the bench and smoke().

This module only builds inputs: Erdős–Rényi, random d-regular and Chung–Lu
graphs in symmetric, row-sorted CSR form (no self loops, no duplicate
edges), plus a packer that concatenates several graphs into one block
diagonal CSR.  It holds none of the optimisation method's arithmetic, so
both the CPU oracle and the CUDA library can be fed from it without sharing
any code with each other.

All generators are driven by ``numpy.random.default_rng(seed)`` (PCG64),
whose streams are identical on x86-64 and aarch64.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "Graph",
    "erdos_renyi",
    "random_regular",
    "chung_lu",
    "from_edges",
    "pack",
    "er_batch_sizes",
]


@dataclasses.dataclass
class Graph:
    """Symmetric CSR adjacency.

    ``row_ptr`` has n+1 int64 entries, ``col_idx`` nnz int32 entries sorted
    ascending inside every row, ``weights`` is None (all ones) or nnz int8
    entries in {-1,+1} with w[u,v] == w[v,u].  ``node_offsets`` (int64,
    num_graphs+1) delimits the member graphs of a packed block-diagonal
    graph; a plain graph has node_offsets == [0, n].
    """

    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    weights: np.ndarray | None = None
    node_offsets: np.ndarray | None = None

    def __post_init__(self):
        if self.node_offsets is None:
            self.node_offsets = np.array([0, self.n], dtype=np.int64)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def num_graphs(self) -> int:
        return len(self.node_offsets) - 1

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def subgraph(self, g: int) -> "Graph":
        """Member graph ``g`` of a packed graph, with local node ids."""
        lo, hi = int(self.node_offsets[g]), int(self.node_offsets[g + 1])
        a, b = int(self.row_ptr[lo]), int(self.row_ptr[hi])
        rp = (self.row_ptr[lo:hi + 1] - a).astype(np.int64)
        ci = (self.col_idx[a:b] - lo).astype(np.int32)
        w = None if self.weights is None else self.weights[a:b].copy()
        return Graph(hi - lo, rp, ci, w)

    def induced(self, k: int) -> "Graph":
        """Subgraph induced on nodes 0..k-1 (used for brute-force checks)."""
        rows, cols = self.edges_directed()
        keep = (rows < k) & (cols < k)
        w = None if self.weights is None else self.weights[keep]
        return from_edges(k, rows[keep], cols[keep], w, symmetric_input=True)

    def edges_directed(self):
        rows = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        return rows, self.col_idx.astype(np.int64)


def from_edges(n: int, u, v, w=None, symmetric_input: bool = False) -> Graph:
    """CSR from an edge list.  Self loops and duplicates are dropped.

    If ``symmetric_input`` is False the list holds each undirected edge
    once and is mirrored here.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if w is not None:
        w = np.asarray(w, dtype=np.int8)
    if not symmetric_input:
        u, v = np.concatenate([u, v]), np.concatenate([v, u])
        if w is not None:
            w = np.concatenate([w, w])
    keep = u != v
    u, v = u[keep], v[keep]
    if w is not None:
        w = w[keep]
    key = u * np.int64(n) + v
    order = np.argsort(key, kind="stable")
    key = key[order]
    first = np.ones(len(key), dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key = key[first]
    if w is not None:
        w = w[order][first]
    rows = key // n
    cols = (key % n).astype(np.int32)
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Graph(n, row_ptr, cols, w)


def _upper_pair(k: np.ndarray, n: int):
    """Map linear indices of the strict upper triangle (row major) to (i, j)."""
    kf = k.astype(np.float64)
    b = 2.0 * n - 1.0
    i = np.floor((b - np.sqrt(b * b - 8.0 * kf)) / 2.0).astype(np.int64)
    i = np.clip(i, 0, n - 2)

    def off(r):
        return r * (n - 1) - (r * (r - 1)) // 2

    # float rounding can leave i off by one in either direction
    for _ in range(3):
        lo = off(i) > k
        i = np.where(lo, i - 1, i)
        hi = off(i + 1) <= k
        i = np.where(hi, i + 1, i)
    j = k - off(i) + i + 1
    return i, j


def erdos_renyi(n: int, p: float, seed: int) -> Graph:
    """G(n, p) by geometric skipping over the n(n-1)/2 node pairs.

    Each pair is present independently with probability p; the gaps
    between present pairs are geometric (Batagelj and Brandes, 2005).
    """
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    if p <= 0.0 or total == 0:
        return from_edges(n, [], [])
    if p >= 1.0:
        ks = np.arange(total, dtype=np.int64)
    else:
        chunks = []
        pos = -1
        expect = int(total * p * 1.02) + 64
        while True:
            gaps = rng.geometric(p, size=expect).astype(np.int64)
            c = pos + np.cumsum(gaps)
            c = c[c < total]
            chunks.append(c)
            if len(c) < expect:
                break
            pos = int(c[-1])
            expect = max(64, int((total - pos) * p * 1.02) + 64)
        ks = np.concatenate(chunks)
    i, j = _upper_pair(ks, n)
    return from_edges(n, i, j)


def random_regular(n: int, d: int, seed: int, signed_weights: bool = False) -> Graph:
    """Uniform simple d-regular graph by the pairing model with restarts.

    With ``signed_weights`` each edge gets a weight drawn uniformly from
    {-1, +1} (the same weight in both directions).
    """
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    rng = np.random.default_rng(seed)
    for _ in range(1000):
        stubs = np.repeat(np.arange(n, dtype=np.int64), d)
        rng.shuffle(stubs)
        a, b = stubs[0::2], stubs[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        key = lo * n + hi
        if len(np.unique(key)) != len(key):
            continue
        w = None
        if signed_weights:
            w = np.where(rng.random(len(lo)) < 0.5, -1, 1).astype(np.int8)
        return from_edges(n, lo, hi, w)
    raise RuntimeError("pairing model did not produce a simple graph")


def chung_lu(n: int, exponent: float, mean_degree: float, seed: int) -> Graph:
    """Chung–Lu power-law graph.

    Expected degrees follow w_i ∝ (i + i0)^(-1/(exponent-1)); about
    n*mean_degree/2 endpoint pairs are drawn with probability ∝ w_u w_v,
    then self loops and duplicates are removed (so the realised mean
    degree is slightly below ``mean_degree``).
    """
    rng = np.random.default_rng(seed)
    i0 = 1.0
    w = (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (exponent - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m = int(round(n * mean_degree / 2.0 * 1.03))
    u = np.searchsorted(cdf, rng.random(m), side="right")
    v = np.searchsorted(cdf, rng.random(m), side="right")
    u = np.minimum(u, n - 1)
    v = np.minimum(v, n - 1)
    return from_edges(n, u, v)


def pack(graphs: list[Graph]) -> Graph:
    """Block-diagonal concatenation of several graphs (node ids shifted)."""
    offs = np.zeros(len(graphs) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([g.n for g in graphs])
    nnzs = np.zeros(len(graphs) + 1, dtype=np.int64)
    nnzs[1:] = np.cumsum([g.nnz for g in graphs])
    n = int(offs[-1])
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(int(nnzs[-1]), dtype=np.int32)
    weighted = any(g.weights is not None for g in graphs)
    wts = np.ones(int(nnzs[-1]), dtype=np.int8) if weighted else None
    for k, g in enumerate(graphs):
        row_ptr[offs[k]:offs[k + 1]] = g.row_ptr[:-1] + nnzs[k]
        col[nnzs[k]:nnzs[k + 1]] = g.col_idx + offs[k]
        if weighted and g.weights is not None:
            wts[nnzs[k]:nnzs[k + 1]] = g.weights
    row_ptr[n] = nnzs[-1]
    return Graph(n, row_ptr, col, wts, offs)


def er_batch_sizes(num_graphs: int, n_lo: int, n_hi: int, seed: int) -> np.ndarray:
    """Node counts n_g ~ U{n_lo..n_hi} for a batch of ER graphs."""
    rng = np.random.default_rng(seed)
    return rng.integers(n_lo, n_hi + 1, size=num_graphs)


# Named workloads (sizes and distributions of the synthetic inputs).
def workload_mis_plain():
    """One ER graph G(200, 0.05) from seed 0 (single trajectory MIS)."""
    return erdos_renyi(200, 0.05, 0)


def workload_mis_batched(num_graphs: int = 512, first_seed: int = 0):
    """ER graphs with n ~ U[700, 800], p = 0.15, seeds first_seed.., packed."""
    sizes = er_batch_sizes(num_graphs, 700, 800, 10_000 + first_seed)
    gs = [erdos_renyi(int(sizes[k]), 0.15, first_seed + k) for k in range(num_graphs)]
    return pack(gs)


def workload_er_table(n: int = 1000, d: float = 100.0, num_graphs: int = 8, first_seed: int = 0):
    """num_graphs ER graphs G(n, p = d/n) (the (n, d) parameterisation of the
    paper's ER experiments), seeds first_seed.., packed."""
    return pack([erdos_renyi(n, d / n, first_seed + k) for k in range(num_graphs)])


def workload_maxcut_regular(n: int = 100_000, signed: bool = False, seed: int = 0):
    """Random 3-regular graph (optionally with uniform ±1 edge weights)."""
    return random_regular(n, 3, seed, signed_weights=signed)


def workload_chung_lu(n: int = 1_000_000, seed: int = 0):
    """Chung–Lu power law, exponent 2.5, mean degree 8."""
    return chung_lu(n, 2.5, 8.0, seed)


def workload_mis_scale(n: int = 10_000_000, mean_degree: float = 10.0, seed: int = 0):
    """ER graph with the given mean degree (p = d/(n-1))."""
    return erdos_renyi(n, mean_degree / (n - 1), seed)

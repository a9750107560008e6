"""Row partition of one graph over several ranks, with the halo of each part.

A graph too large for one GPU is split into P contiguous ranges of rows with
about equal numbers of CSR entries.  Rank r owns rows [starts[r], starts[r+1])
and keeps their CSR rows with local column ids: its own rows first
(0 .. n_own-1, in global order), then one ghost row for every neighbour that
another rank owns (n_own .. n_own+n_halo-1, in ascending global id).  Each
row keeps its entries in the global CSR order, so a sum over a local row
adds the same values in the same order as over the global row, and the
per-row float32 sums of the step do not change with the partition.

Before every step each rank needs the current x rows of its ghosts: rank q
sends to rank r the rows of its own nodes that appear in r's halo
(``send[r]`` on q, ``recv[q]`` on r, both in ascending global id), and r
writes them to its ghost rows.  ``exchange_halo`` does that with one
all-to-all of a ``torch.distributed`` process group (NCCL between GPUs, gloo
on the CPU).

This module plans and moves data only; it holds none of the method's
arithmetic.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Part:
    """Rank `rank`'s share of the graph (see the module docstring)."""

    rank: int
    nparts: int
    row0: int                 # first owned global row
    row1: int                 # end of the owned rows
    row_ptr: np.ndarray       # n_own + 1 int64
    col_local: np.ndarray     # local column ids (own rows first, then ghosts)
    weights: np.ndarray | None
    halo: np.ndarray          # global ids of the ghost rows, ascending
    send: list[np.ndarray]    # send[q]: local ids of own rows that rank q needs
    recv: list[np.ndarray]    # recv[q]: ghost slots (0-based in the halo) filled from rank q

    @property
    def n_own(self) -> int:
        return self.row1 - self.row0

    @property
    def n_halo(self) -> int:
        return len(self.halo)


def row_ranges(row_ptr: np.ndarray, nparts: int) -> np.ndarray:
    """nparts + 1 row boundaries that cut the CSR entries into nearly equal
    parts (every part keeps at least one row when there are enough rows)."""
    n = len(row_ptr) - 1
    nnz = int(row_ptr[-1])
    starts = np.zeros(nparts + 1, dtype=np.int64)
    for r in range(1, nparts):
        starts[r] = np.searchsorted(row_ptr, nnz * r / nparts, side="left")
        starts[r] = min(max(starts[r], starts[r - 1] + (1 if n >= nparts else 0)), n)
    starts[nparts] = n
    return starts


def plan(g, nparts: int) -> list[Part]:
    """The parts of graph `g` (``n``, ``row_ptr``, ``col_idx``, ``weights``)
    for `nparts` ranks."""
    row_ptr = np.asarray(g.row_ptr, dtype=np.int64)
    col = np.asarray(g.col_idx, dtype=np.int64)
    starts = row_ranges(row_ptr, nparts)
    owner = np.searchsorted(starts, np.arange(g.n), side="right") - 1
    parts = []
    for r in range(nparts):
        r0, r1 = int(starts[r]), int(starts[r + 1])
        j0, j1 = int(row_ptr[r0]), int(row_ptr[r1])
        cg = col[j0:j1]
        ghost = (cg < r0) | (cg >= r1)
        halo = np.unique(cg[ghost])
        local = np.where(ghost, (r1 - r0) + np.searchsorted(halo, cg), cg - r0)
        w = None if g.weights is None else np.asarray(g.weights[j0:j1]).copy()
        hown = owner[halo]
        recv = [np.nonzero(hown == q)[0].astype(np.int64) for q in range(nparts)]
        parts.append(Part(r, nparts, r0, r1, (row_ptr[r0:r1 + 1] - j0).astype(np.int64), local.astype(np.int64), w,
                          halo.astype(np.int64), [np.zeros(0, np.int64)] * nparts, recv))
    # rank q sends to rank r the own rows of q that sit in r's halo, in the
    # order of r's halo (ascending global id)
    for r, pr in enumerate(parts):
        for q in range(nparts):
            need = pr.halo[pr.recv[q]]
            parts[q].send = list(parts[q].send)
            parts[q].send[r] = (need - parts[q].row0).astype(np.int64)
    return parts


def exchange_halo(x_local, part: Part, group=None):
    """Fill the ghost rows of ``x_local`` ([n_own + n_halo, B] torch tensor,
    own rows first) with the owners' current rows: one all-to-all over the
    process group.  Every rank of the group calls it with its own part."""
    import torch
    import torch.distributed as dist

    P = part.nparts
    n_own = part.n_own
    rowshape = tuple(x_local.shape[1:])
    send_idx = torch.as_tensor(np.concatenate(part.send) if P else np.zeros(0, np.int64), device=x_local.device)
    send_buf = x_local.index_select(0, send_idx).contiguous()
    recv_counts = [len(part.recv[q]) for q in range(P)]
    recv_buf = torch.empty((sum(recv_counts),) + rowshape, dtype=x_local.dtype, device=x_local.device)
    dist.all_to_all_single(recv_buf, send_buf, output_split_sizes=recv_counts,
                           input_split_sizes=[len(s) for s in part.send], group=group)
    slots = torch.as_tensor(np.concatenate(part.recv) + n_own, device=x_local.device)
    x_local.index_copy_(0, slots, recv_buf)
    return x_local

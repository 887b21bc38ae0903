"""Sharded CountGauss over torch.distributed (the distributed remark of Section 4).

Every process that shares the seed holds the same T: h, sigma and the columns of G~
are functions of (seed, global row index), G of the seed alone.  Two layouts follow:

* Row shards (features): rank p holds rows [start_p, stop_p) of X and computes
  T_p X_p with row offset start_p; T X is the sum over ranks -- one all-reduce of the
  m x d output (sum_outputs).
* Column shards (data points, as in the paper's NMF setting where each server holds
  some of the points): every rank holds all rows and some columns, computes its own
  columns of Z = T X, finds per row the max / min over its columns (with global column
  indices), and a coordinator keeps the largest / smallest, the lowest global index on
  ties (merge_anchor_records).

The helpers below are host logic (sharding, offsets, the collective, the merge);
apply_csr_row_shard and nmf_anchors_column_shard are the library calls that run each
rank's share on its GPU (cg_apply_csr, cg_nmf_anchors_csr) and combine the ranks.  The
collectives move m x d floats (row shards) or m x 4 records (column shards) through
whatever backend the process group has; CUDA results are staged through host memory, so
a gloo group serves as well as NCCL.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_range(total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous near-equal shard [start, stop) of `total` items for `rank`."""
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_csr_rows(row_ptr: np.ndarray, col_idx: np.ndarray, vals: np.ndarray, start: int, stop: int):
    """Rows [start, stop) of a CSR matrix with row_ptr rebased to 0."""
    a, b = int(row_ptr[start]), int(row_ptr[stop])
    return row_ptr[start:stop + 1] - a, col_idx[a:b], vals[a:b]


def shard_csr_cols(row_ptr: np.ndarray, col_idx: np.ndarray, vals: np.ndarray, start: int, stop: int):
    """Columns [start, stop) of a CSR matrix (all rows), column indices rebased to 0."""
    keep = (col_idx >= start) & (col_idx < stop)
    rows = np.repeat(np.arange(row_ptr.size - 1), np.diff(row_ptr))[keep]
    rp = np.zeros(row_ptr.size, row_ptr.dtype)
    np.cumsum(np.bincount(rows, minlength=row_ptr.size - 1), out=rp[1:])
    return rp, (col_idx[keep] - start).astype(col_idx.dtype), vals[keep]


def check_same_shape(t: torch.Tensor, group=None) -> None:
    """Raise ValueError on every rank of `group` unless all ranks hold a tensor of t's shape
    (at most four dimensions).  A collective over tensors of different sizes can hand some
    rank a silently wrong result (gloo: the rank with the shorter tensor), so the sharded
    calls check first, with one all-gather of four integers."""
    if t.dim() > 4:
        raise ValueError("check_same_shape: at most four dimensions")
    mine = torch.tensor(list(t.shape) + [-1] * (4 - t.dim()), dtype=torch.int64)
    shapes = [torch.empty_like(mine) for _ in range(dist.get_world_size(group))]
    dist.all_gather(shapes, mine, group=group)
    if any(not torch.equal(sh, mine) for sh in shapes):
        raise ValueError("ranks hold outputs of different shapes: " + ", ".join(
            str(tuple(int(x) for x in sh if x >= 0)) for sh in shapes))


def sum_outputs(Y: torch.Tensor, group=None, check: bool = True) -> torch.Tensor:
    """In-place sum of the per-rank m x d outputs (row shards).  With `check` the ranks
    first agree that their outputs have the same shape (check_same_shape).  A rank that
    has died or never joins makes the collective raise on the others (the connection
    closes, or the process group's timeout passes)."""
    if check:
        check_same_shape(Y, group)
    dist.all_reduce(Y, op=dist.ReduceOp.SUM, group=group)
    return Y


def local_anchor_records(Z: np.ndarray, col_start: int) -> np.ndarray:
    """Per row of a rank's columns of Z: (max value, global column of the max,
    min value, global column of the min), lowest column on ties.  Shape (m, 4), float64."""
    m, d = Z.shape
    rec = np.full((m, 4), np.nan)
    if d == 0:
        return rec
    jmax = np.argmax(Z, axis=1)
    jmin = np.argmin(Z, axis=1)
    rec[:, 0] = Z[np.arange(m), jmax]
    rec[:, 1] = jmax + col_start
    rec[:, 2] = Z[np.arange(m), jmin]
    rec[:, 3] = jmin + col_start
    return rec


def merge_anchor_records(records: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    """Coordinator merge of the ranks' records: global (imax, imin) per row."""
    m = records[0].shape[0]
    imax = np.zeros(m, np.int64)
    imin = np.zeros(m, np.int64)
    for r in range(m):
        best = None
        worst = None
        for rec in records:
            v, j, w, k = rec[r]
            if np.isnan(v):
                continue
            if best is None or v > best[0] or (v == best[0] and j < best[1]):
                best = (v, j)
            if worst is None or w < worst[0] or (w == worst[0] and k < worst[1]):
                worst = (w, k)
        imax[r] = int(best[1])
        imin[r] = int(worst[1])
    return imax, imin


def gather_anchor_records(rec: np.ndarray, group=None) -> list[np.ndarray]:
    """All ranks' records (every rank receives all, so any rank can act as coordinator).
    The ranks first agree that their record arrays have the same shape (check_same_shape)."""
    t = torch.from_numpy(np.ascontiguousarray(rec, np.float64))
    check_same_shape(t, group)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    return [o.numpy() for o in out]


def _host(t: torch.Tensor) -> torch.Tensor:
    return t.detach().to("cpu", copy=True)


def apply_csr_row_shard(row_ptr, col_idx, vals, d: int, m: int, B: int, seed: int, row_offset: int, group=None,
                        **plan_options) -> torch.Tensor:
    """T X for X sharded by rows over the ranks of `group`: this rank holds rows
    [row_offset, row_offset + n_local) of X as CSR on its GPU (row_ptr local, starting at
    0), computes T_p X_p = G (S_p X_p) with that global row offset (cg_apply_csr), and the
    m x d outputs are summed over the group.  Every rank returns the whole T X (m x d fp32,
    on the rank's device).  plan_options go to CountGauss (precision, scatter, ...)."""
    from . import countgauss
    n_local = int(row_ptr.numel()) - 1
    plan = countgauss.CountGauss(n_local, d, m, B, seed, row_offset=row_offset, **plan_options)
    Y = plan.apply_csr(row_ptr, col_idx, vals)
    plan.check()
    Yh = _host(Y)
    sum_outputs(Yh, group)
    return Yh.to(Y.device)


def nmf_anchors_column_shard(row_ptr, col_idx, vals, d_local: int, m: int, B: int, seed: int, col_offset: int,
                             group=None, **plan_options):
    """Algorithm 1 step 3 for X sharded by columns (the data points of the paper's NMF
    setting): this rank holds all n rows and columns [col_offset, col_offset + d_local) of
    X (column indices local) as CSR on its GPU.  It computes its columns of Z = T X with
    the per-row max / min (cg_nmf_anchors_csr), gathers every rank's (value, global column)
    records and merges them, lowest global column on ties.  Returns (imax, imin), int64
    numpy arrays of m global column indices, on every rank."""
    from . import countgauss
    n = int(row_ptr.numel()) - 1
    if d_local > 0:
        plan = countgauss.CountGauss(n, d_local, m, B, seed, **plan_options)
        Z, jmax, jmin = plan.nmf_anchors(row_ptr, col_idx, vals)
        plan.check()
        Zh = _host(Z).numpy().astype(np.float64)
        jmax = _host(jmax).numpy().astype(np.int64)
        jmin = _host(jmin).numpy().astype(np.int64)
        rows = np.arange(m)
        rec = np.stack([Zh[rows, jmax], jmax + col_offset, Zh[rows, jmin], jmin + col_offset], axis=1)
    else:
        rec = np.full((m, 4), np.nan)
    return merge_anchor_records(gather_anchor_records(rec, group))

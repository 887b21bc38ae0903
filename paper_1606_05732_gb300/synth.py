"""Seeded synthetic inputs shaped like the workloads of the CountGauss paper.

This module generates inputs only: it holds none of the transform's arithmetic and
imports nothing else from the package, so that the CUDA path and the FP64 oracle
can both be fed from it.  Its randomness is numpy's ``default_rng`` (PCG64), a
stream independent of the Philox stream the transform itself draws from.

The paper's datasets (TechTC-300, flow cytometry, breast-cancer expression,
climate) are not available, so these generators stand in for them with the shapes,
densities and value distributions of the benchmark configurations:

* ``csr_bernoulli``: every entry of an n x d matrix is nonzero independently with
  probability p (exact Bernoulli pattern, drawn as geometric gaps over the
  row-major flattened index), values N(0,1) or U[0,1) (nonnegative, NMF-like
  input, Section 3.1 of the paper), float32.
* ``dense_normal``: dense n x d N(0,1) float32.
* ``batch_instances``: the 96 uneven instances of the batched workload.
* ``techtc_pair``: a documents x words matrix shaped like one TechTC-300 pair of
  the SVM experiments (150-280 documents, 10,000-40,000 words); a shape stand-in,
  not the dataset.
* ``wide_csr_device``: a CSR matrix of 2^31 nonzeros or more, drawn on the GPU
  (torch's Philox-based CUDA generator, seeded), with int64 row offsets.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class CSR:
    n: int
    d: int
    row_ptr: np.ndarray  # int64, n+1
    col_idx: np.ndarray  # int32, nnz (sorted within each row)
    vals: np.ndarray     # float32, nnz

    @property
    def nnz(self) -> int:
        return int(self.col_idx.size)

    def to_dense(self) -> np.ndarray:
        X = np.zeros((self.n, self.d), np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        np.add.at(X, (rows, self.col_idx.astype(np.int64)), self.vals.astype(np.float64))
        return X


def _bernoulli_positions(total: int, p: float, rng: np.random.Generator) -> np.ndarray:
    """Sorted flat positions in [0,total) of an i.i.d. Bernoulli(p) pattern."""
    if p <= 0.0 or total == 0:
        return np.zeros(0, np.int64)
    if p >= 1.0:
        return np.arange(total, dtype=np.int64)
    out = []
    pos = -1
    chunk = max(1024, int(total * p * 1.05) + 1024)
    while True:
        gaps = rng.geometric(p, size=chunk).astype(np.int64)
        cs = np.cumsum(gaps) + pos
        keep = cs[cs < total]
        out.append(keep)
        if keep.size < cs.size:
            break
        pos = int(cs[-1])
        chunk = max(1024, chunk // 4)
    return np.concatenate(out)


def csr_bernoulli(n: int, d: int, p: float, seed: int, values: str = "normal") -> CSR:
    """n x d CSR with an i.i.d. Bernoulli(p) pattern; values 'normal' N(0,1) or
    'uniform' U[0,1), float32."""
    rng = np.random.default_rng(seed)
    pos = _bernoulli_positions(n * d, p, rng)
    rows = pos // d
    cols = (pos - rows * d).astype(np.int32)
    counts = np.bincount(rows, minlength=n) if n > 0 else np.zeros(0, np.int64)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if values == "normal":
        vals = rng.standard_normal(pos.size, dtype=np.float32)
    elif values == "uniform":
        vals = rng.random(pos.size, dtype=np.float32)
    else:
        raise ValueError(f"unknown value distribution {values!r}")
    return CSR(n, d, row_ptr, cols, vals)


def csr_from_dense(X: np.ndarray) -> CSR:
    """CSR of the nonzeros of a dense matrix (row-major order), float32 values."""
    X = np.asarray(X)
    n, d = X.shape
    rows, cols = np.nonzero(X)
    counts = np.bincount(rows, minlength=n) if n > 0 else np.zeros(0, np.int64)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, d, row_ptr, cols.astype(np.int32), X[rows, cols].astype(np.float32))


def csr_ragged(n: int, d: int, seed: int, empty_frac: float = 0.3, max_row: int | None = None) -> CSR:
    """Edge-case CSR: a fraction of empty rows, rows of every length up to d
    (including full rows), unsorted columns within rows, N(0,1) values."""
    rng = np.random.default_rng(seed)
    max_row = d if max_row is None else min(max_row, d)
    lengths = rng.integers(0, max_row + 1, size=n)
    lengths[rng.random(n) < empty_frac] = 0
    if n > 2:
        lengths[rng.integers(0, n)] = max_row  # at least one full-length row
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    cols = np.empty(int(row_ptr[-1]), np.int32)
    for i in range(n):
        L = int(lengths[i])
        if L:
            cols[row_ptr[i]:row_ptr[i + 1]] = rng.choice(d, size=L, replace=False)
    vals = rng.standard_normal(cols.size, dtype=np.float32)
    return CSR(n, d, row_ptr, cols, vals)


def techtc_pair(seed: int, docs: int | None = None, words: int | None = None, density: float = 1e-2) -> CSR:
    """Documents x words CSR (one row per document) shaped like one TechTC-300 pair of
    the SVM experiments (Section 5: 150-280 documents, 10,000-40,000 words), with the
    sizes drawn uniformly unless given.  The paper states no density; 1e-2 is taken.
    Nonnegative term weights U[0,1) on an i.i.d. Bernoulli pattern.  A shape stand-in,
    not the dataset."""
    rng = np.random.default_rng(seed)
    docs = int(rng.integers(150, 281)) if docs is None else docs
    words = int(rng.integers(10_000, 40_001)) if words is None else words
    return csr_bernoulli(docs, words, density, seed=seed + 1, values="uniform")


def dense_normal(n: int, d: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, d), dtype=np.float32)


# ------------------------------------------------------------------------------
# Named workloads (sizes of the benchmark configurations).
# ------------------------------------------------------------------------------
WORKLOADS = {
    # small case: n=65,536 x d=16, p=0.05, N(0,1); m=8, B=4096; seed 1
    "small_n65536_d16": dict(n=65536, d=16, p=0.05, values="normal", m=8, B=4096, seed=1),
    # large NMF-like case: n=2^24 x d=64, p=0.05, U[0,1); m=32, B=2^17; seed 2
    "nmf_n16M_d64": dict(n=1 << 24, d=64, p=0.05, values="uniform", m=32, B=1 << 17, seed=2),
    # half the rows of the NMF-like case (CSR 250 MB, still larger than L2), for
    # profiler captures that must stay small
    "nmf_n8M_d64": dict(n=1 << 23, d=64, p=0.05, values="uniform", m=32, B=1 << 17, seed=2),
    # a quarter of the rows of the precision-ladder case (same B and d, so the same
    # 134 MB SX), for profiler captures
    "ladder_n16M_d128": dict(n=1 << 24, d=128, p=0.01, values="normal", m=128, B=1 << 18, seed=3),
    # precision ladder: n=2^26 x d=128, p=0.01, N(0,1); m=128, B=2^18; seed 3
    "ladder_n64M_d128": dict(n=1 << 26, d=128, p=0.01, values="normal", m=128, B=1 << 18, seed=3),
    # differentiation: dense n=2^20 x d=64 (and p=0.02 sparse); m=64, B=2^16; seed 4
    "grad_n1M_d64": dict(n=1 << 20, d=64, p=0.02, values="normal", m=64, B=1 << 16, seed=4),
}


def workload_csr(name: str, scale_rows: float = 1.0) -> tuple[CSR, dict]:
    """CSR input of a named workload; the generator seed is the workload seed.
    `scale_rows` < 1 shrinks n (for sampled CPU timings)."""
    w = dict(WORKLOADS[name])
    n = max(1, int(w["n"] * scale_rows))
    X = csr_bernoulli(n, w["d"], w["p"], seed=w["seed"], values=w["values"])
    w["n"] = n
    return X, w


@dataclasses.dataclass
class BatchInstance:
    n: int
    d: int
    m: int
    B: int
    p: float
    seed: int


def _next_pow2(x: int) -> int:
    return 1 << max(0, (int(x) - 1).bit_length())


def batch_instances(count: int = 96, base_seed: int = 100) -> list[BatchInstance]:
    """Parameters of the batched workload: for instance k (transform seed
    base_seed+k) n log-uniform in [2^12, 2^22], d uniform in {8,16,32,64}, density
    log-uniform in [1e-3, 1e-1], m uniform in {8,16,32,64}, and
    B = min(next power of two >= 2 d^2 m, 2^18, floor(n/4))."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(base_seed + k)
        n = int(round(2.0 ** rng.uniform(12.0, 22.0)))
        d = int(rng.choice([8, 16, 32, 64]))
        p = float(10.0 ** rng.uniform(-3.0, -1.0))
        m = int(rng.choice([8, 16, 32, 64]))
        B = int(min(_next_pow2(2 * d * d * m), 1 << 18, n // 4))
        out.append(BatchInstance(n=n, d=d, m=m, B=max(1, B), p=p, seed=base_seed + k))
    return out


def batch_inputs(instances: list[BatchInstance]) -> list[CSR]:
    """CSR inputs of the batched workload (values N(0,1)); generator seed
    1000 + transform seed, so that inputs and transform draw independent streams."""
    return [csr_bernoulli(t.n, t.d, t.p, seed=1000 + t.seed, values="normal") for t in instances]


def sample_rows(m: int, seed: int, groups: int = 2) -> np.ndarray:
    """Output rows sampled for the plain product at full size: always the first
    and last group of four rows (so rows 0 and m-1), plus random groups, sorted."""
    rng = np.random.default_rng(seed)
    ngroups = math.ceil(m / 4)
    chosen = {0, ngroups - 1}
    while len(chosen) < min(groups, ngroups):
        chosen.add(int(rng.integers(0, ngroups)))
    rows = [r for g in sorted(chosen) for r in range(4 * g, min(4 * g + 4, m))]
    return np.asarray(rows, np.int64)


def wide_csr_device(n: int, d: int, mean_row: int, seed: int, device="cuda"):
    """(row_ptr int64[n+1], col_idx int32[nnz], vals float32[nnz]) on `device`: row
    lengths uniform in [0, 2 mean_row], columns uniform in [0, d) (a row may repeat a
    column; such entries are summed), values U[0,1).  Drawn with a seeded torch
    generator on the device, for matrices too large to build on the host."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    lengths = torch.randint(0, 2 * mean_row + 1, (n,), dtype=torch.int64, device=device, generator=g)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(lengths, 0, out=row_ptr[1:])
    del lengths
    nnz = int(row_ptr[-1].item())
    col_idx = torch.randint(0, d, (nnz,), dtype=torch.int32, device=device, generator=g)
    vals = torch.rand(nnz, dtype=torch.float32, device=device, generator=g)
    return row_ptr, col_idx, vals

"""The seeded input generators: each produces the structure and distribution its
docstring (and the input recipe of the benchmark configurations) states.  CPU only."""
import math

import numpy as np
import pytest

from paper_1606_05732_gb300 import synth


def _check_csr(X):
    rp = X.row_ptr
    assert rp.shape == (X.n + 1,) and rp[0] == 0 and rp[-1] == X.nnz
    assert (np.diff(rp) >= 0).all()
    assert X.col_idx.dtype == np.int32 and X.vals.dtype == np.float32
    assert X.col_idx.size == X.vals.size
    if X.nnz:
        assert X.col_idx.min() >= 0 and X.col_idx.max() < X.d


def test_bernoulli_pattern_density_and_values():
    n, d, p = 20_000, 64, 0.05
    X = synth.csr_bernoulli(n, d, p, seed=5)
    _check_csr(X)
    total = n * d
    sd = math.sqrt(total * p * (1 - p))
    assert abs(X.nnz - total * p) < 6 * sd
    # columns sorted and distinct within each row
    for i in range(0, n, 997):
        c = X.col_idx[X.row_ptr[i]:X.row_ptr[i + 1]]
        assert (np.diff(c) > 0).all()
    # every column about equally likely
    counts = np.bincount(X.col_idx, minlength=d)
    assert counts.min() > 0.8 * counts.mean() and counts.max() < 1.2 * counts.mean()
    assert abs(float(X.vals.mean())) < 0.02 and abs(float(X.vals.std()) - 1.0) < 0.02
    U = synth.csr_bernoulli(n, d, p, seed=5, values="uniform")
    assert U.vals.min() >= 0.0 and U.vals.max() < 1.0 and abs(float(U.vals.mean()) - 0.5) < 0.01
    with pytest.raises(ValueError):
        synth.csr_bernoulli(10, 4, 0.5, seed=1, values="cauchy")


def test_bernoulli_edge_densities_and_determinism():
    assert synth.csr_bernoulli(100, 8, 0.0, seed=1).nnz == 0
    full = synth.csr_bernoulli(50, 8, 1.0, seed=1)
    assert full.nnz == 400 and (np.diff(full.row_ptr) == 8).all()
    a, b = synth.csr_bernoulli(3000, 16, 0.1, seed=9), synth.csr_bernoulli(3000, 16, 0.1, seed=9)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    assert np.array_equal(a.vals, b.vals)
    c = synth.csr_bernoulli(3000, 16, 0.1, seed=10)
    assert not (c.nnz == a.nnz and np.array_equal(c.col_idx, a.col_idx))


def test_ragged_has_empty_and_full_rows():
    X = synth.csr_ragged(5000, 24, seed=3)
    _check_csr(X)
    lengths = np.diff(X.row_ptr)
    assert (lengths == 0).mean() > 0.25 and lengths.max() == 24
    for i in np.flatnonzero(lengths)[:200]:
        c = X.col_idx[X.row_ptr[i]:X.row_ptr[i + 1]]
        assert np.unique(c).size == c.size  # distinct, not necessarily sorted
    capped = synth.csr_ragged(5000, 24, seed=3, max_row=4)
    assert np.diff(capped.row_ptr).max() == 4


def test_dense_from_csr_roundtrip():
    X = synth.csr_bernoulli(200, 12, 0.3, seed=2)
    D = X.to_dense()
    Y = synth.csr_from_dense(D)
    assert np.array_equal(Y.row_ptr, X.row_ptr) and np.array_equal(Y.col_idx, X.col_idx)
    assert np.array_equal(Y.vals, X.vals)


def test_named_workloads_match_the_stated_recipe():
    W = synth.WORKLOADS
    assert W["small_n65536_d16"] == dict(n=65536, d=16, p=0.05, values="normal", m=8, B=4096, seed=1)
    assert W["nmf_n16M_d64"] == dict(n=1 << 24, d=64, p=0.05, values="uniform", m=32, B=1 << 17, seed=2)
    assert W["ladder_n64M_d128"] == dict(n=1 << 26, d=128, p=0.01, values="normal", m=128, B=1 << 18, seed=3)
    assert W["grad_n1M_d64"]["B"] == 1 << 16 and W["grad_n1M_d64"]["m"] == 64
    X, w = synth.workload_csr("nmf_n16M_d64", scale_rows=1 / 1024)
    _check_csr(X)
    assert X.n == w["n"] == (1 << 24) // 1024 and X.d == 64
    assert X.vals.min() >= 0.0  # nonnegative, NMF-like
    Xs, ws = synth.workload_csr("small_n65536_d16")
    assert Xs.n == 65536 and abs(Xs.nnz - 0.05 * 65536 * 16) < 6 * math.sqrt(65536 * 16 * 0.05)


def test_batch_instances_follow_the_stated_ranges():
    inst = synth.batch_instances()
    assert len(inst) == 96
    for k, t in enumerate(inst):
        assert t.seed == 100 + k
        assert (1 << 12) - 1 <= t.n <= (1 << 22) + 1
        assert t.d in (8, 16, 32, 64) and t.m in (8, 16, 32, 64)
        assert 1e-3 <= t.p <= 1e-1
        want = min(1 << max(0, (2 * t.d * t.d * t.m - 1).bit_length()), 1 << 18, t.n // 4)
        assert t.B == max(1, want)
    assert len({t.d for t in inst}) == 4 and len({t.m for t in inst}) == 4
    assert synth.batch_instances()[7] == inst[7]


def test_techtc_pair_shape_and_density():
    for seed in (1, 2, 3):
        A = synth.techtc_pair(seed)
        _check_csr(A)
        assert 150 <= A.n <= 280 and 10_000 <= A.d <= 40_000
        assert abs(A.nnz / (A.n * A.d) - 1e-2) < 1.5e-3
        assert A.vals.min() >= 0.0
    B = synth.techtc_pair(4, docs=280, words=40_000)
    assert (B.n, B.d) == (280, 40_000)


def test_sample_rows_keep_first_and_last_groups():
    rows = synth.sample_rows(32, seed=1, groups=3)
    assert rows[0] == 0 and rows[-1] == 31 and (np.diff(rows) > 0).all()
    assert synth.sample_rows(3, seed=1).tolist() == [0, 1, 2]


def test_wide_generator_structure_on_cpu():
    torch = pytest.importorskip("torch")
    rp, ci, v = synth.wide_csr_device(2000, 16, 5, seed=7, device="cpu")
    assert rp.dtype == torch.int64 and ci.dtype == torch.int32 and v.dtype == torch.float32
    assert int(rp[0]) == 0 and int(rp[-1]) == ci.numel() == v.numel()
    lengths = torch.diff(rp)
    assert int(lengths.min()) >= 0 and int(lengths.max()) <= 10
    assert abs(float(lengths.double().mean()) - 5.0) < 0.3
    assert int(ci.min()) >= 0 and int(ci.max()) < 16
    assert float(v.min()) >= 0.0 and float(v.max()) < 1.0
    rp2, ci2, v2 = synth.wide_csr_device(2000, 16, 5, seed=7, device="cpu")
    assert torch.equal(rp, rp2) and torch.equal(ci, ci2) and torch.equal(v, v2)

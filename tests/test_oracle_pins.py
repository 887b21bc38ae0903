"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks the oracle against something the paper or mathematics fixes:
an independent library implementation of Philox4x32-10, closed forms, invariants,
brute-force materialisation of S, G and T on tiny inputs, exact moment identities
and distribution tests.  A plausible slip anywhere in the oracle (a dropped term,
a wrong sign or index, a transposed operand, a wrong constant) fails one of them.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1606_05732_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# -----------------------------------------------------------------------------
# Generator: Philox4x32-10 against Triton's implementation (library, not ours).
# -----------------------------------------------------------------------------
def _triton_words(reqs):
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, os.path.join(HERE, "_philox_triton_ref.py")],
                         input=json.dumps(reqs), capture_output=True, text=True, env=env,
                         timeout=600)
    if out.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + out.stderr[-300:])
    return np.asarray(json.loads(out.stdout), dtype=np.uint64)


@pytest.fixture(scope="module")
def triton_cases():
    rng = np.random.default_rng(7)
    seeds = [0, 1, 2, 3, 4, 100, 2**32 - 1, 2**32, 2**63 + 12345, 2**64 - 1]
    reqs = []
    for s in seeds:
        for tag in (0, 1, 2):
            for idx in [0, 1, 2**31 - 1, 2**32 - 1, 2**32, int(rng.integers(0, 2**40))]:
                reqs.append([s, idx & 0xFFFFFFFF, idx >> 32, tag, 0])
    # a few arbitrary counters in all four words
    for _ in range(16):
        reqs.append([int(rng.integers(0, 2**63))] + [int(x) for x in rng.integers(0, 2**32, 4)])
    return reqs, _triton_words(reqs)


def test_philox_matches_library_implementation(triton_cases):
    reqs, ref = triton_cases
    for (s, c0, c1, c2, c3), want in zip(reqs, ref):
        got = oracle.philox4x32_10([c0, c1, c2, c3], [s & 0xFFFFFFFF, s >> 32])
        assert got.tolist() == want.tolist(), (s, c0, c1, c2, c3)


def test_stream_layout_words(triton_cases):
    """philox_words(seed, tag, idx) is Philox at counter (lo(idx), hi(idx), tag, 0)
    under key (lo(seed), hi(seed))."""
    reqs, ref = triton_cases
    for (s, c0, c1, c2, c3), want in zip(reqs, ref):
        if c3 != 0 or c2 > 2:
            continue
        idx = c0 | (c1 << 32)
        got = oracle.philox_words(s, c2, idx, 1)[0]
        assert got.tolist() == want.tolist()


# -----------------------------------------------------------------------------
# Hash h and sign sigma (Section 1.1; Section 7).
# -----------------------------------------------------------------------------
@pytest.mark.parametrize("row0", [10**9, 10**9 + 3])
@pytest.mark.parametrize("B", [1, 2, 3, 4096, 100003, 1 << 17, 1 << 18, (1 << 31) - 1, 1 << 32])
def test_hash_is_multiply_high_of_the_rows_word(B, row0):
    """Row i reads word i mod 4 of the tag-0 call at floor(i/4): h = floor(w B / 2^32),
    sigma from the word's lowest bit (rows from an offset that is not a multiple of 4
    start inside a call)."""
    seed, n = 99, 2000
    h, s = oracle.hash_sign(seed, B, row0, n)
    g0 = row0 // 4
    w = oracle.philox_words(seed, 0, g0, (row0 + n - 1) // 4 - g0 + 1).astype(object)
    for t in range(n):
        i = row0 + t
        x = int(w[i // 4 - g0, i % 4])
        # floor(x * B / 2^32): h * 2^32 <= x * B < (h + 1) * 2^32
        assert int(h[t]) * 2**32 <= x * B < (int(h[t]) + 1) * 2**32
        assert s[t] == (-1 if x & 1 else 1)
    assert h.min() >= 0 and h.max() < B


def test_hash_uniform_and_signs_balanced():
    B, n = 256, 1 << 18
    h, s = oracle.hash_sign(5, B, 0, n)
    counts = np.bincount(h, minlength=B)
    chi2 = float(((counts - n / B) ** 2 / (n / B)).sum())
    assert stats.chi2.sf(chi2, B - 1) > 1e-4
    # sign: fair coin, independent of the bucket
    assert abs(s.mean()) < 5 / math.sqrt(n)
    pos = np.bincount(h[s > 0], minlength=B)
    table = np.stack([pos, counts - pos])
    assert stats.chi2_contingency(table)[1] > 1e-4
    # pair-collision rate of distinct rows is 1/B
    hh, _ = oracle.hash_sign(6, B, 0, 20000)
    coll = (hh[:-1] == hh[1:]).mean()
    assert abs(coll - 1 / B) < 5 * math.sqrt((1 / B) / 20000)


def test_countsketch_structure():
    """Every column of S has exactly one nonzero, equal to +1 or -1 (Section 1.1)."""
    n, B = 300, 17
    S = dense_S(11, n, B)
    nz = (S != 0).sum(axis=0)
    assert (nz == 1).all()
    assert set(np.unique(S[S != 0]).tolist()) <= {-1.0, 1.0}


# -----------------------------------------------------------------------------
# Uniforms and Box-Muller normals (unit-variance Gaussians of Theorem 1).
# -----------------------------------------------------------------------------
def test_uniform24_grid_and_symmetry():
    rng = np.random.default_rng(3)
    ws = [0, 1, 511, 512, 2**31, 2**32 - 1] + [int(x) for x in rng.integers(0, 2**32, 2000)]
    for w in ws:
        u = oracle.uniform24(w)
        assert 0.0 < u < 1.0
        k = u * 2**24
        assert k == int(k) and int(k) % 2 == 1  # odd multiple of 2^-24
        # the low 9 bits are not used; complementing the word reflects u about 1/2
        assert oracle.uniform24(w ^ 0x1FF) == u
        assert oracle.uniform24(w) + oracle.uniform24(w ^ 0xFFFFFFFF) == 1.0
    assert oracle.uniform24(0) == 2.0**-24
    assert oracle.uniform24(2**32 - 1) == 1.0 - 2.0**-24
    # monotone in the word
    us = [oracle.uniform24(w) for w in sorted(ws)]
    assert all(a <= b for a, b in zip(us, us[1:]))


def test_box_muller_polar_invariants():
    """Each pair (z0, z1) has squared radius -2 ln u0 and angle 2 pi u1 (mod 2 pi);
    likewise (z2, z3) with u2, u3."""
    w = oracle.philox_words(8, 1, 0, 5000)
    z = oracle.box_muller_words(w)
    for t in range(w.shape[0]):
        u = [oracle.uniform24(int(x)) for x in w[t]]
        for a, b, ur, ua in ((0, 1, u[0], u[1]), (2, 3, u[2], u[3])):
            r2 = z[t, a] ** 2 + z[t, b] ** 2
            assert r2 == pytest.approx(-2.0 * math.log(ur), rel=1e-12, abs=1e-15)
            ang = math.atan2(z[t, b], z[t, a]) % (2 * math.pi)
            want = (2 * math.pi * ua) % (2 * math.pi)
            dang = min(abs(ang - want), 2 * math.pi - abs(ang - want))
            assert dang < 1e-9


def test_box_muller_is_standard_normal():
    z = oracle.box_muller_words(oracle.philox_words(9, 1, 0, 1 << 18))
    for lane in range(4):
        assert stats.kstest(z[:, lane], "norm").pvalue > 1e-4
    flat = z.ravel()
    n = flat.size
    assert abs(flat.mean()) < 5 / math.sqrt(n)
    assert abs(flat.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(flat)) < 5 * math.sqrt(24.0 / n)
    # lanes uncorrelated (in particular the cos/sin pair of one radius)
    C = np.corrcoef(z.T)
    off = C[~np.eye(4, dtype=bool)]
    assert np.abs(off).max() < 5 / math.sqrt(z.shape[0])


def test_gaussian_layout_against_library_words(triton_cases):
    """Entry (r, c) of an R x C Gaussian with tag t is lane r mod 4 of the Box-Muller
    normals of Philox at idx = c * ceil(R/4) + floor(r/4), tag t; words from Triton."""
    R, C, seed = 10, 6, 2**63 + 12345
    groups = math.ceil(R / 4)
    reqs = []
    for c in range(C):
        for g in range(groups):
            idx = c * groups + g
            for tag in (1, 2):
                reqs.append([seed, idx & 0xFFFFFFFF, idx >> 32, tag, 0])
    ref = _triton_words(reqs)
    z = oracle.box_muller_words(ref.astype(np.uint32))
    lut = {tuple(q[1:4]): z[k] for k, q in enumerate(reqs)}
    for tag in (1, 2):
        blk = oracle.gaussian_block(seed, tag, R, 0, R, 0, C)
        for r in range(R):
            for c in range(C):
                idx = c * groups + r // 4
                assert blk[r, c] == lut[(idx & 0xFFFFFFFF, idx >> 32, tag)][r % 4]


def test_gaussian_block_slicing_consistent():
    full = oracle.gaussian_block(4, 1, 13, 0, 13, 0, 40)
    part = oracle.gaussian_block(4, 1, 13, 3, 11, 7, 29)
    np.testing.assert_array_equal(part, full[3:11, 7:29])
    # G and G~ are different streams
    assert not np.array_equal(oracle.gaussian_block(4, 2, 13, 0, 13, 0, 40), full)


# -----------------------------------------------------------------------------
# Brute force: dense S, G, T materialised from the generator (tiny inputs).
# -----------------------------------------------------------------------------
def dense_S(seed, n, B, row_offset=0):
    h, s = oracle.hash_sign(seed, B, row_offset, n)
    S = np.zeros((B, n))
    S[h, np.arange(n)] = s
    return S


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n,d,m,B,seed", [(64, 5, 4, 32, 1), (50, 3, 7, 9, 2), (40, 1, 1, 1, 3),
                                          (33, 8, 13, 64, 2**40 + 3), (1, 1, 1, 1, 0)])
def test_brute_force_dense_T(n, d, m, B, seed):
    X = synth.csr_ragged(n, d, seed=seed)
    Xd = X.to_dense()
    S = dense_S(seed, n, B)
    G = oracle.gaussian_G(seed, m, B)
    T = G @ S
    Y, SX = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, return_sx=True)
    np.testing.assert_allclose(SX, S @ Xd, rtol=0, atol=1e-12)
    assert rel(Y, T @ Xd) < 1e-13
    Yd = oracle.apply_dense(seed, m, B, Xd)
    assert rel(Yd, T @ Xd) < 1e-13


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_contract_range_and_parallel_apply_against_materialised_T(threads):
    """The contraction restricted to columns [b0, b1) of G is G[:, b0:b1] SX[b0:b1] with G
    materialised; the host-parallel apply (row shards with global offsets, column ranges
    of G, shards summed) equals T.X with S and G materialised, with and without a row
    offset, and a range of G's columns gives that part of G.SX."""
    n, d, m, B, seed = 203, 6, 9, 37, 7
    X = synth.csr_ragged(n, d, seed=11)
    Xd = X.to_dense()
    G = oracle.gaussian_G(seed, m, B)
    SX = oracle.sketch_csr(seed, n, d, B, X.row_ptr, X.col_idx, X.vals)
    for b0, b1 in [(0, B), (0, 1), (5, 20), (36, 37), (10, 10)]:
        want = G[:, b0:b1] @ SX[b0:b1]
        got = oracle.contract_range(seed, m, SX, b0, b1)
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
    for off in (0, 1000):
        T = G @ dense_S(seed, n + off, B)[:, off:]
        got = oracle.apply_csr_parallel(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, threads, row_offset=off)
        assert rel(got, T @ Xd) < 1e-13
    part = oracle.apply_csr_parallel(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, threads, b_range=(4, 30))
    assert rel(part, G[:, 4:30] @ SX[4:30]) < 1e-13


def test_brute_force_plain():
    n, d, m, seed = 70, 6, 9, 5
    X = synth.csr_ragged(n, d, seed=4)
    Xd = X.to_dense()
    Gt = oracle.gaussian_block(seed, 2, m, 0, m, 0, n)
    want = Gt @ Xd
    assert rel(oracle.plain_dense(seed, m, Xd), want) < 1e-13
    assert rel(oracle.plain_csr(seed, n, d, m, X.row_ptr, X.col_idx, X.vals), want) < 1e-13
    rows = np.array([0, 3, 4, 8])
    got = oracle.plain_csr(seed, n, d, m, X.row_ptr, X.col_idx, X.vals, rows=rows)
    assert rel(got, want[rows]) < 1e-13


@pytest.mark.parametrize("n,d,m,B,seed", [(64, 5, 4, 32, 1), (50, 3, 7, 9, 2), (40, 1, 1, 1, 3),
                                          (33, 8, 13, 64, 2**40 + 3)])
def test_brute_force_right_projection(n, d, m, B, seed):
    """Section 9's projection X.R with R = T^T: for a d x n matrix A (one row per
    sample), Z = A.(G.S)^T with S and G materialised densely."""
    A = synth.csr_ragged(d, n, seed=seed)
    Ad = A.to_dense()
    T = oracle.gaussian_G(seed, m, B) @ dense_S(seed, n, B)
    Z = oracle.apply_right_csr(seed, n, d, m, B, A.row_ptr, A.col_idx, A.vals)
    assert Z.shape == (d, m)
    assert rel(Z, Ad @ T.T) < 1e-13


def test_right_projection_is_transposed_left():
    """A.T^T = (T.A^T)^T: the right form on A (T's columns added per nonzero) equals
    the scatter-then-contract path on A^T, also with a global column offset."""
    d, n, m, B, seed = 37, 300, 9, 45, 6
    A = synth.csr_bernoulli(d, n, 0.05, seed=3)
    At = synth.csr_from_dense(A.to_dense().T)
    for off in (0, 1000):
        Z = oracle.apply_right_csr(seed, n, d, m, B, A.row_ptr, A.col_idx, A.vals, col_offset=off)
        Y = oracle.apply_csr(seed, n, d, m, B, At.row_ptr, At.col_idx, At.vals, row_offset=off)
        assert rel(Z, Y.T) < 1e-13
    Z0 = oracle.apply_right_csr(seed, n, d, m, B, A.row_ptr, A.col_idx, A.vals)
    assert rel(Z, Z0) > 0.1  # the offset changes which columns of T are drawn


def test_right_unit_matrix_reads_one_column_of_G():
    """A = e_r e_c^T: row r of Z is sigma(c) G[:, h(c)] and every other row is 0."""
    d, n, m, B, seed = 6, 40, 10, 17, 5
    h, s = oracle.hash_sign(seed, B, 0, n)
    G = oracle.gaussian_G(seed, m, B)
    for r, c in [(0, 0), (3, 39), (5, 12)]:
        rp = np.zeros(d + 1, np.int64)
        rp[r + 1:] = 1
        Z = oracle.apply_right_csr(seed, n, d, m, B, rp, np.array([c]), np.array([1.0]))
        np.testing.assert_array_equal(Z[r], s[c] * G[:, h[c]])
        assert not np.delete(Z, r, axis=0).any()


def test_row_offset_is_global_index():
    """A shard with global row offset o uses h, sigma and G~ columns of rows o.. ;
    shard results sum to the unsharded one (distributed remark, Section 4)."""
    n, d, m, B, seed = 90, 4, 5, 16, 12
    X = synth.csr_ragged(n, d, seed=8)
    Y = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals)
    P = oracle.plain_csr(seed, n, d, m, X.row_ptr, X.col_idx, X.vals)
    cuts = [0, 17, 18, 60, 90]
    Ys, Ps = np.zeros_like(Y), np.zeros_like(P)
    for a, b in zip(cuts, cuts[1:]):
        rp = X.row_ptr[a:b + 1] - X.row_ptr[a]
        ci = X.col_idx[X.row_ptr[a]:X.row_ptr[b]]
        v = X.vals[X.row_ptr[a]:X.row_ptr[b]]
        Ys += oracle.apply_csr(seed, b - a, d, m, B, rp, ci, v, row_offset=a)
        Ps += oracle.plain_csr(seed, b - a, d, m, rp, ci, v, row_offset=a)
    assert rel(Ys, Y) < 1e-13 and rel(Ps, P) < 1e-13


# -----------------------------------------------------------------------------
# Special cases with closed forms.
# -----------------------------------------------------------------------------
def test_single_bucket_is_rank_one():
    """B = 1: S X = sigma^T X is one row, so Y = G[:,0] (sigma^T X)."""
    n, d, m, seed = 40, 5, 6, 3
    X = synth.dense_normal(n, d, seed=1).astype(np.float64)
    _, s = oracle.hash_sign(seed, 1, 0, n)
    g = oracle.gaussian_G(seed, m, 1)[:, 0]
    want = np.outer(g, s @ X)
    assert rel(oracle.apply_dense(seed, m, 1, X), want) < 1e-13
    assert np.linalg.matrix_rank(oracle.apply_dense(seed, m, 1, X)) == 1


def test_unit_matrix_reads_one_column_of_G():
    """X = e_i e_j^T: Y[:, j] = sigma(i) G[:, h(i)] and every other column is 0."""
    n, d, m, B, seed = 30, 4, 11, 23, 9
    h, s = oracle.hash_sign(seed, B, 0, n)
    G = oracle.gaussian_G(seed, m, B)
    for i, j in [(0, 0), (7, 3), (29, 1)]:
        X = np.zeros((n, d))
        X[i, j] = 1.0
        Y = oracle.apply_dense(seed, m, B, X)
        np.testing.assert_array_equal(Y[:, j], s[i] * G[:, h[i]])
        assert not np.delete(Y, j, axis=1).any()


def test_scalar_case():
    X = np.array([[2.5]])
    h, s = oracle.hash_sign(1, 3, 0, 1)
    g = oracle.gaussian_G(1, 1, 3)
    assert oracle.apply_dense(1, 1, 3, X)[0, 0] == pytest.approx(g[0, h[0]] * s[0] * 2.5, rel=1e-15)


def test_empty_input():
    X = synth.csr_bernoulli(50, 7, 0.0, seed=1)
    assert X.nnz == 0
    assert not oracle.apply_csr(1, 50, 7, 3, 8, X.row_ptr, X.col_idx, X.vals).any()
    assert not oracle.plain_csr(1, 50, 7, 3, X.row_ptr, X.col_idx, X.vals).any()


def test_duplicate_entries_are_summed():
    rp = np.array([0, 3, 3, 4])
    ci = np.array([1, 1, 0, 2])
    v = np.array([1.0, 2.0, -4.0, 0.5])
    Xd = np.zeros((3, 3))
    for r in range(3):
        for k in range(rp[r], rp[r + 1]):
            Xd[r, ci[k]] += v[k]
    np.testing.assert_allclose(oracle.apply_csr(2, 3, 3, 5, 4, rp, ci, v), oracle.apply_dense(2, 5, 4, Xd),
                               rtol=1e-14, atol=1e-14)


# -----------------------------------------------------------------------------
# Linearity and adjoint: <T X, dY> = <X, T^T dY>; gradcheck on an autograd wrapper.
# -----------------------------------------------------------------------------
def test_adjoint_dot_product_identity():
    n, d, m, B, seed = 120, 6, 5, 32, 4
    rng = np.random.default_rng(0)
    X = rng.standard_normal((n, d))
    dY = rng.standard_normal((m, d))
    lhs = float((oracle.apply_dense(seed, m, B, X) * dY).sum())
    rhs = float((X * oracle.adjoint_dense(seed, n, m, B, dY)).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # W = G^T dY against the materialised G
    G = oracle.gaussian_G(seed, m, B)
    np.testing.assert_allclose(oracle.adjoint_w(seed, m, B, dY), G.T @ dY, rtol=1e-13, atol=1e-13)
    # sparse form: the dense gradient read at the nonzeros
    Xs = synth.csr_ragged(n, d, seed=3)
    dXv = oracle.adjoint_csr(seed, n, m, B, Xs.row_ptr, Xs.col_idx, dY)
    dX = oracle.adjoint_dense(seed, n, m, B, dY)
    rows = np.repeat(np.arange(n), np.diff(Xs.row_ptr))
    np.testing.assert_array_equal(dXv, dX[rows, Xs.col_idx])


def test_linearity_and_finite_differences():
    n, d, m, B, seed = 80, 3, 4, 16, 6
    rng = np.random.default_rng(1)
    X1, X2, E = (rng.standard_normal((n, d)) for _ in range(3))
    T = lambda X: oracle.apply_dense(seed, m, B, X)  # noqa: E731
    assert rel(T(X1 + 2.0 * X2), T(X1) + 2.0 * T(X2)) < 1e-13
    eps = 1e-3
    assert rel((T(X1 + eps * E) - T(X1)) / eps, T(E)) < 1e-9


def test_gradcheck_fp64():
    """Gradcheck of the oracle's forward/adjoint pair at n=256, d=4, m=4, B=64, seed 4."""
    torch = pytest.importorskip("torch")

    class OracleT(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X):
            ctx.n = X.shape[0]
            return torch.from_numpy(oracle.apply_dense(4, 4, 64, X.detach().numpy()))

        @staticmethod
        def backward(ctx, dY):
            return torch.from_numpy(oracle.adjoint_dense(4, ctx.n, 4, 64, dY.detach().numpy()))

    X = torch.randn(256, 4, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(OracleT.apply, (X,), eps=1e-6, atol=1e-7)


# -----------------------------------------------------------------------------
# Moment identities (Section 2 intuition; Section 7, Lemma 4 and its closed form).
# -----------------------------------------------------------------------------
def _cov_within(rows, Sigma, k=5.0):
    """Sample second-moment matrix of zero-mean Gaussian rows against Sigma, entry by
    entry, within k standard errors: Var(C_ab) = (S_aa S_bb + S_ab^2) / N."""
    N = rows.shape[0]
    C = rows.T @ rows / N
    dg = np.diag(Sigma)
    se = np.sqrt((np.outer(dg, dg) + Sigma ** 2) / N)
    assert (np.abs(C - Sigma) < k * se).all(), (C, Sigma, se)


def _mean_within(samples, want, k=5.0):
    samples = np.asarray(samples, np.float64)
    se = samples.std(ddof=1) / math.sqrt(samples.size)
    assert abs(samples.mean() - want) < k * se + 1e-12 * abs(want), (samples.mean(), want, se)


def test_sketch_preserves_squared_norm_in_expectation():
    """E_S ||S X||_F^2 = ||X||_F^2."""
    n, d, B = 60, 4, 8
    X = synth.dense_normal(n, d, seed=2).astype(np.float64)
    vals = [np.sum(oracle.sketch_dense(s, B, X) ** 2) for s in range(3000)]
    _mean_within(vals, np.sum(X ** 2))


def test_conditional_second_moment():
    """Given S, E_G ||G S X||_F^2 = m ||S X||_F^2 (rows of G S X are N(0, X^T S^T S X))."""
    n, d, m, B = 60, 4, 6, 8
    X = synth.dense_normal(n, d, seed=3).astype(np.float64)
    SX = oracle.sketch_dense(77, B, X)
    vals = [np.sum(oracle.contract(s, m, SX) ** 2) for s in range(1000, 4000)]
    _mean_within(vals, m * np.sum(SX ** 2))


def test_unconditional_second_moment():
    """E ||T X||_F^2 = m ||X||_F^2 (no 1/sqrt(m) scaling, unit-variance G)."""
    n, d, m, B = 50, 3, 5, 8
    X = synth.dense_normal(n, d, seed=4).astype(np.float64)
    vals = [np.sum(oracle.apply_dense(s, m, B, X) ** 2) for s in range(4000)]
    _mean_within(vals, m * np.sum(X ** 2))


def test_lemma4_closed_form():
    """E ||X^T S^T S X - X^T X||_F^2 = (||X||_F^4 + ||X^T X||_F^2 - 2 sum_k ||x_k||^4) / B,
    the exact value behind Lemma 4's O(d^2/B) bound; for orthonormal U this is
    (d^2 + d - 2 sum_k ||u_k||^4) / B."""
    n, d, B = 40, 3, 16
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((n, d)))
    want = (d * d + d - 2.0 * np.sum(np.sum(U ** 2, axis=1) ** 2)) / B
    vals = []
    for s in range(4000):
        SU = oracle.sketch_dense(s, B, U)
        vals.append(np.sum((SU.T @ SU - np.eye(d)) ** 2))
    _mean_within(vals, want)
    # general X
    X = rng.standard_normal((n, d))
    rn = np.sum(X ** 2, axis=1)
    want = (np.sum(X ** 2) ** 2 + np.sum((X.T @ X) ** 2) - 2.0 * np.sum(rn ** 2)) / B
    vals = []
    for s in range(4000):
        SX = oracle.sketch_dense(s + 10**6, B, X)
        vals.append(np.sum((SX.T @ SX - X.T @ X) ** 2))
    _mean_within(vals, want)


# -----------------------------------------------------------------------------
# Distributions (Section 7: rows of G S U given S are N(0, U^T S^T S U); Theorem 1).
# -----------------------------------------------------------------------------
def test_plain_rows_are_gaussian_with_covariance_XtX():
    n, d, m = 30, 3, 8
    X = synth.dense_normal(n, d, seed=6).astype(np.float64)
    a = np.array([0.3, -1.0, 0.5])
    rows = np.concatenate([oracle.plain_dense(s, m, X) for s in range(1500)])
    z = rows @ a / math.sqrt(a @ X.T @ X @ a)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    _cov_within(rows, X.T @ X)


def test_conditional_rows_are_gaussian():
    """Given S, rows of G S X are exactly N(0, X^T S^T S X)."""
    n, d, m, B = 40, 3, 8, 6
    X = synth.dense_normal(n, d, seed=7).astype(np.float64)
    SX = oracle.sketch_dense(3, B, X)
    M = SX.T @ SX
    a = np.array([1.0, 0.2, -0.7])
    rows = np.concatenate([oracle.contract(s, m, SX) for s in range(5000, 6500)])
    z = rows @ a / math.sqrt(a @ M @ a)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    _cov_within(rows, M)


def test_unconditional_rows_match_plain_when_B_large():
    """Theorem 1 regime (B >> d^2 m): rows of T X are close to N(0, X^T X)."""
    n, d, m, B = 200, 2, 2, 4096
    rng = np.random.default_rng(8)
    U, _ = np.linalg.qr(rng.standard_normal((n, d)))
    rows = np.concatenate([oracle.apply_dense(s, m, B, U) for s in range(4000)])
    for a in (np.array([1.0, 0.0]), np.array([0.6, 0.8])):
        assert stats.kstest(rows @ a, "norm").pvalue > 1e-4
    _cov_within(rows, np.eye(d))


def _lemma5_statistic(Y, m):
    """max over column pairs i < j of | ||Y (e_i + e_j)||^2 / m - 2 |."""
    d = Y.shape[1]
    best = 0.0
    for i in range(d):
        for j in range(i + 1, d):
            best = max(best, abs(np.sum((Y[:, i] + Y[:, j]) ** 2) / m - 2.0))
    return best


def _lemma5_block_U(d, B):
    L = math.ceil(math.sqrt(B) / d)
    U = np.zeros((L * d, d))
    for i in range(d):
        U[L * i:L * (i + 1), i] = 1.0 / math.sqrt(L)
    return U


def test_lemma5_block_matrix_is_detectably_non_gaussian():
    """Negative control (Lemma 5).  With the block matrix U (column i holds
    L = ceil(sqrt(B)/d) entries 1/sqrt(L) in its own block of rows), a collision
    h(a) = h(b) between two blocks moves ||T U (e_i + e_j)||^2 / m from 2 by 2/L.
    At small B (L = 1, a collision among the d(d-1)/2 block pairs in about a third of
    the draws) the distinguisher max_{i<j} | ||T U (e_i+e_j)||^2/m - 2 | separates
    CountGauss from the plain product; at B >> d^2 m the effect 2/L is buried in the
    chi-square noise and the two are indistinguishable."""
    d, m, seeds = 4, 32, 300
    U = _lemma5_block_U(d, 16)
    plain = [_lemma5_statistic(oracle.plain_dense(s, m, U), m) for s in range(seeds)]
    small = [_lemma5_statistic(oracle.apply_dense(s, m, 16, U), m) for s in range(seeds)]
    assert stats.ks_2samp(small, plain).pvalue < 1e-6
    B = 1 << 13
    U = _lemma5_block_U(d, B)
    plain = [_lemma5_statistic(oracle.plain_dense(s, m, U), m) for s in range(seeds)]
    large = [_lemma5_statistic(oracle.apply_dense(s, m, B, U), m) for s in range(seeds)]
    assert stats.ks_2samp(large, plain).pvalue > 1e-4


# -----------------------------------------------------------------------------
# Algorithm 1 step 3: row argmax / argmin (lowest index on ties) vs numpy.
# -----------------------------------------------------------------------------
def test_row_argmax_argmin():
    rng = np.random.default_rng(9)
    Z = rng.integers(-3, 4, size=(50, 17)).astype(np.float64)
    imax, imin = oracle.row_argmax_argmin(Z)
    np.testing.assert_array_equal(imax, np.argmax(Z, axis=1))
    np.testing.assert_array_equal(imin, np.argmin(Z, axis=1))

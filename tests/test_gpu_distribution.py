"""Distribution checks on the CUDA path itself (the FP64 oracle has its own in
test_oracle_pins.py): samples of rows drawn by the library's kernels, reduced in FP64
on the device (cg_moments_f64), against the distributions the paper states.

 * Rows of the plain G~.X are exactly N(0, X^T X) (G~ has i.i.d. unit-variance entries).
 * Given S, rows of G.(S.X) are exactly N(0, X^T S^T S X) (Section 7).
 * With B >> d^2 m, rows of T.X are close to N(0, X^T X) (Theorem 1).
 * E ||T X||_F^2 = m ||X||_F^2.
Each covariance entry is held to 5 standard errors of a Wishart sample,
Var(C_ab) = (S_aa S_bb + S_ab^2) / N; the projections are KS-tested against N(0, 1).
Also: NMF anchors (Algorithm 1 step 3) against the oracle / numpy.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1606_05732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cg():
    from paper_1606_05732_gb300 import countgauss
    return countgauss


def check_cov(gram, N, Sigma, k=5.0):
    C = gram / N
    dg = np.diag(Sigma)
    se = np.sqrt((np.outer(dg, dg) + Sigma ** 2) / N)
    assert (np.abs(C - Sigma) < k * se).all(), np.abs(C - Sigma).max()


def test_gram_reduction_matches_numpy():
    Y = torch.randn(10007, 37, device="cuda")
    gram, sumsq = cg().moments_f64(Y)
    Yn = Y.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(gram.cpu().numpy(), Yn.T @ Yn, rtol=1e-12, atol=1e-9)
    assert float(sumsq.item()) == pytest.approx(float((Yn ** 2).sum()), rel=1e-12)


def test_plain_rows_are_gaussian_on_device():
    n, d, m, seeds = 4000, 4, 64, 400
    Xn = synth.dense_normal(n, d, seed=11)
    X = synth.csr_from_dense(Xn)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(X.col_idx).cuda()
    v = torch.from_numpy(X.vals).cuda()
    gram = torch.zeros(d, d, dtype=torch.float64, device="cuda")
    rows = []
    for s in range(seeds):
        Y = cg().CountGauss(n, d, m, 64, 1000 + s).plain_csr(rp, ci, v)
        cg().moments_f64(Y, gram)
        rows.append(Y.cpu().numpy())
    XtX = Xn.astype(np.float64).T @ Xn.astype(np.float64)
    check_cov(gram.cpu().numpy(), seeds * m, XtX)
    a = np.array([1.0, -0.5, 0.25, 2.0])
    z = np.concatenate(rows) @ a / math.sqrt(a @ XtX @ a)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_conditional_rows_are_gaussian_on_device():
    """Fixed S (seed 5's sketch), G drawn from other seeds: rows ~ N(0, (SX)^T SX)."""
    n, d, m, B, seeds = 3000, 3, 64, 8, 400
    Xn = synth.dense_normal(n, d, seed=12)
    X = torch.from_numpy(Xn).cuda()
    SX = cg().CountGauss(n, d, m, B, 5).sketch_dense(X)
    M = SX.cpu().numpy().astype(np.float64)
    M = M.T @ M
    gram = torch.zeros(d, d, dtype=torch.float64, device="cuda")
    rows = []
    for s in range(seeds):
        Y = cg().CountGauss(n, d, m, B, 2000 + s).contract(SX)
        cg().moments_f64(Y, gram)
        rows.append(Y.cpu().numpy())
    check_cov(gram.cpu().numpy(), seeds * m, M)
    a = np.array([0.3, 1.0, -0.8])
    z = np.concatenate(rows) @ a / math.sqrt(a @ M @ a)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_theorem1_regime_on_device():
    """B >> d^2 m: rows of T U close to N(0, I) for orthonormal U; E||TU||^2 = m d."""
    n, d, m, B, seeds = 5000, 2, 16, 1 << 14, 600
    rng = np.random.default_rng(13)
    U, _ = np.linalg.qr(rng.standard_normal((n, d)))
    Ut = torch.from_numpy(U.astype(np.float32)).cuda()
    gram = torch.zeros(d, d, dtype=torch.float64, device="cuda")
    sumsq = torch.zeros(1, dtype=torch.float64, device="cuda")
    norms = []
    rows = []
    for s in range(seeds):
        Y = cg().CountGauss(n, d, m, B, 3000 + s).apply_dense(Ut)
        before = float(sumsq.item())
        cg().moments_f64(Y, gram, sumsq)
        norms.append(float(sumsq.item()) - before)
        rows.append(Y.cpu().numpy())
    check_cov(gram.cpu().numpy(), seeds * m, np.eye(d))
    for a in (np.array([1.0, 0.0]), np.array([0.6, 0.8])):
        assert stats.kstest(np.concatenate(rows) @ a, "norm").pvalue > 1e-4
    norms = np.asarray(norms)
    assert abs(norms.mean() - m * d) < 5 * norms.std(ddof=1) / math.sqrt(seeds)


def test_nmf_anchors_match_oracle():
    n, d, m, B, seed = 20000, 50, 24, 2048, 21
    X = synth.csr_bernoulli(n, d, 0.05, seed=4, values="uniform")
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(X.col_idx).cuda()
    v = torch.from_numpy(X.vals).cuda()
    Z, imax, imin = cg().CountGauss(n, d, m, B, seed).nmf_anchors(rp, ci, v)
    Zn = Z.cpu().numpy()
    # step 3 on the device's own Z: exact (index work)
    np.testing.assert_array_equal(imax.cpu().numpy(), np.argmax(Zn, axis=1))
    np.testing.assert_array_equal(imin.cpu().numpy(), np.argmin(Zn, axis=1))
    # and against the oracle's Z, where the top two entries of a row are not within
    # the fp32 error of each other
    Zo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals)
    omax, omin = oracle.row_argmax_argmin(Zo)
    srt = np.sort(Zo, axis=1)
    scale = np.abs(Zo).max(axis=1)
    clear_max = (srt[:, -1] - srt[:, -2]) > 1e-4 * scale
    clear_min = (srt[:, 1] - srt[:, 0]) > 1e-4 * scale
    np.testing.assert_array_equal(imax.cpu().numpy()[clear_max], omax[clear_max])
    np.testing.assert_array_equal(imin.cpu().numpy()[clear_min], omin[clear_min])


@pytest.mark.parametrize("d,m,precision", [(50, 24, "fp32"), (300, 5, "fp32"), (1500, 3, "fp32"), (64, 1, "fp32"),
                                           (128, 128, "bf16"), (40, 9, "fp8")])
def test_fused_anchors_against_row_argmax_and_oracle(d, m, precision):
    """Algorithm 1 step 3 inside the split-K sum (one thread block per row of Z): Z within
    fp32 rounding of cg_apply_csr's, imax / imin exactly the row argmax / argmin of that Z
    (lowest index on ties), for rows of one to 47 column chunks and every contraction."""
    n, B, seed = 6000, 1024, 29
    X = synth.csr_bernoulli(n, d, 0.05, seed=4, values="uniform")
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(X.col_idx).cuda()
    v = torch.from_numpy(X.vals).cuda()
    plan = cg().CountGauss(n, d, m, B, seed, precision=precision)
    Z, imax, imin = plan.nmf_anchors(rp, ci, v)
    Y = plan.apply_csr(rp, ci, v)
    plan.check()
    Zn = Z.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(Zn - Y.cpu().numpy()) <= 1e-6 * np.linalg.norm(Zn)
    np.testing.assert_array_equal(imax.cpu().numpy(), np.argmax(Zn, axis=1))
    np.testing.assert_array_equal(imin.cpu().numpy(), np.argmin(Zn, axis=1))
    if precision == "fp32":
        Zo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals)
        assert np.linalg.norm(Zn - Zo) <= 1e-5 * np.linalg.norm(Zo)


def test_fused_anchors_ties_take_lowest_column():
    """Columns 5 and 17 of X equal, so columns 5 and 17 of Z are equal bit for bit (the
    deterministic scatter's sums do not depend on order); the fused step 3 reports the
    lower column wherever they hold a row's maximum or minimum."""
    n, d, m, B, seed = 4000, 24, 32, 256, 31
    Xd = synth.csr_bernoulli(n, d, 0.1, seed=5, values="uniform").to_dense()
    Xd[:, 5] = 0.0
    Xd[::3, 5] = 50.0  # large, so that column 5 often holds the max or the min
    Xd[:, 17] = Xd[:, 5]
    X = synth.csr_from_dense(Xd)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(X.col_idx).cuda()
    v = torch.from_numpy(X.vals).cuda()
    plan = cg().CountGauss(n, d, m, B, seed, deterministic=True)
    Z, imax, imin = plan.nmf_anchors(rp, ci, v)
    plan.check()
    Zn = Z.cpu().numpy()
    np.testing.assert_array_equal(Zn[:, 5], Zn[:, 17])
    im, jm = imax.cpu().numpy(), imin.cpu().numpy()
    np.testing.assert_array_equal(im, np.argmax(Zn, axis=1))
    np.testing.assert_array_equal(jm, np.argmin(Zn, axis=1))
    assert (im == 5).sum() + (jm == 5).sum() > 0 and not ((im == 17).any() or (jm == 17).any())


def test_argmax_ties_take_lowest_index():
    Z = torch.tensor([[1.0, 3.0, 3.0, -2.0, -2.0], [0.0, 0.0, 0.0, 0.0, 0.0]], device="cuda")
    imax, imin = cg().row_argmax_argmin(Z)
    assert imax.cpu().tolist() == [1, 0]
    assert imin.cpu().tolist() == [3, 0]

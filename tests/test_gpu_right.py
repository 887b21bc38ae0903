"""Parity of the right projection Z = A.T^T (the random projection X.R, R = T^T, of the
SVM application, Section 9; Table 1) with the FP64 oracle, through the C ABI.

A has one row per document and one column per word (TechTC-300-shaped synthetic
pairs).  Bar: relative Frobenius error 1e-5 for FP32 and split-BF16x3, 2e-2 for BF16
and FP8x3.  Expected values come from the oracle only.
"""
import numpy as np
import pytest

import oracle
from paper_1606_05732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def cg():
    from paper_1606_05732_gb300 import countgauss
    return countgauss


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def dev_csr(A):
    return (torch.from_numpy(A.row_ptr.astype(np.int32)).cuda(),
            torch.from_numpy(A.col_idx.astype(np.int32)).cuda(),
            torch.from_numpy(A.vals.astype(np.float32)).cuda())


def project(A, m, B, seed, **kw):
    """Z = A.T^T on the GPU: a plan with n = words (columns of A), d = documents."""
    plan = cg().CountGauss(A.d, A.n, m, B, seed, **kw)
    Z = plan.apply_right_csr(*dev_csr(A)).cpu().numpy()
    plan.check()
    return Z


def expect(A, m, B, seed, col_offset=0):
    return oracle.apply_right_csr(seed, A.d, A.n, m, B, A.row_ptr, A.col_idx, A.vals, col_offset=col_offset)


@pytest.mark.parametrize("docs,words,m,seed", [(150, 10_000, 128, 11), (211, 23_456, 256, 12), (97, 3001, 7, 13)])
def test_techtc_shapes(docs, words, m, seed):
    """TechTC-shaped pairs with B = 5m (Section 5), B not a power of two."""
    A = synth.techtc_pair(seed, docs=docs, words=words)
    B = 5 * m
    Z = project(A, m, B, seed)
    assert Z.shape == (docs, m)
    assert rel(Z, expect(A, m, B, seed)) < FP32_TOL


def test_largest_techtc_pair_m512():
    """The largest pair (280 documents x 40,000 words, 112 K nonzeros) at m = 512,
    B = 2560, the configuration of the last block of Table 1."""
    A = synth.techtc_pair(21, docs=280, words=40_000)
    Z = project(A, 512, 2560, 21)
    assert rel(Z, expect(A, 512, 2560, 21)) < FP32_TOL


@pytest.mark.parametrize("precision,tol", [("bf16x3", 1e-5), ("bf16", 2e-2), ("fp8x3", 2e-2)])
def test_precisions(precision, tol):
    A = synth.techtc_pair(31, docs=180, words=15_000)
    Z = project(A, 256, 1280, 31, precision=precision)
    err = rel(Z, expect(A, 256, 1280, 31))
    print(f"{precision}: rel {err:.3e}")
    assert err < tol


def test_column_code_table():
    """Many documents over few words (nnz > 4 n): the scatter looks the hash and sign
    up in a per-column table instead of drawing them per nonzero."""
    A = synth.csr_bernoulli(3000, 500, 0.05, seed=41, values="uniform")
    assert A.nnz > 4 * A.d
    Z = project(A, 64, 320, 41)
    assert rel(Z, expect(A, 64, 320, 41)) < FP32_TOL
    # with a global column offset the table is drawn for the offset columns
    Zo = project(A, 64, 320, 41, row_offset=70_000)
    assert rel(Zo, expect(A, 64, 320, 41, col_offset=70_000)) < FP32_TOL
    # more documents than the row offsets staged in shared memory (4095)
    A2 = synth.csr_bernoulli(6000, 300, 0.02, seed=42, values="uniform")
    assert A2.nnz > 4 * A2.d
    assert rel(project(A2, 32, 160, 42), expect(A2, 32, 160, 42)) < FP32_TOL


def test_equals_left_transform_of_transpose():
    """A.T^T = (T.A^T)^T: the right projection against cg_apply_csr on A^T (same GPU,
    different scatter and summation order)."""
    A = synth.techtc_pair(51, docs=160, words=12_000)
    At = synth.csr_from_dense(A.to_dense().T)
    plan = cg().CountGauss(A.d, A.n, 128, 640, 51)
    Z = plan.apply_right_csr(*dev_csr(A)).cpu().numpy()
    Y = plan.apply_csr(*dev_csr(At)).cpu().numpy()
    plan.check()
    assert rel(Z, Y.T) < 1e-6


def test_edges():
    """Empty matrix, one document, documents without words, a column offset, ragged
    rows with unsorted columns."""
    m, B, seed = 16, 80, 61
    empty = synth.csr_bernoulli(20, 300, 0.0, seed=1)
    assert not project(empty, m, B, seed).any()
    one = synth.csr_bernoulli(1, 5000, 0.02, seed=2)
    assert rel(project(one, m, B, seed), expect(one, m, B, seed)) < FP32_TOL
    ragged = synth.csr_ragged(400, 700, seed=3, empty_frac=0.5)
    assert rel(project(ragged, m, B, seed), expect(ragged, m, B, seed)) < FP32_TOL
    assert rel(project(ragged, m, B, seed, row_offset=12345),
               expect(ragged, m, B, seed, col_offset=12345)) < FP32_TOL
    sparse = synth.csr_ragged(5000, 64, seed=4, empty_frac=0.9, max_row=3)  # many short rows
    assert rel(project(sparse, m, B, seed), expect(sparse, m, B, seed)) < FP32_TOL


def test_bad_inputs_are_reported():
    """An out-of-range word index and decreasing row offsets are skipped and reported
    through the status word; the plan is usable afterwards."""
    A = synth.techtc_pair(71, docs=50, words=2000)
    rp, ci, v = dev_csr(A)
    plan = cg().CountGauss(A.d, A.n, 32, 160, 71)
    bad_ci = ci.clone()
    bad_ci[A.nnz // 2] = A.d + 7
    plan.apply_right_csr(rp, bad_ci, v)
    with pytest.raises(cg()._lib.CountGaussError):
        plan.check()
    bad_rp = rp.clone()
    r = A.n // 2
    bad_rp[r], bad_rp[r + 1] = rp[r + 1].item() + 1, rp[r].item()
    plan.apply_right_csr(bad_rp, ci, v)
    with pytest.raises(cg()._lib.CountGaussError):
        plan.check()
    Z = plan.apply_right_csr(rp, ci, v).cpu().numpy()
    plan.check()
    assert rel(Z, expect(A, 32, 160, 71)) < FP32_TOL
    with pytest.raises(ValueError):
        plan.apply_right_csr(rp[:-1], ci, v)

"""Host-side pieces of the distance diagnostics (Theorem 1's proof, Lemma 5), without a
GPU: Claim 3's KL divergence against numerical integration, its second-order form,
Pinsker's bound, the test matrices, and the Frobenius closed form against the oracle's
sketches."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1606_05732_gb300 import diagnostics as dg


def _kl_by_integration_1d(var):
    lp = lambda x: -0.5 * x * x - 0.5 * math.log(2 * math.pi)
    lq = lambda x: -0.5 * x * x / var - 0.5 * math.log(2 * math.pi * var)
    val, _ = integrate.quad(lambda x: math.exp(lp(x)) * (lp(x) - lq(x)), -30, 30, epsabs=1e-13, epsrel=1e-12)
    return val


def _kl_by_integration_2d(M):
    Mi = np.linalg.inv(M)
    det = np.linalg.det(M)

    def f(y, x):
        v = np.array([x, y])
        lp = -0.5 * v @ v - math.log(2 * math.pi)
        lq = -0.5 * v @ Mi @ v - math.log(2 * math.pi) - 0.5 * math.log(det)
        return math.exp(lp) * (lp - lq)
    val, _ = integrate.dblquad(f, -12, 12, -12, 12, epsabs=1e-11, epsrel=1e-9)
    return val


@pytest.mark.parametrize("var", [0.25, 0.9, 1.0, 1.7, 6.0])
def test_kl_matches_integration_1d(var):
    """Claim 3 in one dimension against the integral of p ln(p/q)."""
    assert dg.gaussian_kl(np.array([[var]])) == pytest.approx(_kl_by_integration_1d(var), abs=1e-9)


def test_kl_matches_integration_2d():
    M = np.array([[1.3, 0.4], [0.4, 0.8]])
    assert dg.gaussian_kl(M) == pytest.approx(_kl_by_integration_2d(M), abs=1e-7)


def test_kl_identity_zero_and_singular_infinite():
    assert dg.gaussian_kl(np.eye(7)) == 0.0
    assert dg.gaussian_kl(np.diag([1.0, 0.0, 2.0])) == math.inf
    assert dg.tv_upper_bound(math.inf, 4) == 1.0


def test_kl_second_order_is_quarter_frobenius():
    """For M = I + eps E the series of Claims 1-2 leaves 1/4 ||I - M||_F^2 at second order."""
    rng = np.random.default_rng(3)
    E = rng.standard_normal((6, 6))
    E = 0.5 * (E + E.T)
    for eps in (1e-2, 1e-3):
        M = np.eye(6) + eps * E
        ratio = dg.gaussian_kl(M) / (0.25 * np.sum((eps * E) ** 2))
        assert abs(ratio - 1.0) < 5 * eps * np.linalg.norm(E, 2)


def test_kl_rotation_invariant_and_positive():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((5, 5))
    M = A @ A.T / 5 + 0.1 * np.eye(5)
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    assert dg.gaussian_kl(Q @ M @ Q.T) == pytest.approx(dg.gaussian_kl(M), rel=1e-10)
    assert dg.gaussian_kl(M) > 0


def test_pinsker_bound():
    assert dg.tv_upper_bound(0.0, 10) == 0.0
    assert dg.tv_upper_bound(0.02, 10) == pytest.approx(math.sqrt(0.1))
    assert dg.tv_upper_bound(1.0, 10) == 1.0


@pytest.mark.parametrize("make", [lambda: dg.spread_orthonormal_csr(1000, 7), lambda: dg.lemma5_block_csr(4, 16),
                                  lambda: dg.lemma5_block_csr(8, 5000)])
def test_test_matrices_have_orthonormal_columns(make):
    U = make().to_dense()
    np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-6)


def test_lemma5_block_sizes():
    U = dg.lemma5_block_csr(4, 16)  # L = ceil(4 / 4) = 1: U is the identity
    assert U.n == 4 and U.nnz == 4
    U = dg.lemma5_block_csr(8, 5000)  # L = ceil(70.7 / 8) = 9
    assert U.n == 72 and np.all(np.bincount(U.col_idx) == 9)


def test_frobenius_closed_form_against_oracle_sketches():
    """E_S ||U^T S^T S U - I||_F^2 over 3000 oracle CountSketches of a spread U."""
    n, d, B = 60, 4, 16
    U = dg.spread_orthonormal_csr(n, d)
    Ud = U.to_dense()
    vals = []
    for s in range(3000):
        SU = oracle.sketch_csr(s, n, d, B, U.row_ptr, U.col_idx, U.vals)
        vals.append(np.sum((SU.T @ SU - np.eye(d)) ** 2))
    want = dg.frobenius_closed_form(np.sum(Ud ** 2, axis=1), d, B)
    vals = np.array(vals)
    assert abs(vals.mean() - want) < 5 * vals.std() / math.sqrt(len(vals))

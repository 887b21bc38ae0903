"""The distance diagnostics on the device (Theorem 1's proof, Lemma 5): the FP64 sketch
Gram against the oracle, the KL sweep against the closed forms, and Lemma 5's
distinguisher on the device's own T.U and G~.U."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dg():
    from paper_1606_05732_gb300 import diagnostics
    return diagnostics


def test_sketch_gram_matches_oracle():
    U = dg().spread_orthonormal_csr(1 << 16, 8)
    from paper_1606_05732_gb300 import countgauss
    plan = countgauss.CountGauss(U.n, U.d, 4, 1024, 7)
    rp, ci, v = (torch.from_numpy(a).cuda() for a in (U.row_ptr.astype(np.int32), U.col_idx, U.vals))
    M = dg().sketch_gram(plan, rp, ci, v)
    SU = oracle.sketch_csr(7, U.n, U.d, 1024, U.row_ptr, U.col_idx, U.vals)
    Mo = SU.T @ SU
    assert np.linalg.norm(M - Mo) / np.linalg.norm(Mo) < 1e-6
    assert abs(dg().gaussian_kl(M) - dg().gaussian_kl(Mo)) < 1e-5 * max(1.0, dg().gaussian_kl(Mo))


def test_kl_sweep_follows_closed_forms():
    """||M - I||_F^2 averages to (d^2 + d - 2 sum ||u_k||^4) / B; the KL divergence falls
    with B and approaches 1/4 ||M - I||_F^2 (second order of Claims 1-2) once M is close
    to I; Pinsker's bound on m rows falls below 0.1 only for B well above d^2 m."""
    U = dg().spread_orthonormal_csr(1 << 18, 16)
    m = 8
    rows = dg().kl_sweep(U, m, [1 << 10, 1 << 12, 1 << 14, 1 << 16], range(128))
    for r in rows:
        print({k: (round(v, 6) if isinstance(v, float) else v) for k, v in r.items()})
        se = r["frob2_sd"] / math.sqrt(r["samples"])
        assert abs(r["frob2_mean"] - r["frob2_closed_form"]) < 5 * se
    kls = [r["kl_mean"] for r in rows]
    assert all(a > b for a, b in zip(kls, kls[1:]))
    last = rows[-1]
    assert abs(last["kl_mean"] / (0.25 * last["frob2_mean"]) - 1.0) < 0.1
    assert rows[0]["tv_bound_at_median_kl"] > 0.3 and last["tv_bound_at_median_kl"] < 0.1


def test_lemma5_distinguisher_on_device():
    """Lemma 5 on the device: at B = 16 (L = 1, a collision between blocks in about a
    third of the draws) the pair-norm statistic separates T.U from G~.U; at B = 2^13
    (L = 23) the 2/L effect is buried in the chi-square noise."""
    from scipy import stats
    small = dg().lemma5_experiment(4, 32, 16, range(300))
    assert stats.ks_2samp(small["countgauss"], small["plain"]).pvalue < 1e-6
    large = dg().lemma5_experiment(4, 32, 1 << 13, range(300))
    assert stats.ks_2samp(large["countgauss"], large["plain"]).pvalue > 1e-4


def test_pair_norm_statistic_matches_numpy():
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((32, 6)).astype(np.float32)
    want = max(abs(np.sum((Y[:, i].astype(np.float64) + Y[:, j]) ** 2) / 32 - 2.0)
               for i in range(6) for j in range(i + 1, 6))
    assert dg().pair_norm_statistic(torch.from_numpy(Y).cuda()) == pytest.approx(want, rel=1e-6)

"""Seeded random shapes through every scatter form and the FP32 and BF16x3 contractions,
against the FP64 oracle: n, d, m, B and the density drawn over wide ranges (ragged rows
with empty ones, a global row offset), so that grid edges, partial tiles, thread tiles
left idle and slice boundaries fall at places the fixed-shape tests do not choose.
Bar: every SX entry within the worst-case bound of fp32 summation in any order,
gamma_N sum |x| (N the terms of the entry, gamma_N = N u / (1 - N u), u = 2^-24; some drawn
shapes put thousands of cancelling terms into each entry, where a relative Frobenius bar
of 1e-6 does not hold for any fp32 order); Y within 1e-5 (relative Frobenius); the two
deterministic forms bit-identical to each other.
"""
import numpy as np
import pytest

import oracle
from paper_1606_05732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
SCATTERS = ["auto", "atomic", "deferred", "binned", "partition"]


def cg():
    from paper_1606_05732_gb300 import countgauss
    return countgauss


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def sx_bound(seed, n, d, B, X, offset):
    """gamma_N sum |x| per entry of SX (N: the entry's number of terms)."""
    h, _ = oracle.hash_sign(seed, B, offset, n)
    rows = np.repeat(np.arange(n), np.diff(X.row_ptr))
    A = np.zeros((B, d))
    N = np.zeros((B, d))
    np.add.at(A, (h[rows], X.col_idx), np.abs(X.vals.astype(np.float64)))
    np.add.at(N, (h[rows], X.col_idx), 1.0)
    u = 2.0 ** -24
    return N * u / (1.0 - N * u) * A


def draw_case(k):
    """Case k: a shape with at most about 4e5 nonzeros and m B d at most about 3e7."""
    rng = np.random.default_rng(1000 + k)
    n = int(np.exp(rng.uniform(np.log(16), np.log(200000))))
    d = int(np.exp(rng.uniform(0, np.log(300))))
    m = int(np.exp(rng.uniform(0, np.log(200))))
    B = int(np.exp(rng.uniform(0, np.log(20000))))
    while m * B * d > 3e7:
        B = max(1, B // 2)
    max_row = int(min(d, max(1, 4e5 // max(n, 1))))
    offset = int(rng.integers(0, 1 << 40))
    return n, max(1, d), max(1, m), max(1, B), 300 + k, max_row, offset


@pytest.mark.parametrize("k", range(48))
def test_random_shape_every_scatter(k):
    n, d, m, B, seed, max_row, offset = draw_case(k)
    X = synth.csr_ragged(n, d, seed=seed, max_row=max_row)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(X.col_idx.astype(np.int32)).cuda()
    v = torch.from_numpy(X.vals.astype(np.float32)).cuda()
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, row_offset=offset, return_sx=True)
    bound = sx_bound(seed, n, d, B, X, offset)
    for scatter in SCATTERS:
        plan = cg().CountGauss(n, d, m, B, seed, scatter=scatter, row_offset=offset)
        SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
        Y = plan.apply_csr(rp, ci, v).cpu().numpy()
        plan.check()
        assert (np.abs(SX - SXo) <= bound).all(), (scatter, n, d, m, B)
        assert rel(Y, Yo) < FP32_TOL, (scatter, n, d, m, B)
    dets = []
    for scatter in ("atomic", "binned"):
        plan = cg().CountGauss(n, d, m, B, seed, deterministic=True, scatter=scatter, row_offset=offset)
        dets.append(plan.sketch_csr(rp, ci, v).cpu().numpy())
        plan.check()
    np.testing.assert_array_equal(dets[0], dets[1])
    assert (np.abs(dets[0] - SXo) <= bound).all()
    # BF16x3 carries about 16 bits of each operand; its 1e-5 bar is a statement about sums
    # of many products, so it is checked where each entry of Y sums at least 256 of them
    if B >= 256 and m * d >= 64:
        plan = cg().CountGauss(n, d, m, B, seed, precision="bf16x3", row_offset=offset)
        Yb = plan.apply_csr(rp, ci, v).cpu().numpy()
        plan.check()
        assert rel(Yb, Yo) < FP32_TOL, ("bf16x3", n, d, m, B)


@pytest.mark.parametrize("k", range(24))
def test_random_shape_plain_and_adjoint(k):
    """The plain product G~ X and the adjoint at the stored entries, dX_k = sigma(i)
    (G^T dY)[h(i), col_k], on the same random shapes."""
    n, d, m, B, seed, max_row, offset = draw_case(k)
    X = synth.csr_ragged(n, d, seed=seed, max_row=max_row)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(X.col_idx.astype(np.int32)).cuda()
    v = torch.from_numpy(X.vals.astype(np.float32)).cuda()
    plan = cg().CountGauss(n, d, m, B, seed, row_offset=offset)
    Yp = plan.plain_csr(rp, ci, v).cpu().numpy()
    dYn = np.random.default_rng(seed).standard_normal((m, d)).astype(np.float32)
    dXv = plan.adjoint(torch.from_numpy(dYn).cuda(), rp, ci).cpu().numpy()
    plan.check()
    assert rel(Yp, oracle.plain_csr(seed, n, d, m, X.row_ptr, X.col_idx, X.vals, row_offset=offset)) < FP32_TOL
    assert rel(dXv, oracle.adjoint_csr(seed, n, m, B, X.row_ptr, X.col_idx, dYn, row_offset=offset)) < FP32_TOL

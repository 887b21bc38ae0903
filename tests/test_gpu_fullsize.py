"""Parity at the benchmark sizes, in the launch configuration the benchmark uses.

The CountGauss output is compared in full (the oracle sketches all nonzeros and
contracts in FP64); the plain product G~.X is compared on sampled output rows,
which the oracle computes row by row (row r of G~.X depends on row r of G~ only):
the first and last group of four rows plus one more group.
"""
import numpy as np
import pytest

import oracle
from paper_1606_05732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_workload(name):
    from paper_1606_05732_gb300 import countgauss
    X, w = synth.workload_csr(name)
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(X.col_idx).to(dev)
    v = torch.from_numpy(X.vals).to(dev)
    plan = countgauss.CountGauss(X.n, X.d, w["m"], w["B"], w["seed"])
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    Yp = plan.plain_csr(rp, ci, v).cpu().numpy()
    plan.check()
    del rp, ci, v
    return X, w, Y, Yp


@pytest.mark.parametrize("name", ["nmf_n16M_d64", "ladder_n64M_d128"])
def test_fullsize_fp32(name):
    X, w, Y, Yp = run_workload(name)
    Yo = oracle.apply_csr(w["seed"], X.n, X.d, w["m"], w["B"], X.row_ptr, X.col_idx, X.vals)
    err = rel(Y, Yo)
    print(f"{name}: CountGauss fp32 rel Frobenius error {err:.3e}")
    assert err < FP32_TOL
    rows = synth.sample_rows(w["m"], seed=w["seed"], groups=3)
    Ypo = oracle.plain_csr(w["seed"], X.n, X.d, w["m"], X.row_ptr, X.col_idx, X.vals, rows=rows)
    errp = rel(Yp[rows], Ypo)
    print(f"{name}: plain fp32 rel Frobenius error on rows {rows.tolist()}: {errp:.3e}")
    assert errp < FP32_TOL


@pytest.fixture(scope="module")
def ladder_case():
    X, w = synth.workload_csr("ladder_n64M_d128")
    Yo = oracle.apply_csr(w["seed"], X.n, X.d, w["m"], w["B"], X.row_ptr, X.col_idx, X.vals)
    return X, w, Yo


@pytest.mark.parametrize("precision,bound", [("bf16x3", 1e-5), ("bf16", 2e-2), ("fp8x3", 2e-2), ("fp8", 5e-2)])
def test_fullsize_precision_ladder(ladder_case, precision, bound):
    from paper_1606_05732_gb300 import countgauss
    X, w, Yo = ladder_case
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(X.col_idx).to(dev)
    v = torch.from_numpy(X.vals).to(dev)
    plan = countgauss.CountGauss(X.n, X.d, w["m"], w["B"], w["seed"], precision=precision)
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    err = rel(Y, Yo)
    print(f"ladder_n64M_d128 {precision}: rel Frobenius error {err:.3e} (bound {bound})")
    assert err < bound


def test_fullsize_batch_96_instances():
    """The 96-instance batch (seeds 100..195), autotuned, every output against the oracle."""
    from paper_1606_05732_gb300 import countgauss
    params = synth.batch_instances()
    Xs = synth.batch_inputs(params)
    insts = [dict(n=t.n, d=t.d, m=t.m, B=t.B, seed=t.seed,
                  row_ptr=torch.from_numpy(X.row_ptr.astype(np.int32)).cuda(),
                  col_idx=torch.from_numpy(X.col_idx).cuda(), vals=torch.from_numpy(X.vals).cuda())
             for t, X in zip(params, Xs)]
    batch = countgauss.CountGaussBatch(insts)
    batch.autotune(reps=2)
    Ys = [y.cpu().numpy() for y in batch.apply()]
    batch.check()
    worst = 0.0
    for t, X, Y in zip(params, Xs, Ys):
        Yo = oracle.apply_csr(t.seed, t.n, t.d, t.m, t.B, X.row_ptr, X.col_idx, X.vals)
        worst = max(worst, rel(Y, Yo))
    print(f"batch of 96: worst rel Frobenius error {worst:.3e}")
    assert worst < FP32_TOL


def test_fullsize_grad_dense_forward_and_adjoints():
    """The differentiation workload at its benchmark size: dense X 2^20 x 64, m = 64,
    B = 2^16 (forward through the dense sketch, adjoint as a dense gather), and the
    adjoint read at the 1.34 M stored entries of the p = 0.02 pattern, all against the
    oracle in full."""
    from paper_1606_05732_gb300 import countgauss
    w = synth.WORKLOADS["grad_n1M_d64"]
    n, d, m, B, seed = w["n"], w["d"], w["m"], w["B"], w["seed"]
    Xd = synth.dense_normal(n, d, seed=seed)
    Xs = synth.csr_bernoulli(n, d, w["p"], seed=seed)
    dY = np.random.default_rng(seed + 1).standard_normal((m, d)).astype(np.float32)
    dev = torch.device("cuda", 0)
    plan = countgauss.CountGauss(n, d, m, B, seed)
    Y = plan.apply_dense(torch.from_numpy(Xd).to(dev)).cpu().numpy()
    dX = plan.adjoint(torch.from_numpy(dY).to(dev)).cpu().numpy()
    rp = torch.from_numpy(Xs.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(Xs.col_idx).to(dev)
    dXs = plan.adjoint(torch.from_numpy(dY).to(dev), rp, ci).cpu().numpy()
    plan.check()
    err_f = rel(Y, oracle.apply_dense(seed, m, B, Xd.astype(np.float64)))
    dY64 = dY.astype(np.float64)
    err_d = rel(dX, oracle.adjoint_dense(seed, n, m, B, dY64))
    err_s = rel(dXs, oracle.adjoint_csr(seed, n, m, B, Xs.row_ptr, Xs.col_idx, dY64))
    print(f"grad_n1M_d64: forward {err_f:.3e}, dense adjoint {err_d:.3e}, CSR adjoint {err_s:.3e}")
    assert err_f < FP32_TOL and err_d < FP32_TOL and err_s < FP32_TOL


def test_fullsize_deterministic_mode_nmf():
    """Deterministic mode at the NMF-like workload's full size (53.7 M nonzeros, the
    largest nnz of its tests, so the coarsest fixed-point resolution): two runs are
    bit-identical and every SX entry is within one fp32 ulp plus the fixed-point
    resolution per term (2^(L+e-62), 2^e > max|x|, 2^L > nnz) of the oracle's FP64 sum."""
    from paper_1606_05732_gb300 import countgauss
    X, w = synth.workload_csr("nmf_n16M_d64")
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(X.col_idx).to(dev)
    v = torch.from_numpy(X.vals).to(dev)
    plan = countgauss.CountGauss(X.n, X.d, w["m"], w["B"], w["seed"], deterministic=True)
    SX1 = plan.sketch_csr(rp, ci, v).cpu().numpy()
    SX2 = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    del rp, ci, v
    np.testing.assert_array_equal(SX1, SX2)
    Yo, SXo = oracle.apply_csr(w["seed"], X.n, X.d, w["m"], w["B"], X.row_ptr, X.col_idx, X.vals, return_sx=True)
    want = SXo.astype(np.float32)
    L = max(1, int(X.nnz).bit_length())
    e = int(np.frexp(np.abs(X.vals).max())[1])
    per_term = 2.0 ** (L + e - 62)
    rows_per_bucket = np.bincount(oracle.hash_sign(w["seed"], w["B"], 0, X.n)[0], minlength=w["B"])
    bound = np.spacing(np.abs(want)).astype(np.float64) + (rows_per_bucket[:, None] + 1) * per_term
    assert (np.abs(SX1.astype(np.float64) - SXo) <= bound).all()
    assert (SX1 == want).mean() > 0.99
    assert rel(Y, Yo) < FP32_TOL


def test_fullsize_deterministic_mode_ladder():
    """Deterministic mode at the largest workload (2^26 x 128, 85.9 M nonzeros), whose int64
    accumulator (268 MB) is past the L2, so the automatic form sums bucket slices in shared
    memory: bit-identical over two runs and to the global-accumulator form
    (CG_OPT_SCATTER = 1), every SX entry within one fp32 ulp plus the fixed-point resolution
    per term of the oracle's FP64 sum, and Y within the FP32 bar."""
    from paper_1606_05732_gb300 import countgauss
    X, w = synth.workload_csr("ladder_n64M_d128")
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(X.col_idx).to(dev)
    v = torch.from_numpy(X.vals).to(dev)
    plan = countgauss.CountGauss(X.n, X.d, w["m"], w["B"], w["seed"], deterministic=True)
    SX1 = plan.sketch_csr(rp, ci, v).cpu().numpy()
    SX2 = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    del plan
    glob = countgauss.CountGauss(X.n, X.d, w["m"], w["B"], w["seed"], deterministic=True, scatter="atomic")
    SXg = glob.sketch_csr(rp, ci, v).cpu().numpy()
    glob.check()
    del glob, rp, ci, v
    torch.cuda.empty_cache()
    np.testing.assert_array_equal(SX1, SX2)
    np.testing.assert_array_equal(SX1, SXg)
    Yo, SXo = oracle.apply_csr(w["seed"], X.n, X.d, w["m"], w["B"], X.row_ptr, X.col_idx, X.vals, return_sx=True)
    want = SXo.astype(np.float32)
    L = max(1, int(X.nnz).bit_length())
    e = int(np.frexp(np.abs(X.vals).max())[1])
    per_term = 2.0 ** (L + e - 62)
    rows_per_bucket = np.bincount(oracle.hash_sign(w["seed"], w["B"], 0, X.n)[0], minlength=w["B"])
    bound = np.spacing(np.abs(want)).astype(np.float64) + (rows_per_bucket[:, None] + 1) * per_term
    assert (np.abs(SX1.astype(np.float64) - SXo) <= bound).all()
    assert rel(Y, Yo) < FP32_TOL

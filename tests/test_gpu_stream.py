"""Streaming and resuming the sketch: S.X is additive over the rows of X, so row chunks
fed with their global row offsets and CG_OPT_ACCUMULATE build the sketch of the whole
matrix, and a saved SX plus the next row offset resumes an interrupted stream (the
streaming setting of Section 1.1; the seed and the global index fix S)."""
import numpy as np
import pytest

import oracle
from paper_1606_05732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cg():
    from paper_1606_05732_gb300 import countgauss
    return countgauss


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def chunk(X, a, b):
    k0, k1 = int(X.row_ptr[a]), int(X.row_ptr[b])
    return (torch.from_numpy((X.row_ptr[a:b + 1] - k0).astype(np.int32)).cuda(),
            torch.from_numpy(X.col_idx[k0:k1].astype(np.int32)).cuda(),
            torch.from_numpy(X.vals[k0:k1].astype(np.float32)).cuda())


@pytest.mark.parametrize("scatter", ["atomic", "deferred", "binned"])
def test_streamed_chunks_and_resume(scatter):
    n, d, m, B, seed = 30011, 24, 16, 2048, 31
    X = synth.csr_bernoulli(n, d, 0.05, seed=seed)
    cuts = [0, 9000, 21000, n]
    SX = torch.zeros(B, d, dtype=torch.float32, device="cuda")
    saved = None
    for c, (a, b) in enumerate(zip(cuts, cuts[1:])):
        plan = cg().CountGauss(b - a, d, m, B, seed, scatter=scatter, row_offset=a)
        plan.sketch_csr(*chunk(X, a, b), out=SX, accumulate=True)
        plan.check()
        if c == 1:
            saved = SX.cpu().clone()  # checkpoint: SX and the next row offset, 21000
    SXo = oracle.sketch_csr(seed, n, d, B, X.row_ptr, X.col_idx, X.vals)
    assert rel(SX.cpu(), SXo) < 1e-6
    whole = cg().CountGauss(n, d, m, B, seed, scatter=scatter).sketch_csr(*chunk(X, 0, n))
    assert rel(SX.cpu(), whole.cpu()) < 1e-6
    # resume from the checkpoint into a fresh buffer with a fresh plan
    SX2 = saved.cuda()
    last = cg().CountGauss(n - 21000, d, m, B, seed, scatter=scatter, row_offset=21000)
    last.sketch_csr(*chunk(X, 21000, n), out=SX2, accumulate=True)
    assert rel(SX2.cpu(), SXo) < 1e-6
    Y = cg().CountGauss(n, d, m, B, seed).contract(SX2).cpu().numpy()
    assert rel(Y, oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals)) < 1e-5


def test_dense_accumulate_and_errors():
    from paper_1606_05732_gb300 import _lib
    n, d, m, B, seed = 5000, 16, 8, 512, 41
    Xd = synth.dense_normal(n, d, seed=seed)
    SX = torch.zeros(B, d, dtype=torch.float32, device="cuda")
    for a, b in [(0, 1234), (1234, n)]:
        plan = cg().CountGauss(b - a, d, m, B, seed, row_offset=a)
        plan.sketch_dense(torch.from_numpy(Xd[a:b]).cuda(), out=SX, accumulate=True)
        plan.check()
    assert rel(SX.cpu(), oracle.sketch_dense(seed, B, Xd.astype(np.float64))) < 1e-6
    # the default still overwrites
    plan = cg().CountGauss(n, d, m, B, seed)
    plan.sketch_dense(torch.from_numpy(Xd).cuda(), out=SX)
    assert rel(SX.cpu(), oracle.sketch_dense(seed, B, Xd.astype(np.float64))) < 1e-6
    with pytest.raises(ValueError):
        plan.sketch_dense(torch.from_numpy(Xd).cuda(), accumulate=True)
    det = cg().CountGauss(n, d, m, B, seed, deterministic=True)
    X = synth.csr_bernoulli(n, d, 0.05, seed=seed)
    with pytest.raises(_lib.CountGaussError):
        det.sketch_csr(*chunk(X, 0, n), out=SX, accumulate=True)

"""cg_apply_csr_noalloc: the CSR transform for callers that cannot allocate device
memory when they call it (inside allocator callbacks, plugins given only their
input and output buffers, real-time loops that ban cudaMalloc/cudaFree after
start-up).  Its scratch is a fixed device array inside the library, so the test
checks, through the C ABI, that two calls in a row match the workspace entry point
cg_apply_csr and the FP64 oracle within the FP32 tolerance (also for a row shard with
a global row offset), and that plans needing more scratch than the array holds are
refused.

This file sorts last so that a run stopping at its first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1606_05732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
P = ctypes.c_void_p


def rel(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b.astype(np.float64)) / np.linalg.norm(b.astype(np.float64)))


def _stream():
    return P(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("n,d,m,B,seed,p,offset", [(65536, 16, 8, 4096, 1, 0.05, 0), (4099, 37, 13, 1000, 7, 0.2, 0),
                                                    (30011, 24, 16, 2048, 31, 0.05, 21000)])
def test_noalloc_matches_workspace_entry_point(n, d, m, B, seed, p, offset):
    from paper_1606_05732_gb300 import _lib, countgauss
    lib = _lib.load()
    X = synth.csr_bernoulli(n, d, p, seed=seed)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(X.col_idx).cuda()
    v = torch.from_numpy(X.vals).cuda()
    plan = countgauss.CountGauss(n, d, m, B, seed, row_offset=offset)
    want = plan.apply_csr(rp, ci, v).cpu().numpy()  # existing entry point, caller workspace
    exact = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, row_offset=offset)
    for _ in range(2):  # two calls in a row share (and must clear) the same scratch
        Y = torch.full((m, d), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.cg_apply_csr_noalloc(plan._h, P(rp.data_ptr()), P(ci.data_ptr()), P(v.data_ptr()), ci.numel(),
                                      P(Y.data_ptr()), _stream())
        assert st == 0, _lib.STATUS_NAMES.get(st, st)
        torch.cuda.synchronize()
        got = Y.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel(got, want) < FP32_TOL
        assert rel(got, exact) < FP32_TOL


def test_noalloc_rejects_plans_beyond_its_scratch():
    from paper_1606_05732_gb300 import _lib, countgauss
    lib = _lib.load()
    # B.d.4 bytes = 32 MiB of SX alone, more than the 16 MiB array
    plan = countgauss.CountGauss(100, 64, 8, 1 << 17, 1)
    rp = torch.zeros(101, dtype=torch.int32, device="cuda")
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    ev = torch.zeros(1, dtype=torch.float32, device="cuda")
    Y = torch.zeros(8, 64, dtype=torch.float32, device="cuda")
    st = lib.cg_apply_csr_noalloc(plan._h, P(rp.data_ptr()), P(e.data_ptr()), P(ev.data_ptr()), 0,
                                  P(Y.data_ptr()), _stream())
    assert st == 3  # CG_ERR_WORKSPACE

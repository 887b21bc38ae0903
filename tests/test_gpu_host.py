"""cg_apply_csr_host: the transform of a CSR matrix held in host memory, copied to the
device in chunks of rows on a second stream while earlier chunks are scattered.
Results against the FP64 oracle at chunk sizes that cut the matrix into many chunks
(rows split mid-matrix, ragged last chunk, empty rows at the cuts), plus the errors
the host detects before anything is enqueued."""
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


def host_csr(X, pin=True):
    t = (torch.from_numpy(X.row_ptr.astype(np.int32)), torch.from_numpy(X.col_idx.astype(np.int32)),
         torch.from_numpy(X.vals.astype(np.float32)))
    return tuple(x.pin_memory() for x in t) if pin else t


CASES = [
    # n, d, m, B, seed, generator, chunk (0: automatic)
    (65536, 16, 8, 4096, 1, "bern", 0),
    (65536, 16, 8, 4096, 1, "bern", 5000),     # 11 chunks by nonzeros
    (4099, 37, 13, 1000, 7, "ragged", 32),     # ~100 chunks by rows, empty rows
    (4099, 37, 13, 1000, 7, "ragged", 777),
    (777, 128, 128, 4096, 3, "bern", 64),       # d > 64, m = 128
    (300, 1, 5, 7, 12, "ragged", 40),           # d = 1
    (1, 1, 1, 1, 11, "ragged", 32),             # scalar
]


def make(n, d, seed, kind):
    if kind == "ragged":
        return synth.csr_ragged(n, d, seed=seed, max_row=min(d, 32))
    return synth.csr_bernoulli(n, d, 0.05, seed=seed)


@pytest.mark.parametrize("n,d,m,B,seed,kind,chunk", CASES)
def test_host_apply_matches_oracle(n, d, m, B, seed, kind, chunk):
    X = make(n, d, seed, kind)
    plan = cg().CountGauss(n, d, m, B, seed)
    plan.set_host_chunk(chunk)
    Y = plan.apply_csr_host(*host_csr(X)).numpy()
    plan.check()
    Yo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals)
    assert rel(Y, Yo) < FP32_TOL


@pytest.mark.parametrize("n,d,m,B,seed,kind,chunk", CASES[::2])
@pytest.mark.parametrize("mode", ["direct", "copied"])
def test_host_read_modes_match_oracle(n, d, m, B, seed, kind, chunk, mode):
    """Direct reads (the scatter streams the pinned host arrays in place) and chunked
    copies give the oracle's result."""
    X = make(n, d, seed, kind)
    plan = cg().CountGauss(n, d, m, B, seed)
    plan.set_host_read(mode)
    plan.set_host_chunk(chunk)
    Y = plan.apply_csr_host(*host_csr(X)).numpy()
    plan.check()
    assert rel(Y, oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals)) < FP32_TOL


def test_host_direct_read_fallbacks_and_errors():
    """Direct reads asked for pageable arrays fall back to copies; a sub-range of a
    pinned buffer is read in place; malformed offsets are still caught (at the ends on
    the host, inside on the device)."""
    from paper_1606_05732_gb300 import _lib
    n, d, m, B, seed = 30000, 32, 16, 1024, 9
    X = synth.csr_bernoulli(n, d, 0.05, seed=seed)
    want = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals)
    plan = cg().CountGauss(n, d, m, B, seed)
    plan.set_host_read("direct")
    assert rel(plan.apply_csr_host(*host_csr(X, pin=False)).numpy(), want) < FP32_TOL
    rp, ci, v = host_csr(X)
    big = torch.zeros(X.nnz + 64, dtype=torch.float32).pin_memory()
    big[64:] = v
    assert rel(plan.apply_csr_host(rp, ci, big[64:]).numpy(), want) < FP32_TOL
    plan.check()
    bad = rp.clone()
    bad[-1] = X.nnz + 5
    with pytest.raises(_lib.CountGaussError) as e:
        plan.apply_csr_host(bad.pin_memory(), ci, v)
    assert e.value.status == _code("CG_ERR_INVALID_ARG")
    bad = rp.clone()
    bad[500], bad[501] = rp[501].item(), rp[500].item()
    plan.apply_csr_host(bad.pin_memory(), ci, v)
    with pytest.raises(_lib.CountGaussError) as e:
        plan.check()
    assert e.value.status == _code("CG_ERR_DEVICE_BOUNDS")
    plan.check()


def test_host_apply_repeats_and_matches_device_path():
    """Two calls in a row (the staging buffers reused), pageable inputs as well, and
    the device-input path: all within fp32 reduction-order rounding of each other."""
    n, d, m, B, seed = 20000, 64, 32, 2048, 5
    X = synth.csr_bernoulli(n, d, 0.05, seed=seed, values="uniform")
    plan = cg().CountGauss(n, d, m, B, seed)
    plan.set_host_chunk(3000)
    Y1 = plan.apply_csr_host(*host_csr(X)).clone()
    Y2 = plan.apply_csr_host(*host_csr(X, pin=False)).clone()
    dev = [t.cuda() for t in host_csr(X, pin=False)]
    Yd = plan.apply_csr(*dev).cpu()
    plan.check()
    assert rel(Y1, Yd) < 1e-6 and rel(Y2, Yd) < 1e-6


def _code(name):
    from paper_1606_05732_gb300 import _lib
    return next(k for k, v in _lib.STATUS_NAMES.items() if v == name)


def test_host_apply_errors():
    from paper_1606_05732_gb300 import _lib
    n, d, m, B, seed = 1000, 8, 4, 64, 2
    X = synth.csr_bernoulli(n, d, 0.5, seed=seed)
    rp, ci, v = host_csr(X)
    # a row longer than the chunk: unsupported when copied in chunks, fine when read in place
    Xl = synth.csr_ragged(100, 64, seed=3, max_row=64)  # has a full 64-entry row
    long_rows = cg().CountGauss(100, 64, m, B, seed)
    long_rows.set_host_chunk(32)
    long_rows.set_host_read("copied")
    with pytest.raises(_lib.CountGaussError) as e:
        long_rows.apply_csr_host(*host_csr(Xl))
    assert e.value.status == _code("CG_ERR_UNSUPPORTED")
    long_rows.set_host_read("direct")
    Yl = long_rows.apply_csr_host(*host_csr(Xl)).numpy()
    long_rows.check()
    assert rel(Yl, oracle.apply_csr(seed, 100, 64, m, B, Xl.row_ptr, Xl.col_idx, Xl.vals)) < FP32_TOL
    # deterministic plans are not supported
    det = cg().CountGauss(n, d, m, B, seed, deterministic=True)
    with pytest.raises(_lib.CountGaussError) as e:
        det.apply_csr_host(rp, ci, v)
    assert e.value.status == _code("CG_ERR_UNSUPPORTED")
    # row offsets outside [0, nnz] at a chunk boundary: rejected on the host
    plan = cg().CountGauss(n, d, m, B, seed)
    bad = rp.clone()
    bad[-1] = X.nnz + 5
    with pytest.raises(_lib.CountGaussError) as e:
        plan.apply_csr_host(bad, ci, v)
    assert e.value.status == _code("CG_ERR_INVALID_ARG")
    # offsets in range but out of order inside a chunk: skipped and reported by the device
    bad = rp.clone()
    bad[500], bad[501] = rp[501].item(), rp[500].item()
    plan.apply_csr_host(bad, ci, v)
    with pytest.raises(_lib.CountGaussError) as e:
        plan.check()
    assert e.value.status == _code("CG_ERR_DEVICE_BOUNDS")
    plan.check()  # the status word was cleared

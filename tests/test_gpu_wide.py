"""cg_apply_csr_i64 and cg_apply_adjoint_i64: the transform Y = G.(S.X) (Section 1.1;
Algorithm 1 steps 1-2) and its adjoint at the stored entries, for CSR matrices given with
64-bit row offsets, i.e. of 2^31 nonzeros or more.

Parity with the FP64 oracle at sizes it finishes in seconds (several chunks of rows and
a ragged tail, every chunk height), for the one-pass and the deferred scatter; past 2^31
nonzeros (2.3e9 and 2.4e9), agreement with the 32-bit path applied to row blocks with
their global row offsets, which is the same transform by linearity (h and sigma depend
on the global row index only), and sampled rows of SX against their definition.  Malformed
offsets are reported through the status word and skipped.  Bar: relative Frobenius
error 1e-5 (FP32); the adjoint's values are the same arithmetic as the 32-bit path's, so
the two agree bit for bit.
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


def dev_csr64(X):
    return (torch.from_numpy(X.row_ptr.astype(np.int64)).cuda(),
            torch.from_numpy(X.col_idx.astype(np.int32)).cuda(),
            torch.from_numpy(X.vals.astype(np.float32)).cuda())


@pytest.mark.parametrize("rows", [0, 1, 32, 64, 128])
@pytest.mark.parametrize("n,d,m,B,seed,per_row", [(70001, 37, 13, 3001, 31, 6), (4099, 64, 32, 512, 32, 64),
                                                  (100_000, 16, 8, 4096, 33, 1)])
def test_parity_with_oracle(n, d, m, B, seed, per_row, rows):
    """Ragged rows (empty ones, full ones), every chunk height, a row offset."""
    X = synth.csr_ragged(n, d, seed=seed, max_row=per_row)
    plan = cg().CountGauss(n, d, m, B, seed, scatter_rows=rows, row_offset=777)
    Y = plan.apply_csr(*dev_csr64(X)).cpu().numpy()
    plan.check()
    Yo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, row_offset=777)
    assert rel(Y, Yo) < FP32_TOL


@pytest.mark.parametrize("passes", [2, 5])
def test_bucket_range_passes(passes):
    n, d, m, B, seed = 50_000, 24, 16, 2048, 34
    X = synth.csr_bernoulli(n, d, 0.1, seed)
    plan = cg().CountGauss(n, d, m, B, seed, scatter_passes=passes)
    Y = plan.apply_csr(*dev_csr64(X)).cpu().numpy()
    plan.check()
    assert rel(Y, oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals)) < FP32_TOL


def test_empty_matrix_and_empty_rows():
    n, d, m, B, seed = 1000, 8, 4, 64, 35
    plan = cg().CountGauss(n, d, m, B, seed)
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    v = torch.zeros(0, dtype=torch.float32, device="cuda")
    Y = plan.apply_csr(rp, ci, v)
    plan.check()
    assert float(Y.abs().max()) == 0.0


def test_same_as_32_bit_offsets():
    """The two entry points compute the same transform (up to FP32 summation order)."""
    X, w = synth.workload_csr("nmf_n16M_d64", scale_rows=1 / 64)
    rp64, ci, v = dev_csr64(X)
    plan = cg().CountGauss(X.n, X.d, w["m"], w["B"], w["seed"])
    Y64 = plan.apply_csr(rp64, ci, v).cpu().numpy()
    Y32 = plan.apply_csr(rp64.int(), ci, v).cpu().numpy()
    plan.check()
    assert rel(Y64, Y32) < FP32_TOL


@pytest.mark.parametrize("rows", [0, 32, 64, 128, 256])
@pytest.mark.parametrize("n,d,m,B,seed,per_row", [(70001, 37, 13, 3001, 51, 6), (4099, 64, 32, 512, 52, 64),
                                                  (100_000, 16, 8, 4096, 53, 1)])
def test_deferred_parity_with_oracle(n, d, m, B, seed, per_row, rows):
    """The deferred scatter (CG_OPT_SCATTER = 3) with int64 offsets: ragged rows (empty
    ones, full ones), every chunk height, a row offset; Y and SX against the oracle, and SX
    accumulated over two row blocks (each with its global row offset) equal to the whole."""
    X = synth.csr_ragged(n, d, seed=seed, max_row=per_row)
    rp, ci, v = dev_csr64(X)
    plan = cg().CountGauss(n, d, m, B, seed, scatter="deferred", scatter_rows=rows, row_offset=777)
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, row_offset=777, return_sx=True)
    assert rel(Y, Yo) < FP32_TOL
    SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
    plan.check()
    assert rel(SX, SXo) < FP32_TOL
    cut = n // 3
    k0 = int(X.row_ptr[cut])
    a = cg().CountGauss(cut, d, m, B, seed, scatter="deferred", scatter_rows=rows, row_offset=777)
    b = cg().CountGauss(n - cut, d, m, B, seed, scatter="deferred", scatter_rows=rows, row_offset=777 + cut)
    SXa = a.sketch_csr(rp[:cut + 1].contiguous(), ci[:k0], v[:k0])
    b.sketch_csr((rp[cut:] - k0).contiguous(), ci[k0:], v[k0:], out=SXa, accumulate=True)
    a.check()
    b.check()
    assert rel(SXa.cpu().numpy(), SXo) < FP32_TOL


@pytest.mark.parametrize("scatter,rows", [("auto", 1), ("auto", 32), ("auto", 128), ("deferred", 0),
                                          ("deferred", 32), ("deferred", 256)])
def test_malformed_offsets_are_reported(scatter, rows):
    from paper_1606_05732_gb300 import _lib
    n, d, m, B, seed = 20_000, 16, 8, 1024, 36
    X = synth.csr_ragged(n, d, seed=7, max_row=4)
    rp, ci, v = dev_csr64(X)
    plan = cg().CountGauss(n, d, m, B, seed, scatter=scatter, scatter_rows=rows)
    bad = rp.clone()
    bad[n // 2], bad[n // 2 + 1] = rp[n // 2 + 1].item() + 1, rp[n // 2].item()  # decreasing
    plan.apply_csr(bad, ci, v)
    with pytest.raises(_lib.CountGaussError):
        plan.check()
    bad = rp.clone()
    bad[n] = X.nnz + 5  # past nnz
    plan.apply_csr(bad, ci, v)
    with pytest.raises(_lib.CountGaussError):
        plan.check()
    bad = rp.clone()
    bad[7] = -(1 << 40)  # far below the first nonzero
    plan.apply_csr(bad, ci, v)
    with pytest.raises(_lib.CountGaussError):
        plan.check()
    plan.apply_csr(rp, ci, v)
    plan.check()


def test_past_2_pow_31_nonzeros_matches_row_blocks():
    """2^25 rows x 64 columns with 72 nonzeros per row on average: about 2.4e9 nonzeros
    (19 GB of CSR), past what 32-bit offsets hold.  Equals the sum of the 32-bit path
    over two row blocks, each with its global row offset."""
    n, d, m, B, seed = 1 << 25, 64, 32, 1 << 17, 37
    rp, ci, v = synth.wide_csr_device(n, d, 72, seed)
    nnz = ci.numel()
    assert nnz > (1 << 31)
    plan = cg().CountGauss(n, d, m, B, seed)
    Y = plan.apply_csr(rp, ci, v)
    plan.check()
    Yb = torch.zeros_like(Y)
    cut = n // 2
    for r0, r1 in ((0, cut), (cut, n)):
        k0, k1 = int(rp[r0].item()), int(rp[r1].item())
        assert k1 - k0 < (1 << 31) - (1 << 20)
        part = cg().CountGauss(r1 - r0, d, m, B, seed, row_offset=r0)
        Yb += part.apply_csr((rp[r0:r1 + 1] - k0).int(), ci[k0:k1], v[k0:k1])
        part.check()
    assert rel(Y.cpu().numpy(), Yb.cpu().numpy()) < FP32_TOL


def test_deferred_past_2_pow_31_nonzeros_matches_row_blocks_and_oracle():
    """2^24 rows x 128 columns with 136 nonzeros per row on average (about 2.3e9 nonzeros,
    18 GB of CSR) into an SX of 2^18 x 128 (128 MB, past the L2): the automatic choice is
    the deferred scatter with int64 offsets (its workspace holds 8 bytes per nonzero).  Y
    equals the sum of the 32-bit path over two row blocks; SX at 64 sampled buckets, half
    of them in the top quarter (rows the replay pass reduces), equals the definition
    (sum of sigma(i) X[i, :] over the rows with h(i) = b, h and sigma from the oracle) in
    FP64."""
    from paper_1606_05732_gb300 import _lib
    n, d, m, B, seed = 1 << 24, 128, 32, 1 << 18, 38
    rp, ci, v = synth.wide_csr_device(n, d, 136, seed)
    nnz = ci.numel()
    assert nnz > (1 << 31)
    plan = cg().CountGauss(n, d, m, B, seed)
    assert plan.workspace_size(_lib.OP_APPLY_CSR_I64, nnz) >= 8 * nnz
    Y = plan.apply_csr(rp, ci, v)
    plan.check()
    Yb = torch.zeros_like(Y)
    cut = n // 2
    for r0, r1 in ((0, cut), (cut, n)):
        k0, k1 = int(rp[r0].item()), int(rp[r1].item())
        part = cg().CountGauss(r1 - r0, d, m, B, seed, row_offset=r0)
        Yb += part.apply_csr((rp[r0:r1 + 1] - k0).int(), ci[k0:k1], v[k0:k1])
        part.check()
        del part
    assert rel(Y.cpu().numpy(), Yb.cpu().numpy()) < FP32_TOL

    SX = plan.sketch_csr(rp, ci, v)
    plan.check()
    rng = np.random.default_rng(seed)
    sample = np.concatenate([rng.choice(B // 2, 32, replace=False),
                             3 * B // 4 + rng.choice(B // 4, 32, replace=False)]).astype(np.int64)
    h, sg = oracle.hash_sign(seed, B, 0, n)
    rows = np.nonzero(np.isin(h, sample))[0]
    rows_d = torch.from_numpy(rows).cuda()
    starts = rp[rows_d]
    lens = rp[rows_d + 1] - starts
    total = int(lens.sum().item())
    first = torch.cumsum(lens, 0) - lens
    idx = torch.arange(total, device="cuda") - torch.repeat_interleave(first - starts, lens)
    cols = ci[idx].cpu().numpy().astype(np.int64)
    xs = v[idx].cpu().numpy().astype(np.float64)
    owner = np.repeat(rows, lens.cpu().numpy())
    sample = np.sort(sample)
    E = np.zeros((sample.size, d), np.float64)
    np.add.at(E, (np.searchsorted(sample, h[owner]), cols), sg[owner] * xs)
    assert np.count_nonzero(E) > 0
    assert rel(SX[torch.from_numpy(sample).cuda()].cpu().numpy(), E) < FP32_TOL
    del plan, SX, Y, Yb, rp, ci, v
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,d,m,B,seed,per_row", [(70001, 37, 13, 3001, 41, 6), (4099, 64, 32, 512, 42, 64)])
def test_adjoint_parity_with_oracle(n, d, m, B, seed, per_row):
    X = synth.csr_ragged(n, d, seed=seed, max_row=per_row)
    rp, ci, _ = dev_csr64(X)
    dYn = np.random.default_rng(seed).standard_normal((m, d)).astype(np.float32)
    dY = torch.from_numpy(dYn).cuda()
    plan = cg().CountGauss(n, d, m, B, seed, row_offset=99)
    dXv = plan.adjoint(dY, rp, ci)
    plan.check()
    assert rel(dXv.cpu().numpy(), oracle.adjoint_csr(seed, n, m, B, X.row_ptr, X.col_idx, dYn, row_offset=99)) \
        < FP32_TOL
    assert torch.equal(dXv, plan.adjoint(dY, rp.int(), ci))  # same W, same products


def test_autograd_with_wide_offsets():
    """The CSR autograd function takes int64 offsets in both directions."""
    n, d, m, B, seed = 30_000, 16, 8, 1024, 43
    X = synth.csr_bernoulli(n, d, 0.05, seed)
    rp, ci, v = dev_csr64(X)
    plan = cg().CountGauss(n, d, m, B, seed)
    grads = []
    for offsets in (rp, rp.int()):
        vals = v.clone().requires_grad_(True)
        Y = cg().countgauss_csr(vals, offsets, ci, plan)
        (Y * Y).sum().backward()
        grads.append(vals.grad)
    plan.check()
    assert rel(grads[0].cpu().numpy(), grads[1].cpu().numpy()) < FP32_TOL


def test_adjoint_malformed_offsets_are_reported():
    from paper_1606_05732_gb300 import _lib
    n, d, m, B, seed = 5000, 8, 4, 256, 44
    X = synth.csr_ragged(n, d, seed=9, max_row=4)
    rp, ci, _ = dev_csr64(X)
    dY = torch.ones(m, d, device="cuda")
    plan = cg().CountGauss(n, d, m, B, seed)
    bad = rp.clone()
    bad[n] = X.nnz + 1
    plan.adjoint(dY, bad, ci)
    with pytest.raises(_lib.CountGaussError):
        plan.check()
    plan.adjoint(dY, rp, ci)
    plan.check()


def test_adjoint_past_2_pow_31_nonzeros_matches_row_blocks():
    """The gradient at 2.4e9 stored entries equals, bit for bit, the 32-bit path's on two
    row blocks with their global row offsets."""
    n, d, m, B, seed = 1 << 25, 64, 32, 1 << 17, 45
    rp, ci, v = synth.wide_csr_device(n, d, 72, seed)
    del v
    assert ci.numel() > (1 << 31)
    dY = torch.randn(m, d, device="cuda", generator=torch.Generator(device="cuda").manual_seed(seed))
    plan = cg().CountGauss(n, d, m, B, seed)
    dXv = plan.adjoint(dY, rp, ci)
    plan.check()
    cut = n // 2
    for r0, r1 in ((0, cut), (cut, n)):
        k0, k1 = int(rp[r0].item()), int(rp[r1].item())
        part = cg().CountGauss(r1 - r0, d, m, B, seed, row_offset=r0)
        blk = part.adjoint(dY, (rp[r0:r1 + 1] - k0).int(), ci[k0:k1])
        part.check()
        assert torch.equal(dXv[k0:k1], blk)
        del blk


def test_sketch_alone_and_streamed_in_row_chunks():
    """cg_sketch_csr_i64: SX = S.X equals the oracle's; fed as row chunks (each chunk's
    offsets from 0, its global row offset set, accumulating) it gives the same SX."""
    n, d, B, seed = 90_001, 24, 4096, 46
    X = synth.csr_ragged(n, d, seed=seed, max_row=8)
    rp, ci, v = dev_csr64(X)
    SXo = oracle.sketch_csr(seed, n, d, B, X.row_ptr, X.col_idx, X.vals)
    plan = cg().CountGauss(n, d, 4, B, seed)
    SX = plan.sketch_csr(rp, ci, v)
    plan.check()
    assert rel(SX.cpu().numpy(), SXo) < 1e-6
    cuts = [0, 1, 30_000, 30_001, 77_777, n]
    acc = torch.full((B, d), float("nan"), device="cuda")
    for c, (r0, r1) in enumerate(zip(cuts[:-1], cuts[1:])):
        k0, k1 = int(X.row_ptr[r0]), int(X.row_ptr[r1])
        part = cg().CountGauss(r1 - r0, d, 4, B, seed, row_offset=r0)
        part.sketch_csr(rp[r0:r1 + 1] - k0, ci[k0:k1], v[k0:k1], out=acc, accumulate=c > 0)
        part.check()
    assert rel(acc.cpu().numpy(), SXo) < 1e-6


def test_nmf_anchors_with_wide_offsets():
    """Algorithm 1 steps 1-3 with int64 offsets: Z as with int32 offsets, and imax / imin
    the columns of each row's max / min of that Z, lowest index on ties."""
    n, d, m, B, seed = 40_000, 50, 16, 2048, 47
    X = synth.csr_bernoulli(n, d, 0.05, seed, values="uniform")
    rp, ci, v = dev_csr64(X)
    plan = cg().CountGauss(n, d, m, B, seed)
    Z, imax, imin = plan.nmf_anchors(rp, ci, v)
    Z32, _, _ = plan.nmf_anchors(rp.int(), ci, v)
    plan.check()
    assert rel(Z.cpu().numpy(), Z32.cpu().numpy()) < FP32_TOL
    Zc = Z.cpu()
    assert torch.equal(imax.cpu().long(), torch.argmax(Zc, dim=1))
    assert torch.equal(imin.cpu().long(), torch.argmin(Zc, dim=1))

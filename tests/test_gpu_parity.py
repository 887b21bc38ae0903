"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: bucket, sign and Philox words bit-exact; floating results within a relative
Frobenius error of 1e-5 for the FP32 path.  Inputs are seeded and synthetic
(paper_1606_05732_gb300.synth); expected values come from the oracle only.
"""
import math

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


def dev_csr(X):
    return (torch.from_numpy(X.row_ptr.astype(np.int32)).cuda(),
            torch.from_numpy(X.col_idx.astype(np.int32)).cuda(),
            torch.from_numpy(X.vals.astype(np.float32)).cuda())


# -----------------------------------------------------------------------------
# Generator: bit-exact words, buckets and signs; Gaussians to fp32 rounding.
# -----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 3, 2**32 + 7, 2**64 - 1])
@pytest.mark.parametrize("tag", [0, 1, 2])
def test_words_bit_exact(seed, tag):
    for idx0 in [0, 2**32 - 100, 2**40 + 3]:
        got = cg().generate_words(seed, tag, idx0, 1000).cpu().numpy().view(np.uint32)
        want = oracle.philox_words(seed, tag, idx0, 1000)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("B", [1, 3, 4096, 100003, 1 << 17, 1 << 18, (1 << 31) - 1])
def test_hash_sign_bit_exact(B):
    for seed, row0 in [(1, 0), (2, 12345), (2**63 + 5, 2**33)]:
        h, s = cg().generate_hash_sign(seed, B, row0, 5000)
        wh, ws = oracle.hash_sign(seed, B, row0, 5000)
        np.testing.assert_array_equal(h.cpu().numpy(), wh)
        np.testing.assert_array_equal(s.cpu().numpy(), ws)


def test_gaussian_entries_many():
    """8.4 M entries (2^21 Philox calls, so 2^22 uniforms of each role: radius and
    angle) against the FP64 Box-Muller of the same words.  Per entry the fp32 result
    carries a few ulp of relative error in the radius sqrt(-2 ln u) and a few 1e-8 of
    absolute error in cos / sin of 2 pi u, so |z - z64| <= 1e-6 (1 + |z64|); over all
    entries the relative Frobenius error is below 2e-7."""
    R, C = 8, 1 << 20
    got = cg().generate_gaussian(77, 1, R, 0, R, 0, C).cpu().numpy().astype(np.float64)
    want = oracle.gaussian_block(77, 1, R, 0, R, 0, C)
    err = np.abs(got - want)
    print(f"max |dz| = {err.max():.3e}, max |dz|/(1+|z|) = {(err / (1 + np.abs(want))).max():.3e}, "
          f"rel Frobenius {rel(got, want):.3e}")
    assert (err <= 1e-6 * (1.0 + np.abs(want))).all()
    assert rel(got, want) < 2e-7


@pytest.mark.parametrize("tag,R", [(1, 8), (1, 13), (2, 128), (1, 1)])
def test_gaussian_entries(tag, R):
    got = cg().generate_gaussian(5, tag, R, 0, R, 1000, 1700).cpu().numpy()
    want = oracle.gaussian_block(5, tag, R, 0, R, 1000, 1700)
    # fp32 Box-Muller (logf, sqrtf, sincospif) against fp64: a few ulp of fp32
    assert np.abs(got - want).max() < 4e-6 * max(1.0, np.abs(want).max())
    assert rel(got, want) < 1e-6


# -----------------------------------------------------------------------------
# The transform, the plain product and the stages on shapes that span several
# tiles and have ragged tails.
# -----------------------------------------------------------------------------
CASES = [
    # n, d, m, B, seed, generator
    (65536, 16, 8, 4096, 1, "bern0.05"),     # the small workload, full size
    (5000, 64, 32, 2048, 2, "bern0.05u"),    # several tiles
    (4099, 37, 13, 1000, 7, "ragged"),        # nothing a multiple of anything
    (777, 128, 128, 4096, 3, "bern0.02"),    # d > 64 path, m = 128
    (1, 1, 1, 1, 11, "ragged"),               # scalar
    (300, 1, 5, 7, 12, "ragged"),              # d = 1
    (2000, 5, 1, 64, 13, "ragged"),            # m = 1
    (1000, 8, 70, 33, 14, "bern0.3"),          # m > 64, two row blocks
    (100, 4, 4, 1, 15, "bern0.3"),             # B = 1
    (64, 200, 9, 50, 16, "ragged"),            # d > 128, two column blocks
]


def make_input(n, d, seed, kind):
    if kind == "ragged":
        return synth.csr_ragged(n, d, seed=seed)
    p = float(kind[4:].rstrip("u"))
    return synth.csr_bernoulli(n, d, p, seed=seed, values="uniform" if kind.endswith("u") else "normal")


@pytest.mark.parametrize("scatter", ["atomic", "partition", "deferred", "binned"])
@pytest.mark.parametrize("n,d,m,B,seed,kind", CASES)
def test_apply_csr_parity(n, d, m, B, seed, kind, scatter):
    X = make_input(n, d, seed, kind)
    plan = cg().CountGauss(n, d, m, B, seed, scatter=scatter)
    rp, ci, v = dev_csr(X)
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
    plan.check()
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, return_sx=True)
    assert rel(SX, SXo) < 1e-6
    assert rel(Y, Yo) < FP32_TOL, rel(Y, Yo)


@pytest.mark.parametrize("n,d,m,B,seed,kind", CASES[:4] + [(256, 4096, 8, 512, 9, "bern1.0")])
def test_deterministic_mode_is_bit_reproducible_and_exact(n, d, m, B, seed, kind):
    """Deterministic mode sums fixed-point integers (resolution 2^(L+e-62) with
    2^e > max|x|, 2^L > nnz) and rounds once to fp32: repeated runs are bit-identical,
    and every SX entry is within one fp32 ulp plus the fixed-point resolution per term
    of the oracle's FP64 sum; almost all entries equal its fp32 rounding exactly."""
    X = make_input(n, d, seed, kind)
    rp, ci, v = dev_csr(X)
    plan = cg().CountGauss(n, d, m, B, seed, deterministic=True)
    SX1 = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y1 = plan.apply_csr(rp, ci, v).cpu().numpy()
    SX2 = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y2 = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    np.testing.assert_array_equal(SX1, SX2)
    np.testing.assert_array_equal(Y1, Y2)
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, return_sx=True)
    want = SXo.astype(np.float32)
    L = max(1, int(X.nnz).bit_length())
    e = int(np.frexp(np.abs(X.vals).max())[1]) if X.nnz else 0
    per_term = 2.0 ** (L + e - 62)
    rows_per_bucket = np.bincount(oracle.hash_sign(seed, B, 0, n)[0], minlength=B)
    bound = np.spacing(np.abs(want)).astype(np.float64) + (rows_per_bucket[:, None] + 1) * per_term
    assert (np.abs(SX1.astype(np.float64) - SXo) <= bound).all()
    assert (SX1 == want).mean() > 0.99
    assert rel(Y1, Yo) < FP32_TOL


def _nan_inf_equal(got, want):
    """Same NaN positions, same infinities (with sign), finite entries within 1e-6."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(want))
    np.testing.assert_array_equal(np.isposinf(got), np.isposinf(want))
    np.testing.assert_array_equal(np.isneginf(got), np.isneginf(want))
    fin = np.isfinite(want)
    assert rel(got[fin], want[fin]) < 1e-6


@pytest.mark.parametrize("mode", ["atomic", "deferred", "binned", "partition", "deterministic",
                                  "deterministic_binned"])
def test_nonfinite_values_propagate_as_ieee_addition(mode):
    """The rule for NaN and infinite entries of X, the same in every scatter: the SX cell
    they land in is NaN if it receives a NaN or both +Inf and -Inf, else the infinity it
    receives (IEEE addition, as the FP64 oracle computes it); every other cell is unchanged.
    The deterministic mode keeps its bit-reproducible result."""
    n, d, m, B, seed = 20000, 16, 8, 512, 5
    Xd = synth.csr_bernoulli(n, d, 0.05, seed=6).to_dense()
    h, sg = oracle.hash_sign(seed, B, 0, n)
    # two rows sharing a bucket: +Inf from one and -Inf from the other into one cell
    first = {}
    pair = None
    for i in range(n):
        if h[i] in first:
            pair = (first[h[i]], i)
            break
        first[h[i]] = i
    i1, i2 = pair
    Xd[i1, 3] = np.inf * sg[i1]
    Xd[i2, 3] = -np.inf * sg[i2]
    Xd[777, 5] = np.nan
    Xd[1234, 0] = np.inf
    Xd[1234, 1] = -np.inf
    X = synth.csr_from_dense(Xd)
    rp, ci, v = dev_csr(X)
    kw = ({"deterministic": True} if mode == "deterministic" else
          {"deterministic": True, "scatter": "binned"} if mode == "deterministic_binned" else {"scatter": mode})
    plan = cg().CountGauss(n, d, m, B, seed, **kw)
    SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, return_sx=True)
    assert np.isnan(SXo[h[i1], 3]) and np.isnan(SXo).sum() == 2 and np.isinf(SXo).sum() == 2
    _nan_inf_equal(SX, SXo)
    _nan_inf_equal(Y, Yo)
    if mode.startswith("deterministic"):
        np.testing.assert_array_equal(plan.sketch_csr(rp, ci, v).cpu().numpy(), SX)


def test_deterministic_scale_sees_every_value_at_any_alignment():
    """The fixed-point scale comes from max |x| over all stored values; the largest value
    placed first, second, third, second-last or last, with the values starting at each
    of the four 4-byte offsets within 16 bytes, gives the same bits (a missed maximum
    would overflow the fixed-point sums) and the oracle's SX."""
    n, d, m, B, seed = 5000, 16, 8, 256, 21
    X = synth.csr_bernoulli(n, d, 0.1, seed=seed)
    rp, ci, _ = dev_csr(X)
    plan = cg().CountGauss(n, d, m, B, seed, deterministic=True)
    for pos in (0, 1, 2, X.nnz - 2, X.nnz - 1):
        vals = X.vals.copy()
        vals[pos] = 3.0e5
        ref = None
        for off in range(4):
            buf = torch.zeros(X.nnz + 4, dtype=torch.float32, device="cuda")
            buf[off:off + X.nnz] = torch.from_numpy(vals).cuda()
            SX = plan.sketch_csr(rp, ci, buf[off:off + X.nnz]).cpu().numpy()
            if ref is None:
                ref = SX
            else:
                np.testing.assert_array_equal(SX, ref)
        plan.check()
        SXo = oracle.sketch_csr(seed, n, d, B, X.row_ptr, X.col_idx, vals)
        assert rel(ref, SXo) < 1e-6


@pytest.mark.parametrize("rows", [1, 32, 64, 128])
@pytest.mark.parametrize("passes", [1, 3])
@pytest.mark.parametrize("n,d,m,B,seed,kind", [CASES[2], CASES[3], CASES[5], (70001, 128, 16, 5000, 17, "bern0.01")])
def test_scatter_chunk_rows_and_passes(n, d, m, B, seed, kind, rows, passes):
    """Every chunk height and bucket-range pass count gives the oracle's SX: the
    chunk's last row, its ragged tail (n not a multiple of the height) and rows whose
    buckets fall in each range are all reduced exactly once."""
    X = make_input(n, d, seed, kind)
    rp, ci, v = dev_csr(X)
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, return_sx=True)
    plan = cg().CountGauss(n, d, m, B, seed, scatter="atomic", scatter_rows=rows, scatter_passes=passes)
    SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    assert rel(SX, SXo) < 1e-6
    assert rel(Y, Yo) < FP32_TOL
    det = cg().CountGauss(n, d, m, B, seed, deterministic=True, scatter_rows=rows)
    SXd = det.sketch_csr(rp, ci, v).cpu().numpy()
    det.check()
    assert rel(SXd, SXo) < 1e-6


@pytest.mark.parametrize("rows", [32, 64, 128, 256])
def test_deferred_scatter_edges(rows):
    """The deferred scatter (rows of the upper half of the buckets written as records,
    reduced by a second pass): CTA row ranges with ragged ends and empty rows, a row
    offset (shard), and the error report for a bad column index and for out-of-order
    offsets, which it skips like the one-pass scatter."""
    from paper_1606_05732_gb300 import _lib
    n, d, m, B, seed = 70001, 37, 13, 3001, 21
    X = synth.csr_ragged(n, d, seed=5, max_row=6)
    rp, ci, v = dev_csr(X)
    plan = cg().CountGauss(n, d, m, B, seed, scatter="deferred", scatter_rows=rows, row_offset=12345)
    SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, row_offset=12345, return_sx=True)
    assert rel(SX, SXo) < 1e-6
    assert rel(Y, Yo) < FP32_TOL
    bad_ci = ci.clone()
    bad_ci[X.nnz // 2] = d + 3
    plan.sketch_csr(rp, bad_ci, v)
    with pytest.raises(_lib.CountGaussError):
        plan.check()
    bad_rp = rp.clone()
    bad_rp[n // 2], bad_rp[n // 2 + 1] = rp[n // 2 + 1].item() + 1, rp[n // 2].item()
    plan.sketch_csr(bad_rp, ci, v)
    with pytest.raises(_lib.CountGaussError):
        plan.check()
    plan.check()


def _banded_csr(n, d, seed):
    """Rows whose lengths grow along the matrix: the first third 0-2 nonzeros, the middle
    third 1-3, the last third 4-6, so that 256-row chunks hold under 384 nonzeros (staged
    in shared memory), 384 to 1024 (row map, global loads) and over 1024 (binary search)."""
    rng = np.random.default_rng(seed)
    third = n // 3
    lens = np.concatenate([rng.integers(0, 3, third), rng.integers(1, 4, third), rng.integers(4, 7, n - 2 * third)])
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1:] = np.cumsum(lens)
    col_idx = np.concatenate([np.sort(rng.choice(d, k, replace=False)) for k in lens]).astype(np.int32)
    vals = rng.standard_normal(int(row_ptr[-1])).astype(np.float32)
    return synth.CSR(n, d, row_ptr, col_idx, vals)


@pytest.mark.parametrize("ctas", [0, 7])
def test_deferred_staged_pass_paths(ctas):
    """Pass 1 of the deferred scatter stages a chunk's nonzeros in shared memory by bulk
    copies when they fit, and reads them from global memory otherwise (row map or binary
    search): all three kinds of chunk in one matrix, with 16-byte misaligned starts and
    ragged tails; with 7 CTAs each warp takes many chunks in turn (the mbarrier's phases);
    col_idx and vals that are not 16-byte aligned take the plain pass."""
    n, d, m, B, seed = 60001, 37, 13, 3001, 23
    X = _banded_csr(n, d, 3)
    rp, ci, v = dev_csr(X)
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, row_offset=4097, return_sx=True)
    plan = cg().CountGauss(n, d, m, B, seed, scatter="deferred", scatter_rows=256, row_offset=4097, sketch_ctas=ctas)
    SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    assert rel(SX, SXo) < 1e-6
    assert rel(Y, Yo) < FP32_TOL
    # the same arrays one element into larger buffers: 4-byte, not 16-byte, aligned
    ci_buf = torch.empty(X.nnz + 1, dtype=torch.int32, device=ci.device)
    v_buf = torch.empty(X.nnz + 1, dtype=torch.float32, device=v.device)
    ci_buf[1:].copy_(ci)
    v_buf[1:].copy_(v)
    SX2 = plan.sketch_csr(rp, ci_buf[1:], v_buf[1:]).cpu().numpy()
    plan.check()
    assert rel(SX2, SXo) < 1e-6


@pytest.mark.parametrize("n,d,B,kind", [(70001, 37, 3001, "ragged"),      # one tile per lane row, ragged ends
                                         (300_000, 128, 4096, "bern0.01"),  # the ladder's density, 16 slices
                                         (40_000, 64, 100_000, "bern0.05"),  # 196 slices, 3.2 nonzeros per row
                                         (5000, 1, 1 << 20, "bern0.3")])    # d = 1, 32 slices
def test_binned_scatter_edges(n, d, B, kind):
    """The binned scatter (records sorted by bucket slice, each slice summed in shared
    memory): many tiles per CTA with ragged ends, empty rows, a row offset (shard), and the
    error report for a bad column index and for out-of-order offsets, skipped like the
    one-pass scatter does."""
    from paper_1606_05732_gb300 import _lib
    m, seed = 13, 21
    X = make_input(n, d, 5, kind) if kind != "ragged" else synth.csr_ragged(n, d, seed=5, max_row=6)
    rp, ci, v = dev_csr(X)
    plan = cg().CountGauss(n, d, m, B, seed, scatter="binned", row_offset=12345)
    SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, row_offset=12345, return_sx=True)
    assert rel(SX, SXo) < 1e-6
    assert rel(Y, Yo) < FP32_TOL
    bad_ci = ci.clone()
    bad_ci[X.nnz // 2] = d + 3
    SXb = plan.sketch_csr(rp, bad_ci, v).cpu().numpy()
    with pytest.raises(_lib.CountGaussError):
        plan.check()
    # the bad entry is skipped: the rest of the sketch is unchanged
    k = X.nnz // 2
    i = int(np.searchsorted(X.row_ptr, k, side="right") - 1)
    h, s = oracle.hash_sign(seed, B, 12345 + i, 1)
    SXo2 = SXo.copy()
    SXo2[h[0], X.col_idx[k]] -= s[0] * X.vals[k]
    assert rel(SXb, SXo2) < 1e-6
    bad_rp = rp.clone()
    bad_rp[n // 2], bad_rp[n // 2 + 1] = rp[n // 2 + 1].item() + 1, rp[n // 2].item()
    plan.sketch_csr(bad_rp, ci, v)
    with pytest.raises(_lib.CountGaussError):
        plan.check()
    plan.check()


def test_binned_overflow_and_long_tiles():
    """Full rows of 4096 entries: a row's records all land in one slice (8 buckets of 4096
    columns), far past that slice's share of its CTA's region, so they spill to the overflow
    list; a tile of rows holds far more records than the shared staging buffer, so most go
    straight to the regions.  Neither may change the result."""
    n, d, m, B, seed = 256, 4096, 8, 512, 9
    X = synth.csr_bernoulli(n, d, 1.0, seed=3)
    rp, ci, v = dev_csr(X)
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, return_sx=True)
    plan = cg().CountGauss(n, d, m, B, seed, scatter="binned")
    SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    assert rel(SX, SXo) < 1e-6
    assert rel(Y, Yo) < FP32_TOL
    # one row holding a quarter of a sparse matrix's entries
    n, d, B = 20000, 512, 1 << 14
    Xs = synth.csr_bernoulli(n, d, 0.01, seed=4).to_dense()
    Xs[777, :] = np.random.default_rng(1).standard_normal(d).astype(np.float32)
    X = synth.csr_from_dense(Xs)
    rp, ci, v = dev_csr(X)
    plan = cg().CountGauss(n, d, m, B, seed, scatter="binned")
    SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
    plan.check()
    assert rel(SX, oracle.sketch_csr(seed, n, d, B, X.row_ptr, X.col_idx, X.vals)) < 1e-6


@pytest.mark.parametrize("n,d,B,seed,kind", [(70001, 37, 3001, 21, "ragged6"), (4099, 64, 512, 22, "ragged64"),
                                             (100_000, 16, 4096, 23, "ragged1"), (20000, 129, 1 << 13, 24, "bern"),
                                             (256, 4096, 512, 25, "full"), (20000, 512, 1 << 14, 26, "heavy_row")])
def test_deterministic_binned_slices_equal_global_accumulator(n, d, B, seed, kind):
    """The deterministic mode's two forms -- one int64 accumulator in global memory
    (CG_OPT_SCATTER = 1) and int64 sums per bucket slice in shared memory (= 4, automatic
    once the accumulator outgrows the L2) -- add the same fixed-point integers and round once,
    so they agree bit for bit, also where a slice's records spill to the overflow list (full
    rows of 4096 entries; one row holding a quarter of the entries), and with the oracle."""
    if kind.startswith("ragged"):
        X = synth.csr_ragged(n, d, seed=seed, max_row=int(kind[6:]))
    elif kind == "bern":
        X = synth.csr_bernoulli(n, d, 0.03, seed=seed)
    elif kind == "full":
        X = synth.csr_bernoulli(n, d, 1.0, seed=seed)
    else:
        Xs = synth.csr_bernoulli(n, d, 0.01, seed=seed).to_dense()
        Xs[777, :] = np.random.default_rng(1).standard_normal(d).astype(np.float32)
        X = synth.csr_from_dense(Xs)
    rp, ci, v = dev_csr(X)
    m = 8
    glob = cg().CountGauss(n, d, m, B, seed, deterministic=True, scatter="atomic")
    bins = cg().CountGauss(n, d, m, B, seed, deterministic=True, scatter="binned")
    SXg = glob.sketch_csr(rp, ci, v).cpu().numpy()
    SXb = bins.sketch_csr(rp, ci, v).cpu().numpy()
    SXb2 = bins.sketch_csr(rp, ci, v).cpu().numpy()
    Yb = bins.apply_csr(rp, ci, v).cpu().numpy()
    Yg = glob.apply_csr(rp, ci, v).cpu().numpy()
    glob.check()
    bins.check()
    np.testing.assert_array_equal(SXb, SXg)
    np.testing.assert_array_equal(SXb2, SXb)
    np.testing.assert_array_equal(Yb, Yg)
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, return_sx=True)
    assert rel(SXb, SXo) < 1e-6
    assert rel(Yb, Yo) < FP32_TOL


def test_partition_overflow_path():
    """Few, full rows of 4096 entries hashed to 64 slices of 8 buckets: some slice
    receives far more than its share, so its records spill to the overflow list; the
    result must not change."""
    n, d, m, B, seed = 256, 4096, 8, 512, 9
    X = synth.csr_bernoulli(n, d, 1.0, seed=3)
    rp, ci, v = dev_csr(X)
    Yo, SXo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals, return_sx=True)
    for scatter in ("partition", "atomic"):
        plan = cg().CountGauss(n, d, m, B, seed, scatter=scatter)
        SX = plan.sketch_csr(rp, ci, v).cpu().numpy()
        Y = plan.apply_csr(rp, ci, v).cpu().numpy()
        plan.check()
        assert rel(SX, SXo) < 1e-6
        assert rel(Y, Yo) < FP32_TOL


@pytest.mark.parametrize("n,d,m,B,seed,kind", CASES)
def test_plain_parity(n, d, m, B, seed, kind):
    X = make_input(n, d, seed, kind)
    plan = cg().CountGauss(n, d, m, B, seed)
    Y = plan.plain_csr(*dev_csr(X)).cpu().numpy()
    plan.check()
    Yo = oracle.plain_csr(seed, n, d, m, X.row_ptr, X.col_idx, X.vals)
    assert rel(Y, Yo) < FP32_TOL, rel(Y, Yo)


@pytest.mark.parametrize("n,d,m,B,seed", [(4099, 64, 32, 1024, 1), (1000, 37, 13, 100, 2), (333, 128, 64, 700, 3),
                                          (50, 4, 4, 1, 4)])
def test_apply_dense_parity(n, d, m, B, seed):
    Xn = synth.dense_normal(n, d, seed=seed)
    plan = cg().CountGauss(n, d, m, B, seed)
    X = torch.from_numpy(Xn).cuda()
    Y = plan.apply_dense(X).cpu().numpy()
    SX = plan.sketch_dense(X).cpu().numpy()
    Yo, SXo = oracle.apply_dense(seed, m, B, Xn, return_sx=True)
    assert rel(SX, SXo) < 1e-6
    assert rel(Y, Yo) < FP32_TOL


def test_contract_alone_and_deterministic():
    B, d, m, seed = 5000, 24, 20, 9
    SXn = np.random.default_rng(0).standard_normal((B, d)).astype(np.float32)
    plan = cg().CountGauss(10, d, m, B, seed)
    SX = torch.from_numpy(SXn).cuda()
    Y1 = plan.contract(SX).cpu().numpy()
    Y2 = plan.contract(SX).cpu().numpy()
    np.testing.assert_array_equal(Y1, Y2)  # fixed-order split-K reduction
    assert rel(Y1, oracle.contract(seed, m, SXn)) < FP32_TOL


@pytest.mark.parametrize("m,d", [(96, 96), (40, 64), (130, 200), (33, 130), (8, 16), (64, 128)])
def test_contract_blocks_with_idle_threads(m, d):
    """Output blocks of fewer than 256 thread tiles, where 256 is not a multiple of their
    count (96 x 96: a block of 96 tiles leaves threads past the second k-group; 40 x 64:
    160 tiles), besides full blocks: the FFMA contraction against the oracle, twice."""
    B, seed = 4096, 11
    SXn = np.random.default_rng(m * 1000 + d).standard_normal((B, d)).astype(np.float32)
    plan = cg().CountGauss(10, d, m, B, seed)
    SX = torch.from_numpy(SXn).cuda()
    Y1 = plan.contract(SX).cpu().numpy()
    Y2 = plan.contract(SX).cpu().numpy()
    plan.check()
    np.testing.assert_array_equal(Y1, Y2)
    assert rel(Y1, oracle.contract(seed, m, SXn)) < FP32_TOL


def test_empty_inputs():
    n, d, m, B = 200, 8, 8, 32
    X = synth.csr_bernoulli(n, d, 0.0, seed=1)
    plan = cg().CountGauss(n, d, m, B, 3)
    rp, ci, v = dev_csr(X)
    assert not plan.apply_csr(rp, ci, v).any()
    assert not plan.plain_csr(rp, ci, v).any()
    plan0 = cg().CountGauss(0, d, m, B, 3)
    rp0 = torch.zeros(1, dtype=torch.int32, device="cuda")
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    ev = torch.zeros(0, dtype=torch.float32, device="cuda")
    assert not plan0.apply_csr(rp0, e, ev).any()
    assert not plan0.plain_csr(rp0, e, ev).any()
    plan0.check()


def test_row_offset_shards_sum_to_whole():
    """Shards with global row offsets (the distributed remark of Section 4)."""
    n, d, m, B, seed = 10000, 16, 16, 512, 21
    X = synth.csr_bernoulli(n, d, 0.1, seed=5)
    whole = cg().CountGauss(n, d, m, B, seed).apply_csr(*dev_csr(X)).cpu().numpy().astype(np.float64)
    whole_p = cg().CountGauss(n, d, m, B, seed).plain_csr(*dev_csr(X)).cpu().numpy().astype(np.float64)
    acc = np.zeros_like(whole)
    acc_p = np.zeros_like(whole_p)
    cuts = [0, 3333, 3334, 9001, n]
    for a, b in zip(cuts, cuts[1:]):
        sub = synth.CSR(b - a, d, X.row_ptr[a:b + 1] - X.row_ptr[a], X.col_idx[X.row_ptr[a]:X.row_ptr[b]],
                        X.vals[X.row_ptr[a]:X.row_ptr[b]])
        plan = cg().CountGauss(b - a, d, m, B, seed, row_offset=a)
        acc += plan.apply_csr(*dev_csr(sub)).cpu().numpy()
        acc_p += plan.plain_csr(*dev_csr(sub)).cpu().numpy()
    assert rel(acc, whole) < FP32_TOL
    assert rel(acc_p, whole_p) < FP32_TOL


# -----------------------------------------------------------------------------
# Adjoint and autograd.
# -----------------------------------------------------------------------------
@pytest.mark.parametrize("n,d,m,B,seed", [(4099, 64, 64, 1024, 4), (1000, 37, 13, 100, 2), (500, 128, 20, 333, 3)])
def test_adjoint_parity(n, d, m, B, seed):
    rng = np.random.default_rng(seed)
    dYn = rng.standard_normal((m, d)).astype(np.float32)
    plan = cg().CountGauss(n, d, m, B, seed)
    dY = torch.from_numpy(dYn).cuda()
    dX = plan.adjoint(dY).cpu().numpy()
    assert rel(dX, oracle.adjoint_dense(seed, n, m, B, dYn)) < FP32_TOL
    X = synth.csr_ragged(n, d, seed=seed) if d < 100 else synth.csr_bernoulli(n, d, 0.05, seed=seed)
    rp, ci, _ = dev_csr(X)
    dXv = plan.adjoint(dY, rp, ci).cpu().numpy()
    plan.check()
    assert rel(dXv, oracle.adjoint_csr(seed, n, m, B, X.row_ptr, X.col_idx, dYn)) < FP32_TOL
    # dot-product test on the device results: <T X, dY> = <X, T^T dY>
    Xd = torch.from_numpy(synth.dense_normal(n, d, seed=seed + 1)).cuda()
    lhs = float((plan.apply_dense(Xd).double() * dY.double()).sum())
    rhs = float((Xd.double() * torch.from_numpy(dX).cuda().double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * max(1.0, abs(lhs))


def test_autograd_dense_and_csr():
    n, d, m, B, seed = 3000, 16, 8, 256, 6
    plan = cg().CountGauss(n, d, m, B, seed)
    X = torch.from_numpy(synth.dense_normal(n, d, seed=1)).cuda().requires_grad_(True)
    dYn = np.random.default_rng(2).standard_normal((m, d)).astype(np.float32)
    Y = cg().countgauss_dense(X, plan)
    Y.backward(torch.from_numpy(dYn).cuda())
    assert rel(X.grad.cpu().numpy(), oracle.adjoint_dense(seed, n, m, B, dYn)) < FP32_TOL
    Xs = synth.csr_bernoulli(n, d, 0.1, seed=3)
    rp, ci, v = dev_csr(Xs)
    v = v.clone().requires_grad_(True)
    Ys = cg().countgauss_csr(v, rp, ci, plan)
    Ys.backward(torch.from_numpy(dYn).cuda())
    assert rel(v.grad.cpu().numpy(), oracle.adjoint_csr(seed, n, m, B, Xs.row_ptr, Xs.col_idx, dYn)) < FP32_TOL


def test_sketched_least_squares_gradient():
    """Loss 1/2 ||T (X w - b)||^2: T applied to the d = 1 residual, gradient
    X^T T^T T (X w - b), against the oracle."""
    n, d, m, B, seed = 1 << 14, 64, 64, 1 << 12, 4
    rng = np.random.default_rng(4)
    Xn = rng.standard_normal((n, d)).astype(np.float32)
    bn = rng.standard_normal((n, 1)).astype(np.float32)
    wn = rng.standard_normal((d, 1)).astype(np.float32)
    plan = cg().CountGauss(n, 1, m, B, seed)
    X, b = torch.from_numpy(Xn).cuda(), torch.from_numpy(bn).cuda()
    w = torch.from_numpy(wn).cuda().requires_grad_(True)
    r = X @ w - b
    loss = 0.5 * (cg().countgauss_dense(r, plan) ** 2).sum()
    loss.backward()
    r64 = Xn.astype(np.float64) @ wn.astype(np.float64) - bn.astype(np.float64)
    Tr = oracle.apply_dense(seed, m, B, r64)
    g = Xn.astype(np.float64).T @ oracle.adjoint_dense(seed, n, m, B, Tr)
    assert abs(float(loss.detach()) - 0.5 * float(np.sum(Tr ** 2))) < 1e-4 * 0.5 * float(np.sum(Tr ** 2))
    assert rel(w.grad.cpu().numpy(), g) < 1e-4  # X w - b in fp32 (torch) dominates


# -----------------------------------------------------------------------------
# Device bounds checks: a bad column index is skipped and reported, never used.
# -----------------------------------------------------------------------------
def test_bad_column_index_is_reported():
    n, d, m, B = 100, 8, 4, 16
    X = synth.csr_bernoulli(n, d, 0.5, seed=1)
    ci = X.col_idx.copy()
    ci[len(ci) // 2] = d + 5  # out of range: the kernels check before use
    plan = cg().CountGauss(n, d, m, B, 1)
    rp = torch.from_numpy(X.row_ptr.astype(np.int32)).cuda()
    cit = torch.from_numpy(ci).cuda()
    v = torch.from_numpy(X.vals).cuda()
    plan.apply_csr(rp, cit, v)
    with pytest.raises(cg()._lib.CountGaussError if hasattr(cg(), "_lib") else RuntimeError):
        plan.check()
    plan.check()  # cleared


def test_argument_errors_raise():
    """Wrong dtypes are refused before the call (row offsets int32 or int64, column
    indices int32, values float32)."""
    plan = cg().CountGauss(10, 4, 4, 8, 1)
    rp = torch.zeros(11, dtype=torch.int32, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    v = torch.zeros(0, device="cuda")
    for args in ((rp.short(), ci, v), (rp.double(), ci, v), (rp, ci.long(), v), (rp.long(), ci.long(), v),
                 (rp, ci, v.double())):
        with pytest.raises(TypeError):
            plan.apply_csr(*args)


def test_diag_random_reductions_adds_exactly_count():
    """The reduction-rate diagnostic adds 1.0 exactly `count` times (each cell stays an
    exact integer), and spreads the adds over the whole array."""
    a = torch.zeros(100003, device="cuda")
    cg().diag_random_reductions(a, 3_000_000)
    h = a.cpu().numpy().astype(np.float64)
    assert h.sum() == 3_000_000
    assert (h == np.round(h)).all()
    assert (h > 0).mean() > 0.99
    from paper_1606_05732_gb300 import _lib
    with pytest.raises(_lib.CountGaussError):
        cg().diag_random_reductions(a, -1)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("n,d,m,B,seed", [(64, 65536, 4, 8, 51), (1000, 4, 65536, 16, 52)])
def test_largest_d_and_m(n, d, m, B, seed, precision):
    """The widest X (d = 65536 columns: 512 FFMA column tiles, 256 tensor-core ones) and
    the tallest output (m = 65536 rows of G), each at the plan's limit."""
    X = synth.csr_bernoulli(n, d, 0.01 if d > 1000 else 0.5, seed=seed)
    rp, ci, v = dev_csr(X)
    plan = cg().CountGauss(n, d, m, B, seed, precision=precision)
    Y = plan.apply_csr(rp, ci, v).cpu().numpy()
    plan.check()
    Yo = oracle.apply_csr(seed, n, d, m, B, X.row_ptr, X.col_idx, X.vals)
    assert Y.shape == (m, d)
    assert rel(Y, Yo) < FP32_TOL


@pytest.mark.parametrize("n,d,m,seed", [(3000, 300, 512, 61), (2000, 1000, 301, 62)])
def test_plain_in_tiles_of_rows(n, d, m, seed):
    """The plain product for an m x d accumulator larger than shared memory runs in tiles
    of rows of G~ (512 x 300: four tiles of 128; 301 x 1000: nine tiles of 32 and a last
    one of 13 rows, whose Gaussian group is partial); every row against the oracle."""
    X = synth.csr_bernoulli(n, d, 0.05, seed=seed)
    rp, ci, v = dev_csr(X)
    plan = cg().CountGauss(n, d, m, 64, seed, row_offset=5)
    Yp = plan.plain_csr(rp, ci, v).cpu().numpy()
    plan.check()
    want = oracle.plain_csr(seed, n, d, m, X.row_ptr, X.col_idx, X.vals, row_offset=5)
    assert Yp.shape == (m, d)
    assert rel(Yp, want) < FP32_TOL


@pytest.mark.parametrize("shift", [0, 4])
@pytest.mark.parametrize("n,d,B,seed", [(3000, 7, 101, 61), (200_000, 101, 16383, 62)])
def test_small_sketch_cleared_in_place(n, d, B, seed, shift):
    """An SX of at most 8 MB is cleared by a zero-fill kernel that the scatter follows as a
    programmatic dependent.  It clears exactly the B x d floats of a caller's SX (NaN
    beforehand; B x d not a multiple of 4; the floats around them keep their NaN) and the
    sketch equals the oracle's.  An SX not on a 16-byte boundary is refused."""
    X = synth.csr_bernoulli(n, d, 0.02, seed)
    rp, ci, v = dev_csr(X)
    buf = torch.full((B * d + 8,), float("nan"), device="cuda")
    SX = buf[shift:shift + B * d]
    plan = cg().CountGauss(n, d, 4, B, seed)
    plan.sketch_csr(rp, ci, v, out=SX)
    plan.check()
    SXo = oracle.sketch_csr(seed, n, d, B, X.row_ptr, X.col_idx, X.vals)
    assert rel(SX.view(B, d).cpu().numpy(), SXo) < 1e-6
    assert torch.isnan(torch.cat([buf[:shift], buf[shift + B * d:]])).all()
    from paper_1606_05732_gb300 import _lib
    with pytest.raises(_lib.CountGaussError):
        plan.sketch_csr(rp, ci, v, out=buf[shift + 1:shift + 1 + B * d])

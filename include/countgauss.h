/*
 * countgauss.h -- C ABI of libcountgauss, a GB300 (sm_103a) implementation of the
 * CountGauss transform of Kapralov, Potluru and Woodruff, "How to Fake Multiply by
 * a Gaussian Matrix".
 *
 * The transform (Section 1.1 "Our Results"; Section 2, Theorem 1):
 *   X  is n x d (n >> d), sparse (CSR) or dense;
 *   S  is a B x n CountSketch: column i of S has one nonzero, sigma(i) = +-1, at row
 *      h(i) in [0, B)  (Section 1.1; Section 7);
 *   G  is m x B with i.i.d. N(0,1) entries (Theorem 1: unit variance, no scaling);
 *   T = G.S, and T.X is computed as G.(S.X) in O(nnz(X)) + O(m.B.d) work instead
 *   of the O(nnz(X).m) of the plain product G~.X with an m x n Gaussian G~
 *   (Abstract; Section 4; Algorithm 1 steps 1-2).
 *
 * Randomness.  h, sigma, G and G~ are pure functions of (seed, index): Philox4x32-10
 * (Salmon et al., SC'11) with key (lo32(seed), hi32(seed)) and counter
 * (lo32(idx), hi32(idx), tag, 0).  tag 0, idx = floor(i/4) for global row i, w = word
 * i mod 4 of that call: h(i) = floor(w.B/2^32), sigma(i) = -1 iff bit 0 of w is set (one
 * call serves four consecutive rows).  Uniforms u(w) = (2(w>>9)+1).2^-24.  Entry
 * (r, c) of an R x C Gaussian with tag t is lane r%4 of the Box-Muller quadruple
 *   (sqrt(-2 ln u0) cos 2pi u1, sqrt(-2 ln u0) sin 2pi u1,
 *    sqrt(-2 ln u2) cos 2pi u3, sqrt(-2 ln u2) sin 2pi u3)
 * of the call at idx = c.ceil(R/4) + floor(r/4): G is tag 1 (R = m, C = B), G~ is
 * tag 2 (R = m, C = global row).  Because nothing is stored, every process that
 * shares the seed holds the same T (the distributed remark of Section 4); a shard of
 * X whose first row is global row o sets CG_OPT_ROW_OFFSET = o, and the shards'
 * outputs sum to the output of the whole X.
 *
 * Conventions shared by every entry point:
 *   - Every pointer argument named as device memory must be device memory of the
 *     current CUDA device; the caller owns it, allocates it and frees it.  The plan
 *     owns host memory only.
 *   - Dense matrices are row-major fp32.  Y is m x d, SX is B x d, W is B x d.
 *   - CSR X: row_ptr int32[n+1] with row_ptr[0] = 0 and row_ptr[n] = nnz,
 *     col_idx int32[nnz] in [0, d) (any order within a row; duplicates are summed),
 *     vals fp32[nnz].  nnz <= 2^31 - 2^20 (the margin keeps the kernels' 32-bit
 *     indices from overflowing as they step past the last entry).  The *_i64 entry
 *     points take row_ptr int64[n+1] instead, for up to 2^40 entries.
 *   - ws is a device workspace of at least cg_workspace_size() bytes, 256-byte
 *     aligned.  Its first 256 bytes hold a device status word that the kernels set
 *     when a bounds check fails (the offending element is skipped, never accessed)
 *     or a bounded wait gives up; cg_plan_check() reads and clears it.  The caller
 *     zeroes those 256 bytes once when it allocates the workspace; kernels only
 *     ever set bits, so a nonzero word means some call since the last check failed.
 *   - Entry points are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream), never synchronise, never print and never abort.  Argument
 *     errors are found on the host before anything is launched and reported as
 *     CG_ERR_INVALID_ARG / CG_ERR_UNSUPPORTED / CG_ERR_WORKSPACE; a launch failure
 *     is CG_ERR_CUDA.
 *   - A plan may be used from one host thread at a time.
 */
#ifndef COUNTGAUSS_H
#define COUNTGAUSS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CG_API __attribute__((visibility("default")))
#else
#define CG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cg_plan cg_plan;

typedef enum cg_status {
    CG_OK = 0,
    CG_ERR_INVALID_ARG = 1,   /* bad size, null pointer, misaligned buffer */
    CG_ERR_UNSUPPORTED = 2,   /* valid request outside what the library implements */
    CG_ERR_WORKSPACE = 3,     /* ws_bytes smaller than cg_workspace_size() */
    CG_ERR_CUDA = 4,          /* a CUDA call or kernel launch failed */
    CG_ERR_TIMEOUT = 5,       /* a bounded device wait gave up (batched path) */
    CG_ERR_DEVICE_BOUNDS = 6, /* a kernel met an index outside its buffer and skipped it */
    CG_ERR_NO_DEVICE = 7      /* no usable CUDA device */
} cg_status;

typedef enum cg_precision {
    CG_PREC_FP32 = 0,     /* FFMA, fp32 throughout */
    CG_PREC_BF16 = 1,     /* tcgen05 kind::f16, bf16 G and SX, fp32 accumulate in TMEM */
    CG_PREC_BF16X3 = 2,   /* split bf16: hi.hi + hi.lo + lo.hi, fp32 accumulate */
    CG_PREC_FP8_E4M3 = 3, /* tcgen05 kind::f8f6f4, e4m3 with a per-tile scale for every 128 x N tile
                             of SX (absmax / 448) and G quantised as e4m3(64 z) */
    CG_PREC_FP8X3 = 4     /* split e4m3: hi.hi + hi.lo + lo.hi with the same per-tile scales */
} cg_precision;

typedef enum cg_option {
    CG_OPT_PRECISION = 1,     /* cg_precision of the Gaussian contraction (default FP32) */
    CG_OPT_DETERMINISTIC = 2, /* 0: fp32 atomic scatter (default); 1: exact int64 fixed-point
                                 sums of the scatter, rounded once to fp32: independent of
                                 the order of the reductions, so bit-reproducible run to run.
                                 The sums live in one int64 array of B x d in the workspace, or,
                                 once that array is larger than 60 % of the L2 (or with
                                 CG_OPT_SCATTER = 4), in shared memory one slice of buckets at
                                 a time (the binned scatter's slices and workspace, option 4
                                 of CG_OPT_SCATTER); CG_OPT_SCATTER = 1 keeps the array.
                                 Both forms give the same bits. */
    CG_OPT_ROW_OFFSET = 3,    /* global index of local row 0 (default 0) */
    CG_OPT_KSPLIT = 4,        /* CTAs along B in the contraction; 0 = automatic */
    CG_OPT_SKETCH_CTAS = 5,   /* CTAs of the scatter kernel; 0 = automatic */
    CG_OPT_TIMING = 6,        /* 1: record CUDA events around each main kernel launch
                                 (read with cg_plan_timing); 0 (default): off */
    CG_OPT_SCATTER = 7,       /* CSR scatter algorithm (atomic mode): 0 = automatic (default: 3
                                 when SX is larger than 60 % of the L2, else 1),
                                 1 = one L2 reduction per nonzero, 2 = partition the nonzeros by
                                 bucket range and accumulate each range in shared memory, 3 =
                                 reduce the rows of buckets below a split point at once and
                                 write the others as records reduced by a second pass (each
                                 part of SX in L2 in turn: the lower part up to 0.62 of the L2,
                                 at least B/2; workspace + 8 bytes per nonzero; needs
                                 B d < 2^32),
                                 4 = bin the nonzeros by slices of buckets (a power of two,
                                 at most 32768 / d) into 6-byte records and sum each slice in
                                 shared memory (workspace about 14 bytes per nonzero; needs
                                 d <= 32768 and at most 2048 slices) */
    CG_OPT_SCATTER_PASSES = 8, /* bucket-range passes of the atomic CSR scatter (each pass streams
                                 the CSR and reduces the rows of one range of buckets, keeping
                                 that range of SX in L2); 0 = automatic (one pass), 1..16 forced */
    CG_OPT_SCATTER_ROWS = 9,  /* CSR rows per warp chunk of the scatter: 0 = automatic (one row
                                 per lane for n <= 2^18 with under two nonzeros per row, where
                                 latency rules; else the smallest of 32, 64, 128 whose chunk
                                 holds about 96 nonzeros on average; 256 in the deferred scatter
                                 for rows of under 1.5 nonzeros), 32, 64, 128 forced (rows staged in shared memory,
                                 nonzeros swept 32 at a time), 256 forced (deferred scatter only;
                                 the others take it as automatic), or 1 (one row per lane, each
                                 lane walking its own row; one-pass scatters only) */
    CG_OPT_HOST_CHUNK = 10,   /* cg_apply_csr_host: most nonzeros, and most rows, per chunk copied
                                 to the device; 0 = automatic (nnz / 4 within [2^20, 2^24]), else
                                 32 .. 2^30 */
    CG_OPT_ACCUMULATE = 12,   /* cg_sketch_csr / cg_sketch_dense: 0 (default) = SX is overwritten with
                                 S.X; 1 = S.X is added into the caller's SX.  S.X is additive over
                                 the rows of X, so a matrix fed in row chunks (each with its global
                                 row offset, CG_OPT_ROW_OFFSET) sketches into one SX, and a saved SX
                                 plus the next row offset resumes an interrupted stream.  Not with
                                 CG_OPT_DETERMINISTIC or the partitioned scatter (CG_ERR_UNSUPPORTED) */
    CG_OPT_HOST_READ = 11     /* cg_apply_csr_host: how the kernels get the host CSR.  0 = automatic
                                 (copied), 1 = copied in chunks by the copy engine, 2 = direct: the
                                 scatter kernel reads the host arrays in place over the CPU-GPU
                                 link (no chunk-size limit on rows, no staging).  Direct reads need
                                 all three arrays in page-locked memory mapped into the device's
                                 address space; otherwise the call copies in chunks. */
} cg_option;

typedef enum cg_kernel {
    CG_KERNEL_SKETCH = 0,     /* the CSR / dense scatter kernel (not the SX memset) */
    CG_KERNEL_CONTRACT = 1,   /* the Gaussian contraction kernel (not the split-K sum) */
    CG_KERNEL_PLAIN = 2,      /* the plain G~.X kernel (not the split sum) */
    CG_KERNEL_ADJOINT_W = 3,  /* W = G^T.dY */
    CG_KERNEL_GATHER = 4,     /* dX = S^T.W */
    CG_KERNEL_COUNT = 5
} cg_kernel;

typedef enum cg_op {
    CG_OP_APPLY_CSR = 0,
    CG_OP_APPLY_DENSE = 1,
    CG_OP_ADJOINT_DENSE = 2,
    CG_OP_ADJOINT_CSR = 3,
    CG_OP_PLAIN_CSR = 4,
    CG_OP_SKETCH = 5,         /* cg_sketch_csr / cg_sketch_dense alone */
    CG_OP_CONTRACT = 6,       /* cg_contract alone */
    CG_OP_APPLY_CSR_HOST = 7, /* cg_apply_csr_host */
    CG_OP_APPLY_RIGHT_CSR = 8, /* cg_apply_right_csr */
    CG_OP_APPLY_CSR_I64 = 9,   /* cg_apply_csr_i64 */
    CG_OP_SKETCH_I64 = 10      /* cg_sketch_csr_i64 */
} cg_op;

/* ---- plans ---------------------------------------------------------------- */

/* Create a plan for T = G.S with X of n rows and d columns, m output rows, B sketch
 * rows and the given seed (Section 1.1; Theorem 1).  Limits: 0 <= n <= 2^31 - 2^20,
 * 1 <= d <= 65536, 1 <= m <= 65536, 1 <= B < 2^31, B.d < 2^40.  No CUDA call is made.
 * *out receives a host-side handle to free with cg_plan_destroy. */
CG_API cg_status cg_plan_create(int64_t n, int32_t d, int32_t m, int64_t B, uint64_t seed, cg_plan **out);

CG_API cg_status cg_plan_destroy(cg_plan *plan);

/* Set one cg_option.  Values outside the option's range give CG_ERR_INVALID_ARG. */
CG_API cg_status cg_plan_set_option(cg_plan *plan, int32_t option, int64_t value);
CG_API cg_status cg_plan_get_option(const cg_plan *plan, int32_t option, int64_t *value);

/* Device workspace, in bytes, that `op` needs for a call with `nnz` stored entries
 * (ignored for dense ops).  Depends on the plan's options and on the current
 * device's SM count; query it after setting options. */
CG_API cg_status cg_workspace_size(const cg_plan *plan, int32_t op, int64_t nnz, size_t *bytes);

/* Synchronise `stream`, read the device status word in ws and clear it.  Returns
 * CG_OK, CG_ERR_DEVICE_BOUNDS or CG_ERR_TIMEOUT (or CG_ERR_CUDA). */
CG_API cg_status cg_plan_check(const cg_plan *plan, void *ws, void *stream);

CG_API const char *cg_status_string(cg_status status);

/* With CG_OPT_TIMING on, every launch of `kernel` made through this plan is
 * bracketed by a pair of CUDA events on the launching stream.  This call waits for
 * the recorded events, returns the summed elapsed time (ms) and the number of
 * launches since the last call, and forgets them. */
CG_API cg_status cg_plan_timing(cg_plan *plan, int32_t kernel, double *total_ms, int64_t *launches);

/* ---- the transform -------------------------------------------------------- */

/* Y = G.(S.X) for CSR X (Section 1.1; Algorithm 1 steps 1-2).  Stage 1 scatters
 * sigma(i).X[i,:] into row h(i) of SX (B x d, in ws); stage 2 contracts SX with G,
 * generated in-kernel, never stored.  Y (device, m x d) is overwritten. */
CG_API cg_status cg_apply_csr(cg_plan *plan, const int32_t *row_ptr, const int32_t *col_idx,
                       const float *vals, int64_t nnz, float *Y,
                       void *ws, size_t ws_bytes, void *stream);

/* cg_apply_csr for a matrix of 2^31 nonzeros or more: the same transform (Section 1.1;
 * Algorithm 1 steps 1-2) with 64-bit row offsets, row_ptr int64[n+1] (device, 8-byte
 * aligned), col_idx int32[nnz], vals fp32[nnz], 0 <= nnz <= 2^40.  The scatter is the
 * one-pass atomic scatter (CG_OPT_SCATTER 1; CG_OPT_SCATTER_PASSES and
 * CG_OPT_SCATTER_ROWS apply) or the deferred scatter (CG_OPT_SCATTER 3, and automatic
 * for an SX larger than 60 % of the L2, as in cg_apply_csr; the workspace then holds 8
 * bytes per nonzero), each warp chunk of rows taking its offsets relative to its first
 * nonzero.  Y (device, m x d) is overwritten.  Workspace:
 * cg_workspace_size(CG_OP_APPLY_CSR_I64, nnz).  Errors: CG_ERR_INVALID_ARG for null or
 * misaligned pointers or nnz out of range; CG_ERR_UNSUPPORTED with CG_OPT_DETERMINISTIC
 * = 1 or CG_OPT_SCATTER 2 or 4.  Out-of-range column indices, out-of-range or decreasing
 * row offsets, and a chunk of rows (at most 256 consecutive rows) holding more than
 * 2^31 - 2^20 stored entries are reported through the status word, the entries concerned
 * skipped. */
CG_API cg_status cg_apply_csr_i64(cg_plan *plan, const int64_t *row_ptr, const int32_t *col_idx,
                                  const float *vals, int64_t nnz, float *Y,
                                  void *ws, size_t ws_bytes, void *stream);

/* Y = G.(S.X) for dense X (device, n x d, row stride ldx >= d floats). */
CG_API cg_status cg_apply_dense(cg_plan *plan, const float *X, int64_t ldx, float *Y,
                         void *ws, size_t ws_bytes, void *stream);

/* Adjoint: dX = S^T.(G^T.dY) (T is linear, Section 1.1).  dY is m x d (device).
 * row_ptr == NULL: dX is dense n x d (device).  Otherwise dX holds nnz values, the
 * gradient read at the stored entries of the CSR pattern (row_ptr, col_idx).
 * G is regenerated from the seed, W = G^T.dY (B x d) lives in ws. */
CG_API cg_status cg_apply_adjoint(cg_plan *plan, const float *dY, const int32_t *row_ptr,
                           const int32_t *col_idx, int64_t nnz, float *dX,
                           void *ws, size_t ws_bytes, void *stream);

/* cg_apply_adjoint at the stored entries of a CSR pattern with int64 row offsets (2^31
 * nonzeros or more; see cg_apply_csr_i64): dXv[k] = sigma(i).W[h(i), col_idx[k]] for
 * each stored entry k of row i, W = G^T.dY (B x d) in ws.  row_ptr int64[n+1] (device,
 * 8-byte aligned), col_idx int32[nnz], dXv fp32[nnz] (device) overwritten, 0 <= nnz <=
 * 2^40.  Workspace: cg_workspace_size(CG_OP_ADJOINT_CSR, nnz).  Errors:
 * CG_ERR_INVALID_ARG for null or misaligned pointers or nnz out of range; out-of-range
 * column indices and out-of-range or decreasing row offsets are reported through the
 * status word (the entries concerned are skipped). */
CG_API cg_status cg_apply_adjoint_i64(cg_plan *plan, const float *dY, const int64_t *row_ptr,
                                      const int32_t *col_idx, int64_t nnz, float *dXv,
                                      void *ws, size_t ws_bytes, void *stream);

/* The random projection of the SVM application (Section 9, the theorem on the margin;
 * Table 1 times it): Z = A.R with R = T^T, for a CSR matrix A with one row per sample
 * and one column per feature, i.e. A = X^T in the plan's terms.  A has d rows and n
 * columns: row_ptr int32[d+1] (row_ptr[0] = 0, row_ptr[d] = nnz), col_idx int32[nnz]
 * in [0, n), vals fp32[nnz]; column c is T's column CG_OPT_ROW_OFFSET + c.  Computed
 * as (G.(S.A^T))^T: the nonzero A[r, c] is reduced into SX[h(c), r] (B x d, in ws),
 * then SX is contracted with G as in cg_apply_csr (CG_OPT_PRECISION applies) and the
 * result stored transposed.  Z (device, d x m row-major) is overwritten.  Workspace:
 * cg_workspace_size(CG_OP_APPLY_RIGHT_CSR, nnz).  Out-of-range column indices and
 * out-of-range or decreasing row offsets are reported through the status word (the
 * entries concerned are skipped).  CG_OPT_DETERMINISTIC = 1 gives CG_ERR_UNSUPPORTED. */
CG_API cg_status cg_apply_right_csr(cg_plan *plan, const int32_t *row_ptr, const int32_t *col_idx,
                                    const float *vals, int64_t nnz, float *Z,
                                    void *ws, size_t ws_bytes, void *stream);

/* The plain product Y = G~.X that the method replaces (Abstract; Section 4), with
 * the m x n Gaussian G~ generated on the fly, one column per non-empty row of X.
 * Y (device, m x d) is overwritten. */
CG_API cg_status cg_plain_gaussian_apply(cg_plan *plan, const int32_t *row_ptr, const int32_t *col_idx,
                                  const float *vals, int64_t nnz, float *Y,
                                  void *ws, size_t ws_bytes, void *stream);

/* ---- stages (for stage-wise checks and measurement) ----------------------- */

/* SX = S.X alone (Section 1.1: O(nnz(X)) scatter).  SX (device, B x d) is
 * overwritten, or added into with CG_OPT_ACCUMULATE = 1.  Honours CG_OPT_DETERMINISTIC.
 * SX starts on a 16-byte boundary (else CG_ERR_INVALID_ARG), here and in cg_sketch_dense. */
CG_API cg_status cg_sketch_csr(cg_plan *plan, const int32_t *row_ptr, const int32_t *col_idx,
                        const float *vals, int64_t nnz, float *SX,
                        void *ws, size_t ws_bytes, void *stream);

CG_API cg_status cg_sketch_dense(cg_plan *plan, const float *X, int64_t ldx, float *SX,
                          void *ws, size_t ws_bytes, void *stream);

/* cg_sketch_csr for int64 row offsets (as cg_apply_csr_i64): SX = S.X, or SX += S.X with
 * CG_OPT_ACCUMULATE = 1, e.g. over row chunks of a stream, each with its CG_OPT_ROW_OFFSET.
 * Workspace: cg_workspace_size(CG_OP_SKETCH_I64, nnz) (the status word, and the deferred
 * scatter's records when it runs).  Errors as
 * cg_apply_csr_i64, and CG_ERR_INVALID_ARG for an SX off a 16-byte boundary. */
CG_API cg_status cg_sketch_csr_i64(cg_plan *plan, const int64_t *row_ptr, const int32_t *col_idx,
                                   const float *vals, int64_t nnz, float *SX,
                                   void *ws, size_t ws_bytes, void *stream);

/* Y = G.SX alone (SX device, B x d).  Honours CG_OPT_PRECISION. */
CG_API cg_status cg_contract(cg_plan *plan, const float *SX, float *Y,
                      void *ws, size_t ws_bytes, void *stream);

/* ---- NMF anchors (Algorithm 1) ---------------------------------------------------- */

/* Algorithm 1 step 3: imax[r] / imin[r] = column index of the largest / smallest
 * entry of row r of Z (device, m x d fp32 row-major), lowest index on ties.  imax,
 * imin: device int32[m]. */
CG_API cg_status cg_row_argmax_argmin(const float *Z, int32_t m, int32_t d, int32_t *imax, int32_t *imin,
                                      void *stream);

/* Algorithm 1 steps 1-3 for CSR X: Z = T.X as cg_apply_csr (Z device m x d, workspace
 * of CG_OP_APPLY_CSR), and the row argmax / argmin of Z (imax, imin: device int32[m],
 * lowest column on ties) taken by the split-K sum itself, which gives each row of Z to
 * one thread block: no separate pass over Z.  The sums run in a fixed order per row, so
 * Z is reproducible; it may differ from cg_apply_csr's Z in the last bits (another fixed
 * order).  Errors as cg_apply_csr, and CG_ERR_INVALID_ARG for null or misaligned imax /
 * imin. */
CG_API cg_status cg_nmf_anchors_csr(cg_plan *plan, const int32_t *row_ptr, const int32_t *col_idx, const float *vals,
                                    int64_t nnz, float *Z, int32_t *imax, int32_t *imin, void *ws, size_t ws_bytes,
                                    void *stream);

/* The same with int64 row offsets (as cg_apply_csr_i64; workspace of
 * CG_OP_APPLY_CSR_I64). */
CG_API cg_status cg_nmf_anchors_csr_i64(cg_plan *plan, const int64_t *row_ptr, const int32_t *col_idx,
                                        const float *vals, int64_t nnz, float *Z, int32_t *imax, int32_t *imin,
                                        void *ws, size_t ws_bytes, void *stream);

/* ---- distribution checker ----------------------------------------------------------- */

/* FP64 reductions over sample rows Y (device, rows x d fp32 row-major), accumulated
 * into caller buffers (device, zeroed by the caller before the first call):
 *   gram[d x d] += Y^T Y   and   sumsq[0] += ||Y||_F^2   (either may be NULL).
 * Used to check the distributions of Section 7 and Theorem 1 (rows of G.S.X given S
 * are N(0, X^T S^T S X); rows of G~.X are N(0, X^T X)) on the device's own samples. */
CG_API cg_status cg_moments_f64(const float *Y, int64_t rows, int32_t d, double *gram, double *sumsq, void *stream);

/* ---- many instances in one launch ------------------------------------------------ */

/* One CountGauss instance of a batch: its own plan parameters (as cg_plan_create),
 * its CSR input (device, conventions as cg_apply_csr) and its output Y (device,
 * m x d fp32).  Row offset 0, FP32 contraction, atomic scatter. */
typedef struct cg_batch_desc {
    int64_t n;
    int32_t d;
    int32_t m;
    int64_t B;
    uint64_t seed;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const float *vals;
    int64_t nnz;
    float *Y;
} cg_batch_desc;

typedef struct cg_batch_plan cg_batch_plan;

typedef enum cg_batch_option {
    CG_BATCH_OPT_GRAPH = 1,         /* 1 (default): record the launch once in a CUDA graph and replay it */
    CG_BATCH_OPT_SCATTER_NNZ = 2,   /* target nonzeros per scatter work item (default 16384) */
    CG_BATCH_OPT_CONTRACT_FMA = 3,  /* target FMAs per contraction work item (default 2^22) */
    CG_BATCH_OPT_CTAS_PER_SM = 4,   /* persistent CTAs per SM (default 4) */
    CG_BATCH_OPT_WAIT_US = 5,       /* bound on a contraction item's wait for its instance's scatter
                                       (default 2e6 us); on expiry CG_ERR_TIMEOUT via cg_batch_check */
    CG_BATCH_OPT_TEST_DROP_SCATTER_ITEM = 6 /* test hook: leave the first scatter item of instance 0
                                               out of the queue, so that its wait runs out */
} cg_batch_option;

/* Plan a batch (host only; copies the descriptors).  The work of every instance is cut
 * into scatter items (rows) and contraction items (K slabs); one persistent kernel
 * claims them in order, and an instance's contraction items wait (bounded) for its
 * scatter items.  The plan keeps the pointers in the descriptors: the buffers they
 * name must stay valid while the plan is used. */
CG_API cg_status cg_batch_plan_create(const cg_batch_desc *descs, int32_t count, cg_batch_plan **out);
CG_API cg_status cg_batch_plan_destroy(cg_batch_plan *plan);
CG_API cg_status cg_batch_set_option(cg_batch_plan *plan, int32_t option, int64_t value);
CG_API cg_status cg_batch_plan_get_option(const cg_batch_plan *plan, int32_t option, int64_t *value);

/* Device workspace for cg_batch_apply (first 256 bytes: status word, zeroed once by
 * the caller as for cg_apply_csr). */
CG_API cg_status cg_batch_workspace_size(const cg_batch_plan *plan, size_t *bytes);

/* Run every instance: Y_k = G_k.(S_k.X_k).  The first call with a given workspace
 * uploads the instance table and work queue (a host-to-device copy) and, with
 * CG_BATCH_OPT_GRAPH, records the memset and the persistent launch in a CUDA graph;
 * later calls with the same workspace replay the graph on `stream`.  Read the status
 * word with cg_batch_check. */
CG_API cg_status cg_batch_apply(cg_batch_plan *plan, void *ws, size_t ws_bytes, void *stream);

/* Synchronise `stream`, read and clear the status word of a batch workspace:
 * CG_OK, CG_ERR_TIMEOUT or CG_ERR_DEVICE_BOUNDS. */
CG_API cg_status cg_batch_check(const cg_batch_plan *plan, void *ws, void *stream);

/* Autotuner: times the batch `reps` times for each of a small grid of work-item sizes
 * and CTAs per SM (synchronises), keeps the fastest in the plan and returns its time
 * per run in *best_ms (may be NULL). */
CG_API cg_status cg_batch_autotune(cg_batch_plan *plan, void *ws, size_t ws_bytes, void *stream, int32_t reps,
                                   double *best_ms);

/* ---- without a workspace ------------------------------------------------------ */

/* The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory when they apply the transform (code inside an
 * allocator or memory-pool callback, plugins handed only their input and output
 * buffers by a host framework that owns every allocation, real-time loops that ban
 * cudaMalloc/cudaFree after start-up).
 *
 * Same result as cg_apply_csr (FP32 precision, atomic one-pass scatter), but every
 * piece of scratch (SX, the split-K partials, the status word) lives in one fixed
 * device array of CG_NOALLOC_SCRATCH_BYTES inside the library.  The caller passes only
 * inputs and Y.
 *   - Nothing is allocated by the call itself: no cudaMalloc, cudaFree or allocating
 *     library call.
 *   - The array comes into device memory with the library's module.  With lazy module
 *     loading (the CUDA default) that happens at the first call on each device, which
 *     also looks up the array's device address (with that device current) and caches
 *     it per device and context; a device reset or a new context makes the next call
 *     look it up again.  So make one call on each device at start-up, outside allocator
 *     callbacks and before any stream capture, so that later calls only launch
 *     kernels.  A GPU holds the array from that first call until the process exits.
 *   - Plans needing more than CG_NOALLOC_SCRATCH_BYTES of scratch (roughly
 *     B.d.4 + splits.m.d.4 + 512 bytes) are rejected with CG_ERR_WORKSPACE; other
 *     options return CG_ERR_UNSUPPORTED unless the plan is FP32 and not deterministic.
 *   - All calls share the one array, which keeps the last call's contents (each call
 *     clears what must start at zero).  Calls whose kernels overlap on the GPU (two
 *     streams, or two host threads) race on it and corrupt each other's results:
 *     serialise them, e.g. on one stream.
 *   - Device-side bounds reports are not surfaced here; diagnose bad inputs with
 *     cg_apply_csr and cg_plan_check.  CG_OPT_TIMING records nothing for these calls
 *     (cg_plan_timing keeps reporting the plan's other calls). */
#define CG_NOALLOC_SCRATCH_BYTES (16u << 20)

CG_API cg_status cg_apply_csr_noalloc(cg_plan *plan, const int32_t *row_ptr, const int32_t *col_idx,
                                      const float *vals, int64_t nnz, float *Y, void *stream);

/* ---- the generator, exposed for bit-exact checks ---------------------------- */

/* words[4t..4t+3] = Philox4x32-10 words of (seed, tag, idx0 + t), t < count
 * (device uint32 buffer of 4.count). */
CG_API cg_status cg_generate_words(uint64_t seed, uint32_t tag, uint64_t idx0, int64_t count,
                            uint32_t *words, void *stream);

/* h[t], sigma[t] of global rows row0 + t, t < count (device buffers). */
CG_API cg_status cg_generate_hash_sign(uint64_t seed, int64_t B, int64_t row0, int64_t count,
                                int32_t *h, int32_t *sigma, void *stream);

/* Rows [r0, r1) x columns [c0, c1) of the R x C Gaussian with `tag` (1: G, 2: G~),
 * row-major into out (device, (r1-r0) x (c1-c0) floats), with the same fp32
 * Box-Muller the kernels use. */
CG_API cg_status cg_generate_gaussian(uint64_t seed, uint32_t tag, int64_t R, int64_t r0, int64_t r1,
                               int64_t c0, int64_t c1, float *out, void *stream);

/* Y = T.X (as cg_apply_csr) for a CSR X held in HOST memory, with Y written to HOST
 * memory: the end-to-end form, for callers whose data live on the host.  With direct
 * reads (CG_OPT_HOST_READ), the scatter kernel streams the page-locked host arrays
 * itself over the CPU-GPU link and nothing is staged.  Otherwise the rows are
 * cut into chunks of at most CG_OPT_HOST_CHUNK nonzeros and rows (boundaries found by
 * binary search on the host row_ptr before anything is enqueued); an internal copy
 * stream copies chunk c + 1 into one of two staging buffers of the workspace while chunk
 * c is scattered on `stream`, then the contraction runs on `stream` and Y (m x d, row-
 * major) is copied back.  Pinned (page-locked) host memory lets the copies overlap the
 * scatter; pageable memory works but its copies are not asynchronous.  The call returns
 * after enqueueing: Y is valid, and the host arrays may be changed or freed, once
 * `stream` has reached the end of the call (e.g. after cudaStreamSynchronize).
 * row_ptr (n + 1 entries, read by the host during the call), col_idx, vals (nnz entries
 * each): host pointers.  ws: device workspace of cg_workspace_size(plan,
 * CG_OP_APPLY_CSR_HOST, nnz) bytes.  Errors: CG_ERR_INVALID_ARG for null or misaligned
 * pointers or row offsets outside [0, nnz] at a chunk boundary (offsets inside a chunk
 * are checked on the device, as in cg_apply_csr); CG_ERR_UNSUPPORTED for a
 * deterministic plan, the partitioned scatter, or a row with more nonzeros than the
 * chunk size.  Paper: Section 1.1 (the transform); the chunking is an implementation
 * matter with no counterpart in the paper. */
CG_API cg_status cg_apply_csr_host(cg_plan *plan, const int32_t *row_ptr, const int32_t *col_idx,
                                   const float *vals, int64_t nnz, float *Y, void *ws, size_t ws_bytes,
                                   void *stream);

/* ---- diagnostics ----------------------------------------------------------------
 * No counterpart in the paper.  The CSR scatter makes one fp32 reduction into SX per
 * nonzero, so on a GPU whose L2 reduction rate is below what its memory bandwidth
 * could feed, that rate and not HBM bandwidth bounds the scatter.  This call measures
 * the bound: it adds 1.0f at `count` pseudo-random positions of `array` (device,
 * `cells` floats, 4-byte aligned; position of the k-th add = lowbias32(k) mod cells,
 * lowbias32 being C. Wellons' 32-bit integer hash) with the scatter kernel's grid and
 * block shape, asynchronously on `stream`; time it with events around the call.  The
 * sum of `array` grows by exactly `count` (each cell stays an exact integer below
 * 2^24).  Errors: CG_ERR_INVALID_ARG for a null or misaligned array, cells < 1 or
 * cells >= 2^32, count < 0 or count >= 2^32. */
CG_API cg_status cg_diag_random_reductions(float *array, int64_t cells, int64_t count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* COUNTGAUSS_H */

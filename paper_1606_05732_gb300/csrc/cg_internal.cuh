// cg_internal.cuh -- declarations shared by the translation units of libcountgauss.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>

#include "../../include/countgauss.h"
#include "cg_rng.cuh"

struct cg_plan {
    int64_t n;
    int32_t d;
    int32_t m;
    int64_t B;
    uint64_t seed;
    int32_t precision;      // cg_precision
    int32_t deterministic;  // 0 / 1
    int64_t row_offset;
    int64_t ksplit;         // 0 = auto
    int64_t sketch_ctas;    // 0 = auto
    int32_t timing;         // CG_OPT_TIMING
    void *timing_state;     // cg::TimingState*, created on first timed launch
    int32_t scatter;        // CG_OPT_SCATTER
    int32_t scatter_passes; // CG_OPT_SCATTER_PASSES (0 = auto)
    int32_t scatter_rows;   // CG_OPT_SCATTER_ROWS (0 = auto)
    int64_t host_chunk;     // CG_OPT_HOST_CHUNK (0 = auto)
    int32_t host_read;      // CG_OPT_HOST_READ (0 = auto, 1 = copied, 2 = direct)
    int32_t accumulate;     // CG_OPT_ACCUMULATE (cg_sketch_*: 1 = add into SX)
    void *host_state;       // copy stream and events of cg_apply_csr_host, created on first use
};

namespace cg {

// An NVTX range named after a C-ABI call, open for the call's duration (profiler
// timelines show which call enqueued which kernels; without a tool attached it is a no-op).
class NvtxRange {
  public:
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// A pair of events recorded immediately before and after one kernel launch.
struct EventPair {
    cudaEvent_t start = nullptr;
    cudaEvent_t stop = nullptr;
};

// Fresh event pair for a launch of `kernel` through plan p, or nullptr when timing
// is off (cg_api.cu).
const EventPair *timing_pair(cg_plan *p, int kernel);

inline void record(const EventPair *ev, bool start, cudaStream_t s) {
    if (ev != nullptr) cudaEventRecord(start ? ev->start : ev->stop, s);
}

// Programmatic dependent launch: a kernel launched with launch_after_previous may be
// scheduled while the kernel before it in the stream is finishing (its blocks exit), and
// must call pdl_wait() before it reads anything that kernel wrote.  pdl_wait() returns at
// once for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_after_previous(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                                  Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Device status word bits (first word of every workspace).
constexpr int kStatusBounds = 1;
constexpr int kStatusTimeout = 2;

constexpr size_t kStatusBytes = 256;

// Most stored entries of a CSR input: below 2^31 by a margin, so that the kernels' 32-bit
// nonzero indices never overflow when they step past the last entry (by at most a few
// thousand per step).
constexpr int64_t kMaxNnz = (1LL << 31) - (1LL << 20);
// Most rows of X, with the same margin for the kernels' 32-bit row indices.
constexpr int64_t kMaxRows = (1LL << 31) - (1LL << 20);
// Stored entries of a matrix given with 64-bit row offsets (cg_apply_csr_i64).
constexpr int64_t kMaxNnz64 = 1LL << 40;

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// SM count of the current device (cached per device).  Returns 0 without a device.
int num_sms();

// Resident CTAs per SM of `kernel` launched with `threads` threads and `dyn_smem` bytes
// of dynamic shared memory, from its register and shared-memory use and the current
// device's limits; with tmem_cols > 0 also at most 512 / tmem_cols, so that the TMEM
// allocations of all resident CTAs fit an SM together.  1 if a query fails.
int resident_ctas_per_sm(const void *kernel, int threads, size_t dyn_smem, int tmem_cols);

// ---- scatter (cg_sketch.cu) -------------------------------------------------
// The scatter launchers clear SX first unless `clear` is false (then they add into it).
cudaError_t launch_sketch_csr_atomic(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                     uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, int *status,
                                     int ctas, int passes, int rows, const EventPair *ev, cudaStream_t stream,
                                     bool clear = true);
// The same with 64-bit row offsets (a matrix of 2^31 nonzeros or more); each warp chunk of
// rows holds at most kMaxChunkNnz nonzeros, or is skipped and reported as malformed.
cudaError_t launch_sketch_csr_atomic_i64(const long long *row_ptr, const int *col_idx, const float *vals, int n,
                                         int d, uint32_t B, long long nnz, Key key, int64_t row_offset, float *SX,
                                         int *status, int ctas, int passes, int rows, const EventPair *ev,
                                         cudaStream_t stream, bool clear = true);
cudaError_t launch_sketch_dense_atomic(const float *X, int64_t ldx, int n, int d, uint32_t B, Key key,
                                       int64_t row_offset, float *SX, int *status, int ctas, const EventPair *ev,
                                       cudaStream_t stream, bool clear = true);
int sketch_default_ctas();
// Rows [0, n) of a chunk of a CSR matrix into SX (no clearing, one pass): row_ptr holds
// the chunk's n + 1 offsets into the whole matrix, col_idx / vals hold its nonzeros
// [klo, khi), i.e. nonzero k is col_idx[k - klo]; row i of the chunk is global row
// row_offset + i.
cudaError_t launch_sketch_csr_rows_chunk(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                         uint32_t B, int klo, int khi, Key key, int64_t row_offset, float *SX,
                                         int *status, int ctas, int rows, cudaStream_t stream);
// max |x| over the finite values into maxbits[0] (bit pattern of a non-negative float,
// atomicMax) and a non-finite flag into maxbits[1]; the caller zeroes both first.
cudaError_t launch_absmax(const float *vals, int nnz, int *maxbits, cudaStream_t stream);
// Adds every non-finite entry's sigma x to its cell of SX when maxbits[1] is set (the rule
// of the fixed-point sums for NaN and infinities).
cudaError_t launch_add_nonfinite(const int *row_ptr, const int *col_idx, const float *vals, int n, int d, uint32_t B,
                                 int nnz, Key key, int64_t row_offset, const int *maxbits, float *SX,
                                 cudaStream_t stream);
// Deterministic scatter: exact int64 fixed-point sums (scratch of sketch_fixed_scratch_bytes).
size_t sketch_fixed_scratch_bytes(int64_t B, int d);
cudaError_t launch_sketch_csr_fixed(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                    uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, void *scratch,
                                    int *status, int ctas, int rows, const EventPair *ev, cudaStream_t stream);

// Rows per warp chunk of the one-pass scatter for plan p and nnz nonzeros (cg_api.cu).
int one_pass_rows(const cg_plan &p, int64_t nnz);

// ---- deferred scatter (cg_sketch_defer.cu) -----------------------------------------
// SX split at bucket bsplit: one CSR pass reduces the lower part and writes the rest as
// records, a second pass reduces the records (for an SX larger than the L2 holds).
// staged_ok: the CSR arrays are device memory, so pass 1 may stage them in shared memory
// with bulk copies (when col_idx and vals are 16-byte aligned and B d <= 2^31).
bool deferred_supported(int64_t B, int d);
// CTAs of the deferred scatter for n rows and nnz nonzeros (`ctas` > 0: as given;
// `rows`: the CG_OPT_SCATTER_ROWS option).
int sketch_deferred_ctas(int ctas, int64_t n, int64_t nnz, int rows);
size_t sketch_deferred_scratch_bytes(int64_t nnz, int ctas);
cudaError_t launch_sketch_csr_deferred(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                       uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, int *status,
                                       void *scratch, int ctas, int rows, const EventPair *ev, cudaStream_t stream,
                                       bool clear = true, bool staged_ok = true);
// The same with int64 row offsets (each warp chunk rebased to its first nonzero, record
// indices and per-CTA counts 64-bit).
cudaError_t launch_sketch_csr_deferred_i64(const long long *row_ptr, const int *col_idx, const float *vals, int n,
                                           int d, uint32_t B, long long nnz, Key key, int64_t row_offset, float *SX,
                                           int *status, void *scratch, int ctas, int rows, const EventPair *ev,
                                           cudaStream_t stream, bool clear);

// ---- binned scatter (cg_sketch_bin.cu) -----------------------------------------
// Nonzeros binned by bucket range (slices of SX that fit in shared memory), each slice
// summed in shared memory and written once (for an SX larger than the L2 holds).
// With `fixed` the slices hold int64 fixed-point sums (half the buckets per slice): the
// deterministic mode's exact, order-independent sums, bit-identical to those of
// launch_sketch_csr_fixed.
bool binned_supported(int64_t n, int d, int64_t B, bool fixed = false);
size_t sketch_binned_scratch_bytes(int64_t n, int d, int64_t B, int64_t nnz, int ctas, bool fixed = false);
cudaError_t launch_sketch_csr_binned(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                     uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, int *status,
                                     void *scratch, int ctas, const EventPair *ev, cudaStream_t stream,
                                     bool clear = true, bool prefetch = true, bool fixed = false);

// Bytes of the L2 of the current device (cached per device; 0 without a device).
int l2_bytes();

// ---- partitioned scatter (cg_sketch_part.cu) --------------------------------------
struct PartLayout {
    int SB = 0;           // buckets per slice
    int P = 0;            // slices
    int G = 0;            // pass-1 CTAs (one record region per CTA and slice)
    int64_t cap = 0;      // records per region
    size_t gcount_off = 0, amax_off = 0, rkeys_off = 0, rvals_off = 0, okeys_off = 0, ovals_off = 0;
    size_t bytes = 0;     // scratch bytes
};
bool partition_supported(const cg_plan &p);
PartLayout partition_layout(const cg_plan &p, int64_t nnz);
cudaError_t launch_sketch_csr_partitioned(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                          uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, int *status,
                                          void *scratch, const PartLayout &L, const EventPair *ev,
                                          cudaStream_t stream);

// ---- contraction (cg_gauss.cu) ----------------------------------------------
// Y = G.SX (m x d row-major), or with `transpose` its transpose (d x m row-major).
int contract_splits(const cg_plan &p);
size_t contract_partials_bytes(const cg_plan &p);
// With imax / imin the split-K sum is the row-owned one that also writes, per row of Y,
// the column of its maximum and of its minimum (Algorithm 1 step 3).
cudaError_t launch_contract_ffma(const float *SX, int m, int d, int64_t B, Key key, int nsplit, float *partials,
                                 float *Y, const EventPair *ev, cudaStream_t stream, bool transpose = false,
                                 int32_t *imax = nullptr, int32_t *imin = nullptr);
// Y = fixed-order sum of nsplit partials of `total` floats; with tr_cols > 0 the
// (total / tr_cols) x tr_cols result is stored transposed.
cudaError_t launch_reduce_splits(const float *partials, int nsplit, int64_t total, float *Y, cudaStream_t stream,
                                 int tr_cols = 0);
// Y (m x d) = fixed-order sum of nsplit partials, one CTA per row, with each row's argmax
// and argmin columns (lowest index on ties) into imax[m], imin[m].
cudaError_t launch_reduce_rows_anchors(const float *partials, int nsplit, int m, int d, float *Y, int32_t *imax,
                                      int32_t *imin, cudaStream_t stream);

// ---- tensor-core contraction (cg_gauss_tc.cu) -----------------------------------
int contract_tc_splits(const cg_plan &p);
cudaError_t launch_contract_tc(const float *SX, int m, int d, int64_t B, Key key, int precision, int nsplit,
                               float *partials, float *Y, int *status, const EventPair *ev, cudaStream_t stream,
                               bool transpose = false, int32_t *imax = nullptr, int32_t *imin = nullptr);

// ---- right projection Z = A.T^T (cg_right.cu) -------------------------------------
// Scratch bytes of the scatter of a rows x n CSR matrix with nnz nonzeros (the table of
// column codes, when it pays), and the scatter SX[h(c), r] += sigma(c) A[r, c] itself
// (SX is B x rows, cleared here).
size_t right_scratch_bytes(int64_t n, int64_t nnz);
cudaError_t launch_right_scatter(const int *row_ptr, const int *col_idx, const float *vals, int rows, int64_t n,
                                 uint32_t B, int nnz, Key key, int64_t col_offset, void *scratch, float *SX,
                                 int *status, const EventPair *ev, cudaStream_t stream);

// ---- plain product (cg_plain.cu) ---------------------------------------------
// Whether the plain product runs for m x d (in tiles of rows of G~ where the m x d
// accumulator does not fit the shared memory), its CTAs, and its partials' bytes.
bool plain_supported(int m, int d);
int plain_ctas(int m, int d);
size_t plain_partials_bytes(int m, int d);
cudaError_t launch_plain_csr(const int *row_ptr, const int *col_idx, const float *vals, int n, int d, int m,
                             int nnz, Key key, int64_t row_offset, float *partials, float *Y, int *status,
                             const EventPair *ev, cudaStream_t stream);

// ---- adjoint (cg_adjoint.cu) --------------------------------------------------
cudaError_t launch_adjoint_w(const float *dY, int m, int d, int64_t B, Key key, float *W, const EventPair *ev,
                             cudaStream_t stream);
cudaError_t launch_gather_dense(const float *W, int n, int d, uint32_t B, Key key, int64_t row_offset, float *dX,
                                const EventPair *ev, cudaStream_t stream);
cudaError_t launch_gather_csr(const float *W, const int *row_ptr, const int *col_idx, int n, int d, uint32_t B,
                              int nnz, Key key, int64_t row_offset, float *dXv, int *status, const EventPair *ev,
                              cudaStream_t stream);
cudaError_t launch_gather_csr_i64(const float *W, const long long *row_ptr, const int *col_idx, int n, int d,
                                  uint32_t B, long long nnz, Key key, int64_t row_offset, float *dXv, int *status,
                                  const EventPair *ev, cudaStream_t stream);

// ---- generator dumps (cg_api.cu) ---------------------------------------------
cudaError_t launch_generate_words(Key key, uint32_t tag, uint64_t idx0, int64_t count, uint32_t *words,
                                  cudaStream_t stream);
cudaError_t launch_generate_hash_sign(Key key, uint32_t B, int64_t row0, int64_t count, int32_t *h, int32_t *sigma,
                                      cudaStream_t stream);
cudaError_t launch_generate_gaussian(Key key, uint32_t tag, int64_t R, int64_t r0, int64_t r1, int64_t c0,
                                     int64_t c1, float *out, cudaStream_t stream);

}  // namespace cg

// cg_sketch.cu -- stage 1 of the transform: SX = S.X, the O(nnz(X)) CountSketch
// scatter (Section 1.1, the O(nnz(X)) cost of S.X).
//
// Row i of X is added, times sigma(i), into row h(i) of SX (B x d, row-major fp32).
// The scatter is one pass over the CSR arrays: every byte of row_ptr, col_idx and
// vals is read once, with coalesced loads, and each nonzero becomes one fp32
// reduction (RED) into SX, which the caller sizes to stay resident in L2.  The
// bucket and sign of a row are recomputed from the Philox stream by the lane that
// owns the row and shared through shared memory; nothing random is stored.
#include "cg_internal.cuh"
#include "cg_scatter.cuh"

namespace cg {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kUnroll = 4;  // nonzeros in flight per lane

// One warp owns a chunk of consecutive rows at a time: ROWS rows staged in shared
// memory and swept nonzero by nonzero (scatter_chunk), or, with ROWS = 0, 32 rows of
// one lane each (scatter_lanes32).  Each nonzero becomes one reduction into SX (fp32;
// with FIXED, int64 fixed point).
// RP: the type of the row offsets (int, or long long for 2^31 nonzeros or more).
template <bool FIXED, int ROWS, typename RP = int>
__global__ void __launch_bounds__(kThreads)
sketch_csr_kernel(const RP *__restrict__ row_ptr, const int *__restrict__ col_idx, const float *__restrict__ vals,
                  int n, int d, uint32_t B, RP nnz, RP klo, Key key, int64_t row_offset, void *__restrict__ SX,
                  const int *__restrict__ maxbits, int *__restrict__ status, uint32_t blo, uint32_t bhi) {
    constexpr int CH = ROWS == 0 ? 32 : ROWS;
    __shared__ int s_rp[kWarps][ROWS == 0 ? 1 : ROWS + 1];
    __shared__ uint32_t s_h[kWarps][CH];
    __shared__ float s_sg[kWarps][CH];
    const int w = threadIdx.x >> 5;
    const int nchunks = (n + CH - 1) / CH;
    pdl_wait();  // SX may still be being zeroed by the kernel before this one
    const int F = FIXED ? fixed_point_exponent(*maxbits, static_cast<int>(nnz)) : 0;
    int bad = 0;
    for (int c = blockIdx.x * kWarps + w; c < nchunks; c += gridDim.x * kWarps) {
        if constexpr (ROWS == 0)
            scatter_lanes32<FIXED, false, RP>(row_ptr, col_idx, vals, c * CH, n, d, B, nnz, klo, key, row_offset, SX,
                                              F, bad, blo, bhi);
        else
            scatter_chunk<FIXED, ROWS, false, RP>(row_ptr, col_idx, vals, c * CH, n, d, B, nnz, klo, key, row_offset,
                                                  SX, F, s_rp[w], s_h[w], s_sg[w], bad, blo, bhi);
    }
    if (bad) atomicOr(status, kStatusBounds);
}

// Rows per warp chunk: `forced` (1 = one row per lane in chunks of 32, or 32, 64, 128
// rows staged in shared memory) or, for 0, the smallest staged height whose chunk holds
// about 96 nonzeros on average.
int chunk_rows(int n, int64_t nnz, int forced) {
    if (forced == 1 || forced == 32 || forced == 64 || forced == 128) return forced;
    const double per_row = n > 0 ? static_cast<double>(nnz) / n : 0.0;
    if (per_row * 32 >= 96.0) return 32;
    if (per_row * 64 >= 96.0) return 64;
    return 128;
}

int chunk_height(int rows) { return rows == 1 ? 32 : rows; }

template <bool FIXED, int ROWS, typename RP>
void launch_csr_rows_as(bool after_previous, int grid, cudaStream_t stream, const RP *row_ptr, const int *col_idx,
                        const float *vals, int n, int d, uint32_t B, RP nnz, RP klo, Key key, int64_t row_offset,
                        void *SX, const int *maxbits, int *status, uint32_t blo, uint32_t bhi) {
    if (after_previous)
        launch_after_previous(sketch_csr_kernel<FIXED, ROWS, RP>, dim3(grid), dim3(kThreads), 0, stream, row_ptr,
                              col_idx, vals, n, d, B, nnz, klo, key, row_offset, SX, maxbits, status, blo, bhi);
    else
        sketch_csr_kernel<FIXED, ROWS, RP><<<grid, kThreads, 0, stream>>>(row_ptr, col_idx, vals, n, d, B, nnz, klo,
                                                                          key, row_offset, SX, maxbits, status, blo,
                                                                          bhi);
}

// `after_previous`: the scatter is launched as a programmatic dependent of the kernel
// before it (which zeroes SX) and waits for it before its first reduction.
template <bool FIXED, typename RP = int>
void launch_csr_rows(int rows, int grid, cudaStream_t stream, const RP *row_ptr, const int *col_idx,
                     const float *vals, int n, int d, uint32_t B, RP nnz, RP klo, Key key, int64_t row_offset,
                     void *SX, const int *maxbits, int *status, uint32_t blo, uint32_t bhi,
                     bool after_previous = false) {
    if (rows == 1)
        launch_csr_rows_as<FIXED, 0, RP>(after_previous, grid, stream, row_ptr, col_idx, vals, n, d, B, nnz, klo, key,
                                         row_offset, SX, maxbits, status, blo, bhi);
    else if (rows == 128)
        launch_csr_rows_as<FIXED, 128, RP>(after_previous, grid, stream, row_ptr, col_idx, vals, n, d, B, nnz, klo,
                                           key, row_offset, SX, maxbits, status, blo, bhi);
    else if (rows == 64)
        launch_csr_rows_as<FIXED, 64, RP>(after_previous, grid, stream, row_ptr, col_idx, vals, n, d, B, nnz, klo,
                                          key, row_offset, SX, maxbits, status, blo, bhi);
    else
        launch_csr_rows_as<FIXED, 32, RP>(after_previous, grid, stream, row_ptr, col_idx, vals, n, d, B, nnz, klo,
                                          key, row_offset, SX, maxbits, status, blo, bhi);
}

// Zero fill for a small SX ahead of the scatter.  A kernel rather than a memset, so that
// the scatter can be launched as its programmatic dependent: the gap between two
// launches is a visible share of a call that takes a few microseconds.  Values before
// the first 16-byte boundary and after the last one are stored one by one.
constexpr size_t kZeroKernelMaxBytes = size_t(8) << 20;

__global__ void __launch_bounds__(kThreads) zero_fill_kernel(float *__restrict__ p, int64_t count) {
    asm volatile("griddepcontrol.launch_dependents;");
    const uint32_t mis = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p) & 15u);
    int64_t head = mis ? static_cast<int64_t>((16u - mis) >> 2) : 0;
    head = head < count ? head : count;
    const int64_t body = (count - head) >> 2;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
    float4 *v = reinterpret_cast<float4 *>(p + head);
    for (int64_t i = tid; i < body; i += stride) v[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const int64_t rest = head + 4 * body;
    if (tid < head) p[tid] = 0.0f;
    if (tid < count - rest) p[rest + tid] = 0.0f;
}

// max |x| over the stored values, as the bit pattern of a non-negative float (whose
// integer order is its numeric order) combined with atomicMax.  The values up to the
// first 16-byte boundary and past the last one are read one by one, the rest as float4
// with four loads in flight per thread.
__device__ __forceinline__ bool is_finite_bits(float v) { return (__float_as_uint(v) & 0x7F800000u) != 0x7F800000u; }

// max of mx and |v| over finite v; a non-finite v sets `special` instead.
__device__ __forceinline__ float finite_abs_max(float mx, float v, bool &special) {
    if (!is_finite_bits(v)) {
        special = true;
        return mx;
    }
    return fmaxf(mx, fabsf(v));
}

__global__ void __launch_bounds__(kThreads)
absmax_kernel(const float *__restrict__ x, int64_t count, int *__restrict__ maxbits) {
    float mx = 0.0f;
    bool sp = false;  // a NaN or an infinity seen
    const int64_t tid = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x;
    const int64_t nthreads = static_cast<int64_t>(gridDim.x) * kThreads;
    const int64_t lead = static_cast<int64_t>(((16 - (reinterpret_cast<uintptr_t>(x) & 15)) & 15) / 4);
    const int64_t head = lead < count ? lead : count;
    const int64_t quads = (count - head) / 4;
    const int64_t tail0 = head + 4 * quads;
    if (tid < head) mx = finite_abs_max(mx, __ldg(x + tid), sp);
    if (tail0 + tid < count) mx = finite_abs_max(mx, __ldg(x + tail0 + tid), sp);
    const float4 *q = reinterpret_cast<const float4 *>(x + head);
    int64_t i = tid;
    for (; i + 3 * nthreads < quads; i += 4 * nthreads) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldg(q + i + u * nthreads);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            mx = finite_abs_max(finite_abs_max(finite_abs_max(finite_abs_max(mx, v[u].x, sp), v[u].y, sp), v[u].z, sp),
                                v[u].w, sp);
    }
    for (; i < quads; i += nthreads) {
        const float4 v = __ldg(q + i);
        mx = finite_abs_max(finite_abs_max(finite_abs_max(finite_abs_max(mx, v.x, sp), v.y, sp), v.z, sp), v.w, sp);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0f) atomicMax(maxbits, __float_as_int(mx));
    if (__any_sync(0xffffffffu, sp) && (threadIdx.x & 31) == 0) atomicOr(maxbits + 1, 1);
}

// The rule for NaN and infinite values, as IEEE addition applies it in the fp32 scatters:
// the fixed-point sums take finite values only (to_fixed maps the others to 0), so when
// the max-|x| pass saw any (maxbits[1] != 0) this pass adds every non-finite entry to its
// cell of the rounded SX.  Whatever the order, a cell that receives a NaN, or both +Inf
// and -Inf, becomes NaN, and one that receives infinities of one sign becomes that
// infinity, so the result stays run-to-run reproducible.  Each such entry finds its row by
// binary search over row_ptr; column indices out of range are skipped (the scatter
// reported them).
__global__ void __launch_bounds__(kThreads)
add_nonfinite_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col_idx, const float *__restrict__ vals,
                     int n, int d, uint32_t B, int nnz, Key key, int64_t row_offset, const int *__restrict__ maxbits,
                     float *__restrict__ SX) {
    if (maxbits[1] == 0) return;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < nnz; k += gridDim.x * kThreads) {
        const float v = __ldg(vals + k);
        if (is_finite_bits(v)) continue;
        const int j = __ldg(col_idx + k);
        if (static_cast<unsigned>(j) >= static_cast<unsigned>(d)) continue;
        int lo = 0, hi = n - 1;  // the last row i < n with row_ptr[i] <= k
        while (lo < hi) {
            const int mid = lo + (hi - lo + 1) / 2;
            if (__ldg(row_ptr + mid) <= k) lo = mid; else hi = mid - 1;
        }
        if (!(__ldg(row_ptr + lo) <= k && k < __ldg(row_ptr + lo + 1))) continue;  // malformed offsets
        uint32_t h;
        float sg;
        hash_sign(key, static_cast<uint64_t>(row_offset + lo), B, h, sg);
        atomicAdd(SX + static_cast<size_t>(h) * d + j, sg * v);
    }
}

// SX = (float)(acc 2^-F): one rounding of the exact fixed-point sums.
__global__ void __launch_bounds__(kThreads)
fixed_to_float_kernel(const unsigned long long *__restrict__ acc, int64_t count, const int *__restrict__ maxbits,
                      int nnz, float *__restrict__ SX) {
    const int F = fixed_point_exponent(*maxbits, nnz);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * kThreads)
        SX[i] = ldexpf(__ll2float_rn(static_cast<long long>(acc[i])), -F);
}

// Dense X (n x d, row stride ldx), d % 4 == 0, ldx % 4 == 0, X 16-byte aligned:
// a warp owns 32 rows at a time; lane l hashes row l; the 32 x d/4 float4 quads of
// the rows are swept in row-major order (coalesced when ldx == d) and each is one
// vector reduction into SX.
__global__ void __launch_bounds__(kThreads)
sketch_dense_vec4_kernel(const float *__restrict__ X, int64_t ldx, int n, int d, uint32_t B, Key key,
                         int64_t row_offset, float *__restrict__ SX) {
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int nchunks = (n + 31) >> 5;
    const int dq = d >> 2;
    for (int c = blockIdx.x * kWarps + w; c < nchunks; c += gridDim.x * kWarps) {
        const int first = c << 5;
        const int rows = min(32, n - first);
        uint32_t h = 0;
        float sg = 0.0f;
        if (lane < rows) hash_sign(key, static_cast<uint64_t>(row_offset + first + lane), B, h, sg);
        const int total = rows * dq;
        for (int e0 = 0; e0 < total; e0 += 32 * kUnroll) {
            float4 x[kUnroll];
            int rr[kUnroll], qq[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int e = e0 + u * 32 + lane;
                rr[u] = e / dq;
                qq[u] = e - rr[u] * dq;
                x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (e < total)
                    x[u] = __ldg(reinterpret_cast<const float4 *>(X + (first + rr[u]) * ldx) + qq[u]);
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int e = e0 + u * 32 + lane;
                const int src = min(rr[u], 31);
                const uint32_t hh = __shfl_sync(0xffffffffu, h, src);
                const float s = __shfl_sync(0xffffffffu, sg, src);
                if (e < total) {
                    float4 val = make_float4(s * x[u].x, s * x[u].y, s * x[u].z, s * x[u].w);
                    atomicAdd(reinterpret_cast<float4 *>(SX + static_cast<size_t>(hh) * d) + qq[u], val);
                }
            }
        }
    }
}

// Dense X, any d and stride: scalar reductions.
__global__ void __launch_bounds__(kThreads)
sketch_dense_scalar_kernel(const float *__restrict__ X, int64_t ldx, int n, int d, uint32_t B, Key key,
                           int64_t row_offset, float *__restrict__ SX) {
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int nchunks = (n + 31) >> 5;
    for (int c = blockIdx.x * kWarps + w; c < nchunks; c += gridDim.x * kWarps) {
        const int first = c << 5;
        const int rows = min(32, n - first);
        uint32_t h = 0;
        float sg = 0.0f;
        if (lane < rows) hash_sign(key, static_cast<uint64_t>(row_offset + first + lane), B, h, sg);
        const int64_t total = static_cast<int64_t>(rows) * d;
        for (int64_t e0 = 0; e0 < total; e0 += 32) {
            const int64_t e = e0 + lane;
            const int r = static_cast<int>(e / d < 31 ? e / d : 31);
            const uint32_t hh = __shfl_sync(0xffffffffu, h, r);
            const float s = __shfl_sync(0xffffffffu, sg, r);
            if (e < total) {
                const int j = static_cast<int>(e - static_cast<int64_t>(r) * d);
                atomicAdd(SX + static_cast<size_t>(hh) * d + j, s * __ldg(X + (first + r) * ldx + j));
            }
        }
    }
}

}  // namespace

int sketch_default_ctas() {
    const int sms = num_sms();
    return (sms > 0 ? sms : 148) * (2048 / kThreads);
}

namespace {

template <typename RP>
cudaError_t sketch_csr_atomic(const RP *row_ptr, const int *col_idx, const float *vals, int n, int d, uint32_t B,
                              RP nnz, Key key, int64_t row_offset, float *SX, int *status, int ctas, int passes,
                              int rows, const EventPair *ev, cudaStream_t stream, bool clear) {
    const size_t bytes = static_cast<size_t>(B) * d * sizeof(float);
    // A small SX is zeroed by a kernel that the scatter follows as a programmatic
    // dependent (not when the scatter alone is timed between events).
    const bool zero_kernel = clear && n > 0 && bytes > 0 && bytes <= kZeroKernelMaxBytes && ev == nullptr;
    cudaError_t e = cudaSuccess;
    if (zero_kernel) {
        const int64_t count = static_cast<int64_t>(bytes / sizeof(float));
        const int64_t need4 = (count / 4 + kThreads - 1) / kThreads;
        const int sms = num_sms();
        const int64_t cap = static_cast<int64_t>(sms > 0 ? sms : 148) * 2;
        const int zgrid = static_cast<int>(need4 < 1 ? 1 : (need4 < cap ? need4 : cap));
        zero_fill_kernel<<<zgrid, kThreads, 0, stream>>>(SX, count);
        e = cudaGetLastError();
    } else if (clear) {
        e = cudaMemsetAsync(SX, 0, bytes, stream);
    }
    if (e != cudaSuccess || n == 0) return e;
    rows = chunk_rows(n, nnz, rows);
    const int nchunks = (n + chunk_height(rows) - 1) / chunk_height(rows);
    const int need = (nchunks + kWarps - 1) / kWarps;
    const int grid = max(1, min(ctas > 0 ? ctas : sketch_default_ctas(), need));
    record(ev, true, stream);
    // Optionally the buckets are reduced in ranges, one pass over the CSR per range, so
    // that each range's reductions stay in L2.  Automatic is one pass: on GB300 extra
    // passes cost more (every pass re-streams the CSR and re-hashes every row) than the
    // L2 misses they save, even with SX at 134 MB.
    if (passes <= 0) passes = 1;
    if (static_cast<uint32_t>(passes) > B) passes = B > 0 ? static_cast<int>(B) : 1;
    const uint32_t per = static_cast<uint32_t>((static_cast<uint64_t>(B) + passes - 1) / passes);
    for (int p = 0; p < passes; ++p) {
        const uint32_t blo = per * static_cast<uint32_t>(p);
        const uint32_t bhi = p == passes - 1 ? B : blo + per;
        launch_csr_rows<false, RP>(rows, grid, stream, row_ptr, col_idx, vals, n, d, B, nnz, RP(0), key, row_offset,
                                   SX, nullptr, status, blo, bhi, zero_kernel && p == 0);
    }
    record(ev, false, stream);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sketch_csr_atomic(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                     uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, int *status,
                                     int ctas, int passes, int rows, const EventPair *ev, cudaStream_t stream,
                                     bool clear) {
    return sketch_csr_atomic<int>(row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset, SX, status, ctas, passes,
                                  rows, ev, stream, clear);
}

cudaError_t launch_sketch_csr_atomic_i64(const long long *row_ptr, const int *col_idx, const float *vals, int n,
                                         int d, uint32_t B, long long nnz, Key key, int64_t row_offset, float *SX,
                                         int *status, int ctas, int passes, int rows, const EventPair *ev,
                                         cudaStream_t stream, bool clear) {
    return sketch_csr_atomic<long long>(row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset, SX, status, ctas,
                                        passes, rows, ev, stream, clear);
}

cudaError_t launch_sketch_csr_rows_chunk(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                         uint32_t B, int klo, int khi, Key key, int64_t row_offset, float *SX,
                                         int *status, int ctas, int rows, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    rows = chunk_rows(n, khi - klo, rows);
    const int nchunks = (n + chunk_height(rows) - 1) / chunk_height(rows);
    const int need = (nchunks + kWarps - 1) / kWarps;
    const int grid = max(1, min(ctas > 0 ? ctas : sketch_default_ctas(), need));
    launch_csr_rows<false>(rows, grid, stream, row_ptr, col_idx, vals, n, d, B, khi, klo, key, row_offset, SX, nullptr,
                           status, 0u, B);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const float *vals, int nnz, int *maxbits, cudaStream_t stream) {
    if (nnz <= 0) return cudaSuccess;
    const int sms = num_sms() > 0 ? num_sms() : 148;
    absmax_kernel<<<sms * (2048 / kThreads), kThreads, 0, stream>>>(vals, nnz, maxbits);
    return cudaGetLastError();
}

cudaError_t launch_add_nonfinite(const int *row_ptr, const int *col_idx, const float *vals, int n, int d, uint32_t B,
                                 int nnz, Key key, int64_t row_offset, const int *maxbits, float *SX,
                                 cudaStream_t stream) {
    if (nnz <= 0 || n <= 0) return cudaSuccess;
    const int sms = num_sms() > 0 ? num_sms() : 148;
    add_nonfinite_kernel<<<sms * 2, kThreads, 0, stream>>>(row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset,
                                                           maxbits, SX);
    return cudaGetLastError();
}

size_t sketch_fixed_scratch_bytes(int64_t B, int d) {
    return 256 + static_cast<size_t>(B) * d * sizeof(unsigned long long);
}

cudaError_t launch_sketch_csr_fixed(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                    uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, void *scratch,
                                    int *status, int ctas, int rows, const EventPair *ev, cudaStream_t stream) {
    int *maxbits = static_cast<int *>(scratch);
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + 256);
    const int64_t cells = static_cast<int64_t>(B) * d;
    cudaError_t e = cudaMemsetAsync(scratch, 0, sketch_fixed_scratch_bytes(B, d), stream);
    if (e != cudaSuccess) return e;
    const int sms = num_sms() > 0 ? num_sms() : 148;
    record(ev, true, stream);
    if (nnz > 0) absmax_kernel<<<sms * (2048 / kThreads), kThreads, 0, stream>>>(vals, nnz, maxbits);
    if (n > 0) {
        rows = chunk_rows(n, nnz, rows);
        const int nchunks = (n + chunk_height(rows) - 1) / chunk_height(rows);
        const int need = (nchunks + kWarps - 1) / kWarps;
        const int grid = max(1, min(ctas > 0 ? ctas : sketch_default_ctas(), need));
        launch_csr_rows<true>(rows, grid, stream, row_ptr, col_idx, vals, n, d, B, nnz, 0, key, row_offset, acc,
                              maxbits, status, 0u, B);
    }
    const int64_t blocks = (cells + kThreads - 1) / kThreads;
    fixed_to_float_kernel<<<static_cast<unsigned>(blocks < sms * 8 ? (blocks > 0 ? blocks : 1) : sms * 8), kThreads, 0,
                            stream>>>(acc, cells, maxbits, nnz, SX);
    if (nnz > 0 && n > 0)
        add_nonfinite_kernel<<<sms * 2, kThreads, 0, stream>>>(row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset,
                                                               maxbits, SX);
    record(ev, false, stream);
    return cudaGetLastError();
}

cudaError_t launch_sketch_dense_atomic(const float *X, int64_t ldx, int n, int d, uint32_t B, Key key,
                                       int64_t row_offset, float *SX, int *status, int ctas, const EventPair *ev,
                                       cudaStream_t stream, bool clear) {
    (void)status;
    cudaError_t e = clear ? cudaMemsetAsync(SX, 0, static_cast<size_t>(B) * d * sizeof(float), stream) : cudaSuccess;
    if (e != cudaSuccess || n == 0) return e;
    const int nchunks = (n + 31) / 32;
    const int need = (nchunks + kWarps - 1) / kWarps;
    const int grid = max(1, min(ctas > 0 ? ctas : sketch_default_ctas(), need));
    const bool vec = (d % 4 == 0) && (ldx % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    record(ev, true, stream);
    if (vec)
        sketch_dense_vec4_kernel<<<grid, kThreads, 0, stream>>>(X, ldx, n, d, B, key, row_offset, SX);
    else
        sketch_dense_scalar_kernel<<<grid, kThreads, 0, stream>>>(X, ldx, n, d, B, key, row_offset, SX);
    record(ev, false, stream);
    return cudaGetLastError();
}

}  // namespace cg

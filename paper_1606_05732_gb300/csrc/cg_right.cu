// cg_right.cu -- the scatter of the right projection Z = A.T^T (the random projection
// X.R, R = T^T, of the SVM application, Section 9; Table 1 times it).  A is a rows x n
// CSR matrix with one row per sample and one column per feature.  Column c of T is
// sigma(c) G[:, h(c)], so A.T^T = (G.(S.A^T))^T: the nonzero A[r, c] is reduced into
// SX[h(c), r] of a B x rows sketch, and the contraction of the left transform, stored
// transposed, gives Z.  The hash and sign belong to the column index here, so they are
// drawn per nonzero, or looked up in a table of per-column codes when the columns
// repeat often enough to pay for it.
#include <algorithm>

#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr int kRightThreads = 256;
constexpr int kRightPer = 4;                     // nonzeros per lane
constexpr int kRightChunk = 32 * kRightPer;      // consecutive nonzeros per warp task
constexpr uint32_t kSignBit = 0x80000000u;

// The table of column codes pays when the nonzeros hash each column more than this
// many times on average (a code costs one Philox call; a lookup, one cached load).
constexpr int64_t kTableRepeats = 4;

bool uses_table(int64_t n, int64_t nnz) { return n > 0 && nnz > kTableRepeats * n; }

// code(c) = h(c) | (sign bit if sigma(c) = -1), for the n columns of A (B < 2^31, so
// h leaves the top bit free).
__global__ void __launch_bounds__(kRightThreads)
column_codes_kernel(Key key, int64_t col_offset, int n, uint32_t B, uint32_t *__restrict__ codes) {
    for (int64_t c = static_cast<int64_t>(blockIdx.x) * kRightThreads + threadIdx.x; c < n;
         c += static_cast<int64_t>(gridDim.x) * kRightThreads) {
        uint32_t h;
        float s;
        hash_sign(key, static_cast<uint64_t>(col_offset + c), B, h, s);
        codes[c] = h | (s < 0.0f ? kSignBit : 0u);
    }
}

// Row offsets of up to this many rows are staged in shared memory by every CTA (one
// coalesced read), so that finding the row of a nonzero costs no global round trips.
constexpr int kSmemRows = 4095;

// The row r >= r0 with rp[r] <= k < rp[r + 1], given rp[r0] <= k < rp[rows]: the next
// offset first (long rows), else a binary search over the rest.  rp is the shared copy
// of the row offsets or row_ptr itself.
__device__ __forceinline__ int row_of(const int *rp, int r0, int rows, int k) {
    if (rp[r0 + 1] > k) return r0;
    int lo = r0 + 1, hi = rows;  // rp[lo] <= k < rp[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rp[mid] <= k)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Each warp takes 128 consecutive nonzeros [base, base + 128) of A (lane l the ones at
// base + l + 32 u, so that the column / value loads are coalesced), draws or looks up
// their columns' buckets and signs (four independent chains per lane), finds their
// rows, and reduces sigma(c) A[r, c] into SX[h(c), r].  Offsets that are out of range or
// out of order, and column indices outside [0, n), are skipped and reported.  With
// SMEM_ROWS (rows <= kSmemRows) the row offsets are read from a shared copy.
template <bool TABLE, bool SMEM_ROWS>
__global__ void __launch_bounds__(kRightThreads)
right_scatter_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col_idx, const float *__restrict__ vals,
                     int rows, int n, uint32_t B, int nnz, Key key, int64_t col_offset,
                     const uint32_t *__restrict__ codes, float *__restrict__ SX, int *status) {
    __shared__ int s_rp[SMEM_ROWS ? kSmemRows + 1 : 1];
    const int *rp = row_ptr;
    if (SMEM_ROWS) {
        for (int t = threadIdx.x; t <= rows; t += kRightThreads) s_rp[t] = __ldg(row_ptr + t);
        __syncthreads();
        rp = s_rp;
    }
    const int kbeg = rp[0], kend = rp[rows];
    int bad = 0;
    for (int t = blockIdx.x * kRightThreads + threadIdx.x; t < rows; t += gridDim.x * kRightThreads)
        if (rp[t] > rp[t + 1]) bad = 1;
    if (kbeg < 0 || kend > nnz || kbeg > kend) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusBounds);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (static_cast<int64_t>(blockIdx.x) * kRightThreads + threadIdx.x) >> 5;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (kRightThreads / 32);
    for (int64_t base = kbeg + warp0 * kRightChunk; base < kend; base += nwarps * kRightChunk) {
        int col[kRightPer];
        float v[kRightPer];
#pragma unroll
        for (int u = 0; u < kRightPer; ++u) {
            const int64_t k = base + u * 32 + lane;
            col[u] = -1;
            v[u] = 0.0f;
            if (k < kend) {
                col[u] = __ldg(col_idx + k);
                v[u] = __ldg(vals + k);
            }
        }
        uint32_t h[kRightPer];
        float s[kRightPer];
#pragma unroll
        for (int u = 0; u < kRightPer; ++u) {
            h[u] = 0;
            s[u] = 0.0f;
            const int c = col[u];
            if (static_cast<unsigned>(c) < static_cast<unsigned>(n)) {
                if (TABLE) {
                    const uint32_t code = __ldg(codes + c);
                    h[u] = code & ~kSignBit;
                    s[u] = (code & kSignBit) ? -1.0f : 1.0f;
                } else {
                    hash_sign(key, static_cast<uint64_t>(col_offset + c), B, h[u], s[u]);
                }
            } else if (base + u * 32 + lane < kend) {
                bad = 1;
            }
        }
        int r = 0;
#pragma unroll
        for (int u = 0; u < kRightPer; ++u) {
            const int64_t k = base + u * 32 + lane;
            if (k >= kend) break;
            r = row_of(rp, r, rows, static_cast<int>(k));
            if (s[u] != 0.0f) atomicAdd(SX + static_cast<size_t>(h[u]) * rows + r, s[u] * v[u]);
        }
    }
    if (bad) atomicOr(status, kStatusBounds);
}

}  // namespace

size_t right_scratch_bytes(int64_t n, int64_t nnz) {
    return uses_table(n, nnz) ? static_cast<size_t>(n) * sizeof(uint32_t) : 0;
}

cudaError_t launch_right_scatter(const int *row_ptr, const int *col_idx, const float *vals, int rows, int64_t n,
                                 uint32_t B, int nnz, Key key, int64_t col_offset, void *scratch, float *SX,
                                 int *status, const EventPair *ev, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(SX, 0, static_cast<size_t>(B) * rows * sizeof(float), stream);
    if (e != cudaSuccess) return e;
    const int sms = num_sms() > 0 ? num_sms() : 148;
    const int64_t cap = static_cast<int64_t>(sms) * 8;
    const bool table = uses_table(n, nnz);
    uint32_t *codes = static_cast<uint32_t *>(scratch);
    if (table) {
        const int64_t g = std::min<int64_t>(cap, (n + kRightThreads - 1) / kRightThreads);
        column_codes_kernel<<<static_cast<unsigned>(g), kRightThreads, 0, stream>>>(key, col_offset,
                                                                                    static_cast<int>(n), B, codes);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t tasks = (static_cast<int64_t>(nnz) + kRightChunk - 1) / kRightChunk;
    const int64_t per_cta = kRightThreads / 32;
    const int64_t need = std::max<int64_t>((tasks + per_cta - 1) / per_cta, (rows + kRightThreads - 1) / kRightThreads);
    const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(cap, need)));
    record(ev, true, stream);
    const uint32_t *cp = table ? codes : nullptr;
    const int nn = static_cast<int>(n);
    if (rows <= kSmemRows) {
        if (table)
            right_scatter_kernel<true, true><<<grid, kRightThreads, 0, stream>>>(row_ptr, col_idx, vals, rows, nn, B,
                                                                              nnz, key, col_offset, cp, SX, status);
        else
            right_scatter_kernel<false, true><<<grid, kRightThreads, 0, stream>>>(row_ptr, col_idx, vals, rows, nn, B,
                                                                               nnz, key, col_offset, cp, SX, status);
    } else if (table) {
        right_scatter_kernel<true, false><<<grid, kRightThreads, 0, stream>>>(row_ptr, col_idx, vals, rows, nn, B,
                                                                           nnz, key, col_offset, cp, SX, status);
    } else {
        right_scatter_kernel<false, false><<<grid, kRightThreads, 0, stream>>>(row_ptr, col_idx, vals, rows, nn, B,
                                                                            nnz, key, col_offset, cp, SX, status);
    }
    record(ev, false, stream);
    return cudaGetLastError();
}

}  // namespace cg

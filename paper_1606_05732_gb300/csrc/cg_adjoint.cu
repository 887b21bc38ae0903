// cg_adjoint.cu -- the adjoint of the transform.  T = G.S is linear (Section 1.1),
// so the gradient of <T.X, dY> with respect to X is T^T.dY = S^T.(G^T.dY):
//   W  = G^T.dY            (B x d; G regenerated from the seed, never stored)
//   dX = S^T.W             dense:  dX[i, :] = sigma(i) W[h(i), :]
//                          CSR:    dX_k     = sigma(i) W[h(i), col_idx[k]] for the
//                                  stored entries k of row i (the gradient with
//                                  respect to the stored values).
#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBB = 64;  // columns b of G per CTA
constexpr int kKR = 32;  // rows r of G per step

// CTA (bt, bn): W[b0 .. b0+64, n0 .. n0+BN) = sum over r of G[r, b] dY[r, j].
// Thread (ti, tj) owns b in [b0 + 4 ti, b0 + 4 ti + 4) and j in [n0 + TN tj, +TN).
template <int TN>
__global__ void __launch_bounds__(kThreads)
adjoint_w_kernel(const float *__restrict__ dY, int m, int d, int64_t B, Key key, float *__restrict__ W) {
    constexpr int BN = 16 * TN;
    __shared__ __align__(16) float sG[kKR][kBB];
    __shared__ __align__(16) float sY[kKR][BN];
    const int64_t b0 = static_cast<int64_t>(blockIdx.x) * kBB;
    const int n0 = blockIdx.y * BN;
    const int bn = min(BN, d - n0);
    const int t = threadIdx.x;
    const int ti = t & 15;
    const int tj = t >> 4;
    const uint64_t groups = static_cast<uint64_t>((m + 3) >> 2);

    float acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;

    for (int r0 = 0; r0 < m; r0 += kKR) {
        // G[r0 .. r0+32, b0 .. b0+64): 8 quads of rows x 64 columns.
        for (int q = t; q < (kKR / 4) * kBB; q += kThreads) {
            const int bl = q % kBB;
            const int gl = q / kBB;
            const int64_t b = b0 + bl;
            const uint64_t g = static_cast<uint64_t>(r0 / 4 + gl);
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (b < B && g < groups) z = gauss_quad(key, kTagG, groups, static_cast<uint64_t>(b), g);
            const int rr = 4 * gl;
            sG[rr + 0][bl] = (r0 + rr + 0 < m) ? z.x : 0.0f;
            sG[rr + 1][bl] = (r0 + rr + 1 < m) ? z.y : 0.0f;
            sG[rr + 2][bl] = (r0 + rr + 2 < m) ? z.z : 0.0f;
            sG[rr + 3][bl] = (r0 + rr + 3 < m) ? z.w : 0.0f;
        }
        for (int q = t; q < kKR * BN; q += kThreads) {
            const int rr = q / BN;
            const int cc = q % BN;
            sY[rr][cc] = (r0 + rr < m && cc < bn) ? __ldg(dY + static_cast<size_t>(r0 + rr) * d + n0 + cc) : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kKR; ++rr) {
            const float4 a = *reinterpret_cast<const float4 *>(&sG[rr][4 * ti]);
            float bv[TN];
#pragma unroll
            for (int j4 = 0; j4 < TN / 4; ++j4) {
                const float4 x = *reinterpret_cast<const float4 *>(&sY[rr][TN * tj + 4 * j4]);
                bv[4 * j4 + 0] = x.x;
                bv[4 * j4 + 1] = x.y;
                bv[4 * j4 + 2] = x.z;
                bv[4 * j4 + 3] = x.w;
            }
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                acc[0][j] = fmaf(a.x, bv[j], acc[0][j]);
                acc[1][j] = fmaf(a.y, bv[j], acc[1][j]);
                acc[2][j] = fmaf(a.z, bv[j], acc[2][j]);
                acc[3][j] = fmaf(a.w, bv[j], acc[3][j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t b = b0 + 4 * ti + i;
        if (b >= B) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = TN * tj + j;
            if (c < bn) W[b * d + n0 + c] = acc[i][j];
        }
    }
}

// dX[i, :] = sigma(i) W[h(i), :] for dense dX (n x d, contiguous).  The vector path keeps
// kGatherUnroll reads of W (L2-resident) in flight per lane before their stores, which
// are streaming (dX is written once and not read back by this kernel).
constexpr int kGatherUnroll = 4;

__global__ void __launch_bounds__(kThreads)
gather_dense_kernel(const float *__restrict__ W, int n, int d, uint32_t B, Key key, int64_t row_offset,
                    bool vec, float *__restrict__ dX) {
    pdl_wait();  // W comes from the kernel launched before
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int nchunks = (n + 31) >> 5;
    for (int c = blockIdx.x * kWarps + w; c < nchunks; c += gridDim.x * kWarps) {
        const int first = c << 5;
        const int rows = min(32, n - first);
        uint32_t h = 0;
        float sg = 0.0f;
        if (lane < rows) hash_sign(key, static_cast<uint64_t>(row_offset + first + lane), B, h, sg);
        if (vec) {
            const int dq = d >> 2;
            const int total = rows * dq;
            for (int e0 = 0; e0 < total; e0 += 32 * kGatherUnroll) {
                float4 x[kGatherUnroll];
                float s[kGatherUnroll];
                int r[kGatherUnroll], q[kGatherUnroll];
#pragma unroll
                for (int u = 0; u < kGatherUnroll; ++u) {
                    const int e = e0 + u * 32 + lane;
                    r[u] = min(e / dq, 31);
                    q[u] = e - r[u] * dq;
                    const uint32_t hh = __shfl_sync(0xffffffffu, h, r[u]);
                    s[u] = __shfl_sync(0xffffffffu, sg, r[u]);
                    x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (e < total) x[u] = __ldg(reinterpret_cast<const float4 *>(W + static_cast<size_t>(hh) * d) + q[u]);
                }
#pragma unroll
                for (int u = 0; u < kGatherUnroll; ++u) {
                    if (e0 + u * 32 + lane < total)
                        __stcs(reinterpret_cast<float4 *>(dX + static_cast<size_t>(first + r[u]) * d) + q[u],
                               make_float4(s[u] * x[u].x, s[u] * x[u].y, s[u] * x[u].z, s[u] * x[u].w));
                }
            }
        } else {
            const int64_t total = static_cast<int64_t>(rows) * d;
            for (int64_t e0 = 0; e0 < total; e0 += 32) {
                const int64_t e = e0 + lane;
                const int r = static_cast<int>(e / d < 31 ? e / d : 31);
                const uint32_t hh = __shfl_sync(0xffffffffu, h, r);
                const float s = __shfl_sync(0xffffffffu, sg, r);
                if (e < total) {
                    const int j = static_cast<int>(e - static_cast<int64_t>(r) * d);
                    dX[static_cast<size_t>(first + r) * d + j] = s * __ldg(W + static_cast<size_t>(hh) * d + j);
                }
            }
        }
    }
}

// dX_k = sigma(i) W[h(i), col_idx[k]] for the stored entries of CSR rows.  RP is the
// type of the row offsets and nonzero indices: int, or long long for 2^31 nonzeros or more.
template <typename RP>
__global__ void __launch_bounds__(kThreads)
gather_csr_kernel(const float *__restrict__ W, const RP *__restrict__ row_ptr, const int *__restrict__ col_idx,
                  int n, int d, uint32_t B, RP nnz, Key key, int64_t row_offset, float *__restrict__ dXv,
                  int *__restrict__ status) {
    __shared__ RP s_rp[kWarps][33];
    pdl_wait();  // W comes from the kernel launched before
    __shared__ uint32_t s_h[kWarps][32];
    __shared__ float s_sg[kWarps][32];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int nchunks = (n + 31) >> 5;
    int bad = 0;
    for (int c = blockIdx.x * kWarps + w; c < nchunks; c += gridDim.x * kWarps) {
        const int first = c << 5;
        const int i = first + lane;
        const int last = min(first + 32, n);
        const RP end = __ldg(row_ptr + last);
        RP rp = end;
        uint32_t h = 0;
        float sg = 0.0f;
        if (i < n) {
            rp = __ldg(row_ptr + i);
            hash_sign(key, static_cast<uint64_t>(row_offset + i), B, h, sg);
        }
        s_rp[w][lane] = rp;
        s_h[w][lane] = h;
        s_sg[w][lane] = sg;
        __syncwarp();
        const RP beg = s_rp[w][0];
        if (beg < 0 || end > nnz || beg > end) {
            bad = 1;
            __syncwarp();
            continue;
        }
        for (RP k = beg + lane; k < end; k += 32) {
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (s_rp[w][lo + step] <= k) lo += step;
            const int j = __ldg(col_idx + k);
            if (static_cast<unsigned>(j) < static_cast<unsigned>(d))
                dXv[k] = s_sg[w][lo] * __ldg(W + static_cast<size_t>(s_h[w][lo]) * d + j);
            else
                bad = 1;
        }
        __syncwarp();
    }
    if (bad) atomicOr(status, kStatusBounds);
}

int gather_ctas() { return (num_sms() > 0 ? num_sms() : 148) * (2048 / kThreads); }

}  // namespace

cudaError_t launch_adjoint_w(const float *dY, int m, int d, int64_t B, Key key, float *W, const EventPair *ev,
                             cudaStream_t stream) {
    const int64_t gb = (B + kBB - 1) / kBB;
    record(ev, true, stream);
    if (d > 64) {
        adjoint_w_kernel<8><<<dim3(static_cast<unsigned>(gb), (d + 127) / 128), kThreads, 0, stream>>>(dY, m, d, B,
                                                                                                        key, W);
    } else {
        adjoint_w_kernel<4><<<dim3(static_cast<unsigned>(gb), (d + 63) / 64), kThreads, 0, stream>>>(dY, m, d, B,
                                                                                                      key, W);
    }
    record(ev, false, stream);
    return cudaGetLastError();
}

cudaError_t launch_gather_dense(const float *W, int n, int d, uint32_t B, Key key, int64_t row_offset, float *dX,
                                const EventPair *ev, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int nchunks = (n + 31) / 32;
    const int grid = max(1, min(gather_ctas(), (nchunks + kWarps - 1) / kWarps));
    const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(dX) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(W) & 15) == 0);
    record(ev, true, stream);
    const cudaError_t e = launch_after_previous(gather_dense_kernel, dim3(grid), dim3(kThreads), 0, stream, W, n, d, B,
                                                key, row_offset, vec, dX);
    if (e != cudaSuccess) return e;
    record(ev, false, stream);
    return cudaGetLastError();
}

namespace {

template <typename RP>
cudaError_t gather_csr(const float *W, const RP *row_ptr, const int *col_idx, int n, int d, uint32_t B, RP nnz,
                       Key key, int64_t row_offset, float *dXv, int *status, const EventPair *ev,
                       cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int nchunks = (n + 31) / 32;
    const int grid = max(1, min(gather_ctas(), (nchunks + kWarps - 1) / kWarps));
    record(ev, true, stream);
    const cudaError_t e = launch_after_previous(gather_csr_kernel<RP>, dim3(grid), dim3(kThreads), 0, stream, W,
                                                row_ptr, col_idx, n, d, B, nnz, key, row_offset, dXv, status);
    record(ev, false, stream);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

cudaError_t launch_gather_csr(const float *W, const int *row_ptr, const int *col_idx, int n, int d, uint32_t B,
                              int nnz, Key key, int64_t row_offset, float *dXv, int *status, const EventPair *ev,
                              cudaStream_t stream) {
    return gather_csr<int>(W, row_ptr, col_idx, n, d, B, nnz, key, row_offset, dXv, status, ev, stream);
}

cudaError_t launch_gather_csr_i64(const float *W, const long long *row_ptr, const int *col_idx, int n, int d,
                                  uint32_t B, long long nnz, Key key, int64_t row_offset, float *dXv, int *status,
                                  const EventPair *ev, cudaStream_t stream) {
    return gather_csr<long long>(W, row_ptr, col_idx, n, d, B, nnz, key, row_offset, dXv, status, ev, stream);
}

}  // namespace cg

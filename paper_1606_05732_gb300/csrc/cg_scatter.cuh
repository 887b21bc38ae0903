// cg_scatter.cuh -- one warp scatters 32 consecutive CSR rows into SX (the O(nnz)
// stage of Section 1.1), shared by the scatter kernel and the batched kernel.
#pragma once
#include "cg_internal.cuh"

namespace cg {

constexpr int kScatterUnroll = 4;  // nonzeros in flight per lane

// Rows [first, min(first + 32, n)) of a CSR matrix: lane l hashes row first + l and
// loads its row_ptr entry into the warp's shared arrays s_rp[33], s_h[32], s_sg[32];
// the rows' nonzeros [beg, end) are swept 32 x kScatterUnroll at a time with coalesced
// loads, each nonzero finds its row by a 5-step binary search over s_rp and becomes
// one fp32 reduction SX[h, j] += sigma x.  Out-of-range column indices and malformed
// row offsets are skipped and reported through `bad`.
__device__ __forceinline__ void scatter_chunk32(const int *__restrict__ row_ptr, const int *__restrict__ col_idx,
                                                const float *__restrict__ vals, int first, int n, int d, uint32_t B,
                                                int nnz, Key key, int64_t row_offset, float *__restrict__ SX,
                                                int *s_rp, uint32_t *s_h, float *s_sg, int &bad) {
    const int lane = threadIdx.x & 31;
    const int i = first + lane;
    const int last = min(first + 32, n);
    const int end = __ldg(row_ptr + last);
    int rp = end;
    uint32_t h = 0;
    float sg = 0.0f;
    if (i < n) {
        rp = __ldg(row_ptr + i);
        hash_sign(key, static_cast<uint64_t>(row_offset + i), B, h, sg);
    }
    s_rp[lane] = rp;
    s_h[lane] = h;
    s_sg[lane] = sg;
    if (lane == 0) s_rp[32] = end;
    __syncwarp();
    const int beg = s_rp[0];
    if (beg < 0 || end > nnz || beg > end) {  // malformed row_ptr: skip the chunk
        bad = 1;
        __syncwarp();
        return;
    }
    for (int k0 = beg; k0 < end; k0 += 32 * kScatterUnroll) {
        int col[kScatterUnroll];
        float v[kScatterUnroll];
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const int k = k0 + u * 32 + lane;
            col[u] = -1;
            v[u] = 0.0f;
            if (k < end) {
                col[u] = __ldg(col_idx + k);
                v[u] = __ldg(vals + k);
            }
        }
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const int k = k0 + u * 32 + lane;
            if (k < end) {
                int lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (s_rp[lo + step] <= k) lo += step;
                const int j = col[u];
                if (static_cast<unsigned>(j) < static_cast<unsigned>(d))
                    atomicAdd(SX + static_cast<size_t>(s_h[lo]) * d + j, s_sg[lo] * v[u]);
                else
                    bad = 1;
            }
        }
    }
    __syncwarp();
}

}  // namespace cg

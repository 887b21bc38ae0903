// cg_plain.cu -- the plain product Y = G~.X with an m x n Gaussian G~ (Abstract;
// Section 4: the O(nnz(X) m) computation that CountGauss replaces).
//
// G~ is never stored: column i of G~ (m normals, ceil(m/4) Philox calls) is drawn
// for every non-empty row i of X, and Y[:, j] += G~[:, i] X[i, j] for each stored
// entry of the row.  Columns of G~ for empty rows meet only zeros and are skipped.
// The work is the generation (Philox + log + sincos per two normals) plus
// m FMAs per nonzero, so the kernel is bound by ALU issue, not by memory.
//
// A CTA keeps its own m x d accumulator in shared memory (column-major, so that
// lanes holding consecutive rows r of one column j hit consecutive banks) and adds
// into it with shared-memory atomics; warps take chunks of 32 rows, draw the
// columns of up to P non-empty rows into a per-warp buffer, then sweep those rows'
// nonzeros.  Each CTA writes one m x d partial, summed in a fixed order afterwards.
#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSmemLimit = 200 * 1024;

inline int rows_per_pass(int m) { return max(1, min(32, 1024 / max(1, m))); }

inline size_t plain_smem_bytes(int m, int d) {
    const size_t acc = (static_cast<size_t>(m) * d + 3) & ~static_cast<size_t>(3);
    const size_t gbuf = static_cast<size_t>(kWarps) * rows_per_pass(m) * m;
    return (acc + gbuf) * sizeof(float) + kWarps * 32 * sizeof(int);
}

__global__ void __launch_bounds__(kThreads)
plain_csr_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col_idx, const float *__restrict__ vals,
                 int n, int d, int m, int nnz, Key key, int64_t row_offset, int P, float *__restrict__ part,
                 int *__restrict__ status) {
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int md = m * d;
    const int acc_floats = (md + 3) & ~3;
    float *Yacc = smem;  // [d][m]
    float *gbuf = smem + acc_floats + w * P * m;
    int *slot_lane = reinterpret_cast<int *>(smem + acc_floats + kWarps * P * m) + w * 32;
    for (int e = threadIdx.x; e < md; e += kThreads) Yacc[e] = 0.0f;
    __syncthreads();

    const int ngroups = (m + 3) >> 2;
    const int nchunks = (n + 31) >> 5;
    int bad = 0;
    for (int c = blockIdx.x * kWarps + w; c < nchunks; c += gridDim.x * kWarps) {
        const int i = (c << 5) + lane;
        int rp0 = 0, rp1 = 0;
        if (i < n) {
            rp0 = __ldg(row_ptr + i);
            rp1 = __ldg(row_ptr + i + 1);
            if (rp0 < 0 || rp1 > nnz || rp0 > rp1) {  // malformed row_ptr: skip the row
                bad = 1;
                rp0 = rp1 = 0;
            }
        }
        unsigned pending = __ballot_sync(0xffffffffu, rp1 > rp0);
        while (pending) {
            unsigned take = 0, rest = pending;
            for (int q = 0; q < P && rest; ++q) {
                const unsigned low = rest & (0u - rest);
                take |= low;
                rest ^= low;
            }
            pending = rest;
            const int np = __popc(take);
            if ((take >> lane) & 1u) slot_lane[__popc(take & ((1u << lane) - 1u))] = lane;
            __syncwarp();
            // Columns of G~ for the np rows of this pass.
            for (int t = lane; t < np * ngroups; t += 32) {
                const int slot = t / ngroups;
                const int g = t - slot * ngroups;
                const int row = (c << 5) + slot_lane[slot];
                const float4 z = gauss_quad(key, kTagGTilde, static_cast<uint64_t>(ngroups),
                                            static_cast<uint64_t>(row_offset + row), static_cast<uint64_t>(g));
                float *dst = gbuf + slot * m + 4 * g;
                const int r0 = 4 * g;
                if (r0 + 0 < m) dst[0] = z.x;
                if (r0 + 1 < m) dst[1] = z.y;
                if (r0 + 2 < m) dst[2] = z.z;
                if (r0 + 3 < m) dst[3] = z.w;
            }
            __syncwarp();
            // Y[:, j] += G~[:, i] x for each stored (j, x) of the pass's rows.
            for (int slot = 0; slot < np; ++slot) {
                const int l = slot_lane[slot];
                const int kb = __shfl_sync(0xffffffffu, rp0, l);
                const int ke = __shfl_sync(0xffffffffu, rp1, l);
                const float *g = gbuf + slot * m;
                if (m >= 32) {
                    for (int k = kb; k < ke; ++k) {
                        const int j = __ldg(col_idx + k);
                        const float v = __ldg(vals + k);
                        if (static_cast<unsigned>(j) < static_cast<unsigned>(d)) {
                            float *col = Yacc + static_cast<size_t>(j) * m;
                            for (int r = lane; r < m; r += 32) atomicAdd(col + r, g[r] * v);
                        } else {
                            bad = 1;
                        }
                    }
                } else {
                    const int per = 32 / m;
                    const int sub = lane / m;
                    const int r = lane - sub * m;
                    for (int k0 = kb; k0 < ke; k0 += per) {
                        const int k = k0 + sub;
                        if (sub < per && k < ke) {
                            const int j = __ldg(col_idx + k);
                            const float v = __ldg(vals + k);
                            if (static_cast<unsigned>(j) < static_cast<unsigned>(d))
                                atomicAdd(Yacc + static_cast<size_t>(j) * m + r, g[r] * v);
                            else
                                bad = 1;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
    if (bad) atomicOr(status, kStatusBounds);
    __syncthreads();
    float *out = part + static_cast<size_t>(blockIdx.x) * md;
    for (int e = threadIdx.x; e < md; e += kThreads) {
        const int r = e / d;
        const int j = e - r * d;
        out[e] = Yacc[j * m + r];
    }
}

}  // namespace

bool plain_supported(int m, int d) { return plain_smem_bytes(m, d) <= static_cast<size_t>(kSmemLimit); }

int plain_ctas(int m, int d) {
    const int sms = num_sms() > 0 ? num_sms() : 148;
    const size_t per = plain_smem_bytes(m, d);
    int resident = static_cast<int>((227 * 1024) / (per + 1024));
    resident = max(1, min(resident, 2048 / kThreads));
    return sms * resident;
}

cudaError_t launch_plain_csr(const int *row_ptr, const int *col_idx, const float *vals, int n, int d, int m,
                             int nnz, Key key, int64_t row_offset, float *partials, float *Y, int *status,
                             const EventPair *ev, cudaStream_t stream) {
    const size_t smem = plain_smem_bytes(m, d);
    cudaError_t e = cudaFuncSetAttribute(plain_csr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int nchunks = (n + 31) / 32;
    const int grid = max(1, min(plain_ctas(m, d), (nchunks + kWarps - 1) / kWarps));
    record(ev, true, stream);
    plain_csr_kernel<<<grid, kThreads, smem, stream>>>(row_ptr, col_idx, vals, n, d, m, nnz, key, row_offset,
                                                       rows_per_pass(m), partials, status);
    record(ev, false, stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_splits(partials, grid, static_cast<int64_t>(m) * d, Y, stream);
}

}  // namespace cg

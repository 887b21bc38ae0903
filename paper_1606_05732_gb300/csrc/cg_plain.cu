// cg_plain.cu -- the plain product Y = G~.X with an m x n Gaussian G~ (Abstract;
// Section 4: the O(nnz(X) m) computation that CountGauss replaces).
//
// G~ is never stored: column i of G~ (m normals, ceil(m/4) Philox calls) is drawn
// for every non-empty row i of X, and Y[:, j] += G~[:, i] X[i, j] for each stored
// entry of the row.  Columns of G~ for empty rows meet only zeros and are skipped.
// The work is the generation (Philox + log + sincos per two normals) plus m
// multiply-adds per nonzero into an accumulator, so the kernel is bound by
// instruction issue, not by memory.
//
// A CTA keeps its own m x d accumulator in shared memory (column-major, so that lanes
// holding consecutive rows r of one column j hit consecutive banks) and adds into it
// with shared-memory atomics.  A warp takes chunks of 32 rows; per pass it takes the
// chunk's next (up to P) non-empty rows, draws their columns of G~ into a per-warp
// buffer (two independent Philox/Box-Muller chains per lane and step), then sweeps the
// pass's nonzeros -- contiguous in CSR order -- 32 at a time with coalesced loads,
// each lane finding its nonzero's row by binary search; each nonzero's m-wide update is
// broadcast to the lanes by shuffles.  The kernel is specialised for the common m (8,
// 16, 32, 64, 128) so that the per-nonzero loops have constant trip counts.  Each CTA
// writes one m x d partial, summed in a fixed order afterwards.  When m x d does not fit
// the shared memory, the kernel runs once per tile of rows of G~ (and of Y), each launch
// drawing only its own rows of G~ (no entry is drawn twice).
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
    return (acc + gbuf) * sizeof(float) + kWarps * 65 * sizeof(int);
}

// M > 0: the kernel for m == M, whose loops over the m rows of a column of G~ have
// compile-time trip counts; M == 0: any m.
template <int M>
__global__ void __launch_bounds__(kThreads, 4)  // at most 64 registers: four CTAs per SM
plain_csr_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col_idx, const float *__restrict__ vals,
                 int n, int d, int m_rt, int groups_total, int g_off, int nnz, Key key, int64_t row_offset, int P,
                 float *__restrict__ part, int *__restrict__ status) {
    extern __shared__ __align__(16) float smem[];
    const int m = M > 0 ? M : m_rt;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int md = m * d;
    const int acc_floats = (md + 3) & ~3;
    float *Yacc = smem;  // [d][m]
    float *gbuf = smem + acc_floats + w * P * m;
    int *slot_beg = reinterpret_cast<int *>(smem + acc_floats + kWarps * P * m) + w * 65;  // [33]
    int *slot_lane = slot_beg + 33;                                                          // [32]
    for (int e = threadIdx.x; e < md; e += kThreads) Yacc[e] = 0.0f;
    __syncthreads();

    const int ngroups = (m + 3) >> 2;
    const int nchunks = (n + 31) >> 5;
    // m < 32: `per` nonzeros per step, lanes [sub m, sub m + m) on nonzero sub
    const int per = m < 32 ? 32 / m : 1;
    const int sub = m < 32 ? lane / m : 0;
    const int rr = m < 32 ? lane - sub * m : lane;
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
            // the next (up to) P non-empty rows of the chunk, in order
            unsigned take = 0, rest = pending;
            for (int q = 0; q < P && rest; ++q) {
                const unsigned low = rest & (0u - rest);
                take |= low;
                rest ^= low;
            }
            pending = rest;
            const int np = __popc(take);
            const bool mine = (take >> lane) & 1u;
            const int my_slot = __popc(take & ((1u << lane) - 1u));
            if (mine) {
                slot_beg[my_slot] = rp0;
                slot_lane[my_slot] = lane;
            }
            // the rows' nonzeros are contiguous only when no non-empty row lies between
            // them, which holds because the rows taken are consecutive non-empty rows and
            // empty rows add no nonzeros; the pass ends where its last row ends
            const int last_lane = 31 - __clz(take);
            const int kend = __shfl_sync(0xffffffffu, rp1, last_lane);
            if (lane == 0) slot_beg[np] = kend;
            __syncwarp();
            // Columns of G~ for the np rows of this pass: two independent quads per step.
            const int nq = np * ngroups;
            for (int t0 = lane; t0 < nq; t0 += 64) {
                const int t1 = t0 + 32;
                const int s0 = t0 / ngroups, g0 = t0 - s0 * ngroups;
                const int s1 = t1 / ngroups, g1 = t1 - s1 * ngroups;
                const int row0 = (c << 5) + slot_lane[s0];
                const int row1 = (c << 5) + (t1 < nq ? slot_lane[s1] : 0);
                // rows 4 (g_off + g) .. of the m_total x n Gaussian (groups_total groups)
                const float4 z0 = gauss_quad(key, kTagGTilde, static_cast<uint64_t>(groups_total),
                                             static_cast<uint64_t>(row_offset + row0),
                                             static_cast<uint64_t>(g_off + g0));
                float4 z1 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (t1 < nq)
                    z1 = gauss_quad(key, kTagGTilde, static_cast<uint64_t>(groups_total),
                                    static_cast<uint64_t>(row_offset + row1), static_cast<uint64_t>(g_off + g1));
                float *d0 = gbuf + s0 * m + 4 * g0;
                if (4 * g0 + 0 < m) d0[0] = z0.x;
                if (4 * g0 + 1 < m) d0[1] = z0.y;
                if (4 * g0 + 2 < m) d0[2] = z0.z;
                if (4 * g0 + 3 < m) d0[3] = z0.w;
                if (t1 < nq) {
                    float *d1 = gbuf + s1 * m + 4 * g1;
                    if (4 * g1 + 0 < m) d1[0] = z1.x;
                    if (4 * g1 + 1 < m) d1[1] = z1.y;
                    if (4 * g1 + 2 < m) d1[2] = z1.z;
                    if (4 * g1 + 3 < m) d1[3] = z1.w;
                }
            }
            __syncwarp();
            // Y[:, j] += G~[:, i] x over the pass's nonzeros [kbeg, kend), 32 at a time:
            // lane l loads nonzero k0 + l (coalesced) and finds its slot; then each
            // nonzero's m-wide update is broadcast to the lanes by shuffles.
            const int kbeg = slot_beg[0];
            for (int k0 = kbeg; k0 < kend; k0 += 32) {
                const int k = k0 + lane;
                int j = -1, sl = 0;
                float v = 0.0f;
                if (k < kend) {
                    j = __ldg(col_idx + k);
                    v = __ldg(vals + k);
                    int lo = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (lo + step < np && slot_beg[lo + step] <= k) lo += step;
                    sl = lo;
                    if (static_cast<unsigned>(j) >= static_cast<unsigned>(d)) {
                        bad = 1;
                        j = -1;
                    }
                }
                const int cnt = min(32, kend - k0);
                if (M >= 32 && M % 32 == 0) {
                    for (int u = 0; u < cnt; ++u) {
                        const int ju = __shfl_sync(0xffffffffu, j, u);
                        const float vu = __shfl_sync(0xffffffffu, v, u);
                        const int su = __shfl_sync(0xffffffffu, sl, u);
                        if (ju < 0) continue;  // warp-uniform
                        float *col = Yacc + ju * M + lane;
                        const float *g = gbuf + su * M + lane;
#pragma unroll
                        for (int q = 0; q < M / 32; ++q) atomicAdd(col + 32 * q, g[32 * q] * vu);
                    }
                } else if (m >= 32) {
                    for (int u = 0; u < cnt; ++u) {
                        const int ju = __shfl_sync(0xffffffffu, j, u);
                        const float vu = __shfl_sync(0xffffffffu, v, u);
                        const int su = __shfl_sync(0xffffffffu, sl, u);
                        if (ju < 0) continue;  // warp-uniform
                        float *col = Yacc + ju * m;
                        const float *g = gbuf + su * m;
                        for (int r = lane; r < m; r += 32) atomicAdd(col + r, g[r] * vu);
                    }
                } else {
                    for (int u0 = 0; u0 < cnt; u0 += per) {
                        const int u = u0 + sub;
                        const int src = u < 32 ? u : 31;
                        const int ju = __shfl_sync(0xffffffffu, j, src);
                        const float vu = __shfl_sync(0xffffffffu, v, src);
                        const int su = __shfl_sync(0xffffffffu, sl, src);
                        if (sub < per && u < cnt && ju >= 0) atomicAdd(Yacc + ju * m + rr, gbuf[su * m + rr] * vu);
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

using PlainKernel = void (*)(const int *, const int *, const float *, int, int, int, int, int, int, Key, int64_t, int,
                            float *, int *);

PlainKernel plain_kernel_for(int m) {
    switch (m) {
        case 8: return plain_csr_kernel<8>;
        case 16: return plain_csr_kernel<16>;
        case 32: return plain_csr_kernel<32>;
        case 64: return plain_csr_kernel<64>;
        case 128: return plain_csr_kernel<128>;
        default: return plain_csr_kernel<0>;
    }
}

// Rows of G~ per launch: all m where the m x d accumulator fits, else the largest of
// 128, 64, 32, 16, 8, 4 that fits (0 if none does).
int plain_tile_rows(int m, int d) {
    if (plain_smem_bytes(m, d) <= static_cast<size_t>(kSmemLimit)) return m;
    for (int t : {128, 64, 32, 16, 8, 4})
        if (t < m && plain_smem_bytes(t, d) <= static_cast<size_t>(kSmemLimit)) return t;
    return 0;
}

}  // namespace

bool plain_supported(int m, int d) { return plain_tile_rows(m, d) > 0; }

size_t plain_partials_bytes(int m, int d) {
    const int mt = plain_tile_rows(m, d) > 0 ? plain_tile_rows(m, d) : m;
    return static_cast<size_t>(plain_ctas(m, d)) * mt * d * sizeof(float);
}

int plain_ctas(int m, int d) {
    m = plain_tile_rows(m, d) > 0 ? plain_tile_rows(m, d) : m;
    const int sms = num_sms() > 0 ? num_sms() : 148;
    const size_t per = plain_smem_bytes(m, d);
    int resident = static_cast<int>((227 * 1024) / (per + 1024));
    resident = max(1, min(resident, 2048 / kThreads));
    if (num_sms() > 0)  // registers may allow fewer (one full wave, no partial second one)
        resident = min(resident, resident_ctas_per_sm(reinterpret_cast<const void *>(plain_kernel_for(m)), kThreads,
                                                      per, 0));
    return sms * resident;
}

cudaError_t launch_plain_csr(const int *row_ptr, const int *col_idx, const float *vals, int n, int d, int m,
                             int nnz, Key key, int64_t row_offset, float *partials, float *Y, int *status,
                             const EventPair *ev, cudaStream_t stream) {
    const int mt = plain_tile_rows(m, d);
    if (mt <= 0) return cudaErrorInvalidValue;
    const int groups_total = (m + 3) / 4;
    const int nchunks = (n + 31) / 32;
    const int grid = max(1, min(plain_ctas(m, d), (nchunks + kWarps - 1) / kWarps));
    // one launch (and one split sum into rows q0 .. q0 + rows of Y) per tile of rows of G~
    for (int q0 = 0; q0 < m; q0 += mt) {
        const int rows = min(mt, m - q0);
        const size_t smem = plain_smem_bytes(rows, d);
        const PlainKernel kernel = plain_kernel_for(rows);
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        record(ev, q0 == 0, stream);
        kernel<<<grid, kThreads, smem, stream>>>(row_ptr, col_idx, vals, n, d, rows, groups_total, q0 / 4, nnz, key,
                                                 row_offset, rows_per_pass(rows), partials, status);
        if (q0 + mt >= m) record(ev, false, stream);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_reduce_splits(partials, grid, static_cast<int64_t>(rows) * d, Y + static_cast<size_t>(q0) * d, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cg

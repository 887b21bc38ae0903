// cg_scatter.cuh -- one warp scatters a chunk of consecutive CSR rows into SX (the O(nnz)
// stage of Section 1.1), shared by the scatter kernel and the batched kernel.
#pragma once
#include "cg_internal.cuh"

namespace cg {

constexpr int kScatterUnroll = 4;  // nonzeros in flight per lane

// L2 policy for data read exactly once (the CSR stream): evict it first, so that it
// does not push the sketch SX, which is reduced into over and over, out of L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ int ld_stream_i32(const int *p, uint64_t pol) {
    int v;
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ long long ld_stream_i64(const long long *p, uint64_t pol) {
    long long v;
    asm volatile("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    return v;
}

// Largest number of nonzeros in one warp chunk of a matrix with 64-bit row offsets: the
// chunk's offsets are taken relative to its first nonzero and swept in 32-bit integers.
constexpr long long kMaxChunkNnz = (1LL << 31) - (1LL << 20);

__device__ __forceinline__ float ld_stream_f32(const float *p, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

// Scale of the fixed-point sums: F = 62 - L - e with max|x| < 2^e and nnz < 2^L, so
// every term is below 2^(62-L) and no sum of nnz terms leaves the int64 range.  Each
// term is resolved to 2^-F = 2^(L+e-62) absolute (about 1e-11 of max|x| at nnz ~ 5e7).
__device__ __forceinline__ int fixed_point_exponent(int maxbits, int nnz) {
    const float mx = __int_as_float(maxbits);
    int e = 0;
    if (mx > 0.0f) frexpf(mx, &e);  // mx < 2^e
    const int L = nnz > 0 ? 32 - __clz(nnz) : 1;  // nnz < 2^L
    return 62 - L - e;
}

// Fixed-point image of v: round(v 2^F) as a two's-complement 64-bit integer, with
// integer operations only.  The caller picks F so that |v| 2^F < 2^62.
__device__ __forceinline__ unsigned long long to_fixed(float v, int F) {
    const uint32_t u = __float_as_uint(v);
    const int be = static_cast<int>((u >> 23) & 0xFFu);
    if (be == 0xFF) return 0ull;  // not finite: contributes nothing
    const uint32_t mant = (u & 0x7FFFFFu) | (be ? 0x800000u : 0u);
    const int sh = (be ? be : 1) - 150 + F;  // |v| = mant 2^(exp - 150), times 2^F
    long long q;
    if (sh >= 0)
        q = static_cast<long long>(mant) << (sh < 39 ? sh : 39);
    else if (sh > -25)
        q = static_cast<long long>((mant + (1u << (-sh - 1))) >> (-sh));  // round half up
    else
        q = 0;
    return static_cast<unsigned long long>((u >> 31) ? -q : q);
}

// Rows [first, min(first + ROWS, n)) of a CSR matrix (ROWS = 32, 64 or 128): lane l
// loads the row_ptr entries of rows first + l + 32 r and hashes those rows into the
// warp's shared arrays s_rp[ROWS + 1], s_h[ROWS], s_sg[ROWS]; the rows' nonzeros
// [beg, end) are swept 32 x kScatterUnroll at a time with coalesced evict-first loads,
// each nonzero finds its row by a log2(ROWS)-step binary search over s_rp and becomes
// one reduction into SX: fp32, or with FIXED the 64-bit integer to_fixed(x, F) into an
// integer SX (order-independent sums).  Taller chunks put more nonzeros behind each
// pair of dependent memory round trips (row_ptr, then the nonzeros), which is what
// very sparse rows need.  Row offsets index col_idx / vals from klo: nonzero k of the
// matrix is col_idx[k - klo] (klo = 0 for a whole matrix; the first nonzero of a chunk of
// rows copied on its own), and offsets outside [klo, nnz] or out of order are malformed.  Out-of-range
// column indices and malformed row offsets are skipped and reported through `bad`.  Only
// rows whose bucket lies in [blo, bhi) are reduced (bucket-range passes); blo = 0,
// bhi = B reduces every row.
// With SKIP_EMPTY, empty rows get no bucket and sign: a warp whose rows are all empty
// skips the hash (worth it for inputs with mostly empty rows).
// RP is the type of the row offsets, nnz and klo: int, or long long for matrices of 2^31
// nonzeros or more.  With long long the chunk's offsets are rebased to its first nonzero
// (col_idx / vals are then read from that nonzero on) and kept in 32-bit integers; a
// chunk of more than kMaxChunkNnz nonzeros is reported as malformed.
template <bool FIXED, int ROWS, bool SKIP_EMPTY = false, typename RP = int>
__device__ __forceinline__ void scatter_chunk(const RP *__restrict__ row_ptr, const int *__restrict__ col_idx,
                                              const float *__restrict__ vals, int first, int n, int d, uint32_t B,
                                              RP nnz_in, RP klo_in, Key key, int64_t row_offset,
                                              void *__restrict__ SX, int F, int *s_rp, uint32_t *s_h, float *s_sg,
                                              int &bad, uint32_t blo = 0u, uint32_t bhi = 0xFFFFFFFFu) {
    static_assert(ROWS == 32 || ROWS == 64 || ROWS == 128, "chunk height");
    constexpr int R = ROWS / 32;
    const int lane = threadIdx.x & 31;
    const uint64_t pol = l2_evict_first_policy();
    const int last = min(first + ROWS, n);
    int end, nnz, klo;
    int rp[R];
    bool malformed = false;
    if constexpr (sizeof(RP) == 4) {
        nnz = nnz_in;
        klo = klo_in;
        end = __ldg(row_ptr + last);
#pragma unroll
        for (int r = 0; r < R; ++r) {  // all row_ptr loads in flight before the hashing
            const int i = first + r * 32 + lane;
            rp[r] = i < n ? ld_stream_i32(row_ptr + i, pol) : end;
        }
    } else {
        const long long end64 = __ldg(row_ptr + last);
        long long rp64[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = first + r * 32 + lane;
            rp64[r] = i < n ? ld_stream_i64(row_ptr + i, pol) : end64;
        }
        const long long base = __shfl_sync(0xffffffffu, rp64[0], 0);  // row_ptr[first]
        malformed = base < klo_in || end64 > nnz_in || end64 < base || end64 - base > kMaxChunkNnz;
        const long long span = malformed ? 0 : end64 - base;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long rel = rp64[r] - base;
            rp[r] = rel >= 0 && rel <= span ? static_cast<int>(rel) : -1;  // -1 breaks the order check
            malformed |= rel < 0 || rel > span;
        }
        malformed = __any_sync(0xffffffffu, malformed);
        end = static_cast<int>(span);
        nnz = end;
        klo = 0;
        if (!malformed) {
            col_idx += base - klo_in;
            vals += base - klo_in;
        }
    }
    if (SKIP_EMPTY) {
#pragma unroll
        for (int r = 0; r < R; ++r) s_rp[r * 32 + lane] = rp[r];
        if (lane == 0) s_rp[ROWS] = end;
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = first + r * 32 + lane;
        uint32_t h = 0;
        float sg = 0.0f;
        if (i < n && (!SKIP_EMPTY || rp[r] < s_rp[r * 32 + lane + 1]))
            hash_sign(key, static_cast<uint64_t>(row_offset + i), B, h, sg);
        if (!SKIP_EMPTY) s_rp[r * 32 + lane] = rp[r];
        s_h[r * 32 + lane] = h;
        s_sg[r * 32 + lane] = sg;
    }
    if (!SKIP_EMPTY && lane == 0) s_rp[ROWS] = end;
    __syncwarp();
    const int beg = s_rp[0];
    bool ordered = true;
#pragma unroll
    for (int r = 0; r < R; ++r) ordered &= s_rp[r * 32 + lane] <= s_rp[r * 32 + lane + 1];
    if (malformed || beg < klo || end > nnz || !__all_sync(0xffffffffu, ordered)) {  // malformed: skip the chunk
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
            if (k0 + u * 32 < end && k < end) {  // first test warp-uniform: empty slots cost nothing
                col[u] = ld_stream_i32(col_idx + (k - klo), pol);
                v[u] = ld_stream_f32(vals + (k - klo), pol);
            }
        }
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            if (k0 + u * 32 >= end) break;  // warp-uniform
            const int k = k0 + u * 32 + lane;
            if (k < end) {
                int lo = 0;
#pragma unroll
                for (int step = ROWS / 2; step > 0; step >>= 1)
                    if (s_rp[lo + step] <= k) lo += step;
                const int j = col[u];
                const uint32_t hb = s_h[lo];
                if (hb < blo || hb >= bhi) continue;  // another pass reduces this row
                if (static_cast<unsigned>(j) < static_cast<unsigned>(d)) {
                    const size_t at = static_cast<size_t>(hb) * d + j;
                    if (FIXED)
                        atomicAdd(static_cast<unsigned long long *>(SX) + at, to_fixed(s_sg[lo] * v[u], F));
                    else
                        atomicAdd(static_cast<float *>(SX) + at, s_sg[lo] * v[u]);
                } else {
                    bad = 1;
                }
            }
        }
    }
    __syncwarp();
}

// Rows [first, min(first + 32, n)) with one row per lane and no shared memory, for very
// sparse rows (about two nonzeros or fewer per row): lane l hashes row first + l and, if
// its bucket lies in [blo, bhi), walks the row's own nonzeros k = row_ptr[i] ..
// row_ptr[i + 1] - 1, one reduction each.  The warp takes as many steps as its longest
// row; the lanes' loads of one step fall in the chunk's short, contiguous range of
// col_idx / vals (indexed from klo as in scatter_chunk).  Out-of-range column indices
// and malformed row offsets are skipped and reported through `bad`.
// RP as in scatter_chunk (each lane walks its own row in RP arithmetic).
template <bool FIXED, bool SKIP_EMPTY = false, typename RP = int>
__device__ __forceinline__ void scatter_lanes32(const RP *__restrict__ row_ptr, const int *__restrict__ col_idx,
                                                const float *__restrict__ vals, int first, int n, int d, uint32_t B,
                                                RP nnz, RP klo, Key key, int64_t row_offset, void *__restrict__ SX,
                                                int F, int &bad, uint32_t blo = 0u, uint32_t bhi = 0xFFFFFFFFu) {
    const int lane = threadIdx.x & 31;
    const uint64_t pol = l2_evict_first_policy();
    const int i = first + lane;
    RP beg = 0;
    if constexpr (sizeof(RP) == 4)
        beg = i < n ? ld_stream_i32(row_ptr + i, pol) : 0;
    else
        beg = i < n ? ld_stream_i64(row_ptr + i, pol) : 0;
    RP end = __shfl_down_sync(0xffffffffu, beg, 1);  // row_ptr[i + 1] from the next lane
    if (i < n) {
        if (lane == 31 || i + 1 == n) end = __ldg(row_ptr + i + 1);
        if (beg < klo || end > nnz || beg > end) {  // malformed row offsets: skip the row
            bad = 1;
            end = beg;
        }
        uint32_t h = 0;
        float sg = 0.0f;
        if (!SKIP_EMPTY || beg < end) hash_sign(key, static_cast<uint64_t>(row_offset + i), B, h, sg);
        if (h < blo || h >= bhi) end = beg;  // another pass reduces this row
        const size_t base = static_cast<size_t>(h) * d;
        for (RP k = beg; k < end; ++k) {
            const int j = ld_stream_i32(col_idx + (k - klo), pol);
            const float v = ld_stream_f32(vals + (k - klo), pol);
            if (static_cast<unsigned>(j) < static_cast<unsigned>(d)) {
                if (FIXED)
                    atomicAdd(static_cast<unsigned long long *>(SX) + base + j, to_fixed(sg * v, F));
                else
                    atomicAdd(static_cast<float *>(SX) + base + j, sg * v);
            } else {
                bad = 1;
            }
        }
    }
    __syncwarp();
}

// The 32-row chunk (one row per lane).
template <bool FIXED, bool SKIP_EMPTY = false>
__device__ __forceinline__ void scatter_chunk32(const int *__restrict__ row_ptr, const int *__restrict__ col_idx,
                                                const float *__restrict__ vals, int first, int n, int d, uint32_t B,
                                                int nnz, Key key, int64_t row_offset, void *__restrict__ SX, int F,
                                                int *s_rp, uint32_t *s_h, float *s_sg, int &bad) {
    scatter_chunk<FIXED, 32, SKIP_EMPTY>(row_ptr, col_idx, vals, first, n, d, B, nnz, 0, key, row_offset, SX, F,
                                         s_rp, s_h, s_sg, bad);
}

}  // namespace cg

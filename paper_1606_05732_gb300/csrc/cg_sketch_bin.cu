// cg_sketch_bin.cu -- SX = S.X (Section 1.1, the O(nnz(X)) stage) for an SX larger than
// the L2 holds, with shared-memory sums instead of one L2 reduction per nonzero.
//
// A random fp32 reduction costs one L2 tag lookup at the slice the SM talks to, and a
// second one at the owning slice when the address lives on the other die; the lookup rate,
// not DRAM, caps a one-reduction-per-nonzero scatter (about 206 G/s on GB300 with SX in
// L2, and far less once SX outgrows it).  Here the B buckets are cut into P slices of SB
// buckets (SB a power of two, SB d <= 32768), small enough for one slice of SX (at most
// 128 KB) to sit in shared memory, and the scatter runs in two passes:
//   pass 1 (bin)    persistent CTAs take tiles of rows.  Each row is hashed once; one
//                   shared-memory atomic per row reserves the row's run among the tile's
//                   records of its slice; the records (slice-local cell h' d + j as 16 bits,
//                   sigma x as fp32) are sorted by slice in shared memory, each slice's run
//                   gets its place in that slice's record stream from one global atomic per
//                   tile and slice, and the runs are written out coalesced.  All CTAs append
//                   to the same P streams, so the L2 completes their lines before writing
//                   them back.  Records past a stream's capacity (1.0625x its even share
//                   plus 1024) go to an overflow list.  The next tile's CSR ranges are
//                   prefetched into L2 while the current tile is sorted.
//   pass 2 (reduce) one CTA per slice streams its records into shared-memory atomics and
//                   writes the slice of SX once; the last CTA to finish adds the overflow
//                   list (normally empty) with global atomics.
// DRAM traffic: the CSR once, 6 bytes of record per nonzero written and read once, SX
// written once.  Sums are fp32 in an order that depends on timing, as with the atomic
// scatter -- or, in the deterministic mode's form, the exact int64 fixed-point sums of
// the deterministic scatter (two reduce CTAs per slice, one half of its cells each, after
// a max-|x| pass), which do not depend on the order.
#include <algorithm>

#include "cg_internal.cuh"
#include "cg_scatter.cuh"

namespace cg {

namespace {

constexpr int kBinThreads = 512;
constexpr int kReduceThreads = 1024;
constexpr uint32_t kNoKey = 0xFFFFu;  // a record that adds nothing (bad column index)
constexpr int kSliceFloats = 32768;   // shared-memory slice of SX: 128 KB at most
constexpr uint32_t kFixedCells = 16384;  // int64 cells of one reduce CTA in the fixed-point form
constexpr int kMaxSlices = 2048;
constexpr int kStageRecords = 5632;   // records of a tile sorted in shared memory (two CTAs per SM)

struct BinArgs {
    const int *row_ptr;
    const int *col_idx;
    const float *vals;
    int n, nnz, d;
    uint32_t B;
    Key key;
    int64_t row_offset;
    int sb_log2;       // buckets per slice = 2^sb_log2
    int P;             // slices
    int rows_per_cta;  // a multiple of the tile height
    int T;             // staged records per tile
    int prefetch;      // L2 prefetch of the next tile (off when the CSR is host memory read in place)
    int scap;          // records per slice stream (a multiple of 8)
    uint16_t *rkeys;   // slice streams: slice-local cell
    float *rvals;      //                sigma x
    int *cursor;       // [P] records appended to each stream; then the overflow count, pass 2's arrivals
    uint2 *orec;       // overflow records: (global cell, sigma x bits)
    int ocap;
    int *status;
};

__device__ __forceinline__ void st_u16(uint16_t *p, uint16_t v) {
    asm volatile("st.global.u16 [%0], %1;" ::"l"(p), "h"(v) : "memory");
}

// L2 prefetch of bytes [lo, hi) of a global array, 16-byte aligned inside the range.
__device__ __forceinline__ void prefetch_l2(const void *lo, const void *hi) {
    uintptr_t a = (reinterpret_cast<uintptr_t>(lo) + 15) & ~static_cast<uintptr_t>(15);
    const uintptr_t e = reinterpret_cast<uintptr_t>(hi) & ~static_cast<uintptr_t>(15);
    for (; a < e; a += (1u << 20)) {
        const uint32_t len = static_cast<uint32_t>(e - a < (1u << 20) ? e - a : (1u << 20));
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(len) : "memory");
    }
}

// Record (slice s, slice-local cell key, value x) at position r of slice s's stream; past
// the stream's capacity it goes to the overflow list (bad keys are dropped there).
__device__ __forceinline__ void put_record(const BinArgs &a, int s, int r, uint32_t key, float x, int &bad) {
    if (r < a.scap) {
        const long long at = static_cast<long long>(s) * a.scap + r;
        st_u16(a.rkeys + at, static_cast<uint16_t>(key));
        a.rvals[at] = x;
    } else if (key != kNoKey) {
        int *ocount = a.cursor + a.P;
        const int o = atomicAdd(ocount, 1);
        if (o < a.ocap)
            a.orec[o] = make_uint2((static_cast<uint32_t>(s) << a.sb_log2) * static_cast<uint32_t>(a.d) + key,
                                   __float_as_uint(x));
        else
            bad = 1;
    }
}

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Rows [lo, hi] of row_ptr (hi inclusive) into s_rp by asynchronous 4-byte copies.
__device__ __forceinline__ void copy_row_ptr(const int *row_ptr, int lo, int hi, int *s_rp) {
    for (int i = threadIdx.x; i <= hi - lo; i += kBinThreads) cp_async4(s_rp + i, row_ptr + lo + i);
    cp_async_commit();
}

// Row of a tile held in slot q of thread t: with four or more rows per thread, groups
// of four consecutive rows (so that one Philox call hashes a group, the four rows of a
// call), else rows q kBinThreads + t.
template <int RPL>
__device__ __forceinline__ int bin_row(int q, int t) {
    return RPL >= 4 ? 4 * ((q >> 2) * kBinThreads + t) + (q & 3) : q * kBinThreads + t;
}

template <int RPL>
__global__ void __launch_bounds__(kBinThreads, RPL <= 8 ? 2 : 1) bin_pass_kernel(BinArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int TR = kBinThreads * RPL;
    int *s_in_col = reinterpret_cast<int *>(smem);            // the tile's nonzeros: column
    float *s_in_val = reinterpret_cast<float *>(s_in_col + a.T);  //                     value
    uint32_t *s_rec = reinterpret_cast<uint32_t *>(s_in_val + a.T);  // cell | slice << 16 | sign << 31
    int *s_rp = reinterpret_cast<int *>(s_rec + a.T);          // the tile's row offsets
    int *s_cnt = s_rp + TR + 1;                                 // records of the tile per slice
    int *s_base = s_cnt + a.P;                                  // first staging slot per slice
    int *s_gpos = s_base + a.P;                                 // the tile's place in each stream
    uint16_t *s_src = reinterpret_cast<uint16_t *>(s_gpos + a.P);  // input slot of each staging slot
    __shared__ int s_wsum[kBinThreads / 32];
    __shared__ int s_total;
    constexpr int kPer = (kMaxSlices + kBinThreads - 1) / kBinThreads;  // slices per thread in the scan

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int r0 = static_cast<int>(
        min(static_cast<long long>(a.n), static_cast<long long>(blockIdx.x) * a.rows_per_cta));
    const int r1 = static_cast<int>(min(static_cast<long long>(a.n), static_cast<long long>(r0) + a.rows_per_cta));
    const int A0 = __ldg(a.row_ptr + r0), A1 = __ldg(a.row_ptr + r1);
    if (!(0 <= A0 && A0 <= A1 && A1 <= a.nnz)) {  // malformed offsets at the CTA's ends: no records
        if (t == 0) atomicOr(a.status, kStatusBounds);
        return;
    }
    for (int i = t; i < a.P; i += kBinThreads) s_cnt[i] = 0;
    const uint32_t smask = (1u << a.sb_log2) - 1u;
    const uint32_t d = static_cast<uint32_t>(a.d);
    const int per = (a.P + kBinThreads - 1) / kBinThreads;
    const int i0 = min(a.P, t * per), i1 = min(a.P, i0 + per);
    int bad = 0;
    if (t == 0 && a.prefetch) {  // the first tile's nonzeros
        const int k1 = __ldg(a.row_ptr + min(r1, r0 + TR));
        if (A0 <= k1 && k1 <= A1) {
            prefetch_l2(a.col_idx + A0, a.col_idx + k1);
            prefetch_l2(a.vals + A0, a.vals + k1);
        }
    }
    copy_row_ptr(a.row_ptr, r0, min(r1, r0 + TR), s_rp);

    for (int tr0 = r0; tr0 < r1; tr0 += TR) {
        const int tr1 = min(r1, tr0 + TR);
        cp_async_wait<0>();
        __syncthreads();  // s_rp holds row_ptr[tr0 .. tr1]; the previous tile is written out
        const int K0 = s_rp[0], K1 = s_rp[tr1 - tr0];
        const bool fast_in = A0 <= K0 && K0 <= K1 && K1 <= A1 && K1 - K0 <= a.T;
        if (fast_in) {  // the tile's nonzeros into shared memory while the rows are hashed
            for (int i = t; i < K1 - K0; i += kBinThreads) {
                cp_async4(s_in_col + i, a.col_idx + K0 + i);
                cp_async4(s_in_val + i, a.vals + K0 + i);
            }
        }
        cp_async_commit();
        if (t == 0 && a.prefetch && tr1 < r1) {  // the next tile into L2
            const int nlast = min(r1, tr1 + TR);
            prefetch_l2(a.row_ptr + tr1, a.row_ptr + nlast + 1);
            const int kn0 = K1, kn1 = __ldg(a.row_ptr + nlast);
            if (A0 <= kn0 && kn0 <= kn1 && kn1 <= A1) {
                prefetch_l2(a.col_idx + kn0, a.col_idx + kn1);
                prefetch_l2(a.vals + kn0, a.vals + kn1);
            }
        }
        // ---- A: hash the rows, reserve each row's run in its slice -------------------
        int kb[RPL], len[RPL], off[RPL];
        uint32_t code[RPL];
        int row_bad = 0;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int i = bin_row<RPL>(q, t);
            int k0 = 0, k1 = 0;
            if (tr0 + i < tr1) {
                k0 = s_rp[i];
                k1 = s_rp[i + 1];
                if (k0 < A0 || k1 > A1 || k0 > k1) {  // malformed offsets: skip the row
                    row_bad = 1;
                    k1 = k0;
                }
            }
            kb[q] = k0;
            len[q] = k1 - k0;
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            code[q] = 0;
            off[q] = 0;
        }
        if (RPL >= 4 && ((a.row_offset + tr0) & 3) == 0) {  // uniform: a thread's groups of four are calls
#pragma unroll
            for (int g = 0; g < RPL / 4; ++g) {
                if ((len[4 * g] | len[4 * g + 1] | len[4 * g + 2] | len[4 * g + 3]) == 0) continue;
                const uint4 w = stream_words(
                    a.key, static_cast<uint64_t>(a.row_offset + tr0 + bin_row<RPL>(4 * g, t)) >> 2, kTagHash);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (len[4 * g + j] == 0) continue;
                    const uint32_t h = __umulhi(ws[j], a.B);
                    code[4 * g + j] = h | (ws[j] << 31);  // sigma = -1 for an odd word
                    off[4 * g + j] = atomicAdd(&s_cnt[h >> a.sb_log2], len[4 * g + j]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                if (len[q] > 0) {
                    uint32_t h;
                    float sg;
                    hash_sign(a.key, static_cast<uint64_t>(a.row_offset + tr0 + bin_row<RPL>(q, t)), a.B, h, sg);
                    code[q] = h | (sg < 0.0f ? 0x80000000u : 0u);
                    off[q] = atomicAdd(&s_cnt[h >> a.sb_log2], len[q]);
                }
            }
        }
        bad |= row_bad;
        // rows with ordered offsets inside the CTA's range cover [K0, K1) exactly once
        const int tile_bad = __syncthreads_or(row_bad);
        // ---- B: slice offsets in the staging buffer; each slice's run asks for its place
        // in the slice's stream (the answers are awaited after the staging phase)
        int cnts[kPer], gpos[kPer];
        {
            int sum = 0;
#pragma unroll
            for (int e = 0; e < kPer; ++e) {
                cnts[e] = i0 + e < i1 ? s_cnt[i0 + e] : 0;
                sum += cnts[e];
            }
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_wsum[warp] = incl;
            __syncthreads();
            int run = incl - sum;
            for (int w = 0; w < warp; ++w) run += s_wsum[w];
            if (t == kBinThreads - 1) s_total = run + sum;
#pragma unroll
            for (int e = 0; e < kPer; ++e) {
                gpos[e] = 0;
                if (i0 + e < i1) {
                    s_base[i0 + e] = run;
                    if (cnts[e] > 0) gpos[e] = atomicAdd(a.cursor + i0 + e, cnts[e]);
                    s_cnt[i0 + e] = 0;
                    run += cnts[e];
                }
            }
        }
        __syncthreads();  // s_base visible; s_rp no longer read
        if (tr1 < r1)
            copy_row_ptr(a.row_ptr, tr1, min(r1, tr1 + TR), s_rp);
        else
            cp_async_commit();  // an empty group keeps the group count uniform
        const int total = s_total;
        if (fast_in && !tile_bad && total <= a.T) {  // uniform over the CTA
            // ---- C: each row writes its record template into its staging slots and, per
            // slot, the input slot of its nonzero (shared memory only)
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                if (len[q] == 0) continue;
                const uint32_t h = code[q] & 0x7FFFFFFFu;
                const uint32_t s = h >> a.sb_log2;
                const uint32_t tmpl = ((h & smask) * d) | (s << 16) | (code[q] & 0x80000000u);
                const int pos = s_base[s] + off[q];
                const int rel = kb[q] - K0;
                for (int j = 0; j < len[q]; ++j) {
                    s_rec[pos + j] = tmpl;
                    s_src[pos + j] = static_cast<uint16_t>(rel + j);
                }
            }
#pragma unroll
            for (int e = 0; e < kPer; ++e)
                if (i0 + e < i1) s_gpos[i0 + e] = gpos[e];
            cp_async_wait<1>();  // the tile's nonzeros (the next row offsets may still be in flight)
        } else {
            // A tile with more records than the staging buffer (or with malformed offsets):
            // its rows are walked by their lanes from global memory; staged records carry
            // their column already (input column 0), the rest go straight to the streams.
#pragma unroll
            for (int e = 0; e < kPer; ++e)
                if (i0 + e < i1) s_gpos[i0 + e] = gpos[e];
            cp_async_wait<1>();  // no copy may still land in the input buffer
            __syncthreads();
            const uint64_t pol = l2_evict_first_policy();
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                if (len[q] == 0) continue;
                const uint32_t h = code[q] & 0x7FFFFFFFu;
                const uint32_t s = h >> a.sb_log2;
                const uint32_t cell0 = (h & smask) * d;
                const uint32_t neg = code[q] & 0x80000000u;
                const int pos = s_base[s] + off[q];
                const int gp = s_gpos[s] + off[q];
                for (int j = 0; j < len[q]; ++j) {
                    const int col = ld_stream_i32(a.col_idx + kb[q] + j, pol);
                    const float v = ld_stream_f32(a.vals + kb[q] + j, pol);
                    uint32_t key = kNoKey;
                    if (static_cast<unsigned>(col) < d)
                        key = cell0 + static_cast<uint32_t>(col);
                    else
                        bad = 1;
                    const float x = __uint_as_float(__float_as_uint(v) ^ neg);
                    if (pos + j < a.T) {
                        s_rec[pos + j] = key | (s << 16);
                        s_in_col[pos + j] = 0;
                        s_in_val[pos + j] = x;
                        s_src[pos + j] = static_cast<uint16_t>(pos + j);
                    } else {
                        put_record(a, static_cast<int>(s), gp + j, key, x, bad);
                    }
                }
            }
        }
        __syncthreads();
        // ---- D: the sorted runs to their streams, coalesced -------------------------------
        const int nst = min(total, a.T);
        for (int i = t; i < nst; i += kBinThreads) {
            const uint32_t tm = s_rec[i];
            const int src = s_src[i];
            const int col = s_in_col[src];
            const float v = s_in_val[src];
            const int s = static_cast<int>((tm >> 16) & 0x7FFu);
            uint32_t key = kNoKey;
            if (static_cast<unsigned>(col) < d)
                key = (tm & 0xFFFFu) + static_cast<uint32_t>(col);
            else
                bad = 1;
            put_record(a, s, s_gpos[s] + (i - s_base[s]), key, __uint_as_float(__float_as_uint(v) ^ (tm & 0x80000000u)),
                       bad);
        }
    }
    if (bad) atomicOr(a.status, kStatusBounds);
}

// Pass 2: CTA s sums slice s (buckets [s SB, min((s+1) SB, B))) of SX in shared memory
// from its record stream and writes it once (adding to SX when `accumulate`); the last CTA
// to arrive adds the overflow records.  With FIXED the cells hold int64 fixed-point sums
// (to_fixed(x, F), F from maxbits and nnz as in the deterministic scatter), `parts` CTAs
// share a slice (each reads the whole stream and keeps its cells), and each CTA adds the
// overflow records of its own cells before the one rounding to fp32 -- exact and
// order-independent, so the result is bit-identical to the fixed-point scatter's.
template <bool FIXED>
__global__ void __launch_bounds__(kReduceThreads)
bin_reduce_kernel(const uint16_t *__restrict__ rkeys, const float *__restrict__ rvals, int *__restrict__ cursor,
                  int P, int scap, int sb_log2, int d, uint32_t B, float *__restrict__ SX, int accumulate, int ocap,
                  const uint2 *__restrict__ orec, const int *__restrict__ maxbits, int nnz, int parts) {
    extern __shared__ __align__(16) unsigned char slice_raw[];
    float *slice = reinterpret_cast<float *>(slice_raw);
    unsigned long long *slice64 = reinterpret_cast<unsigned long long *>(slice_raw);
    __shared__ int s_last;
    // With FIXED, `parts` CTAs share slice s, CTA `part` summing its cells
    // [part kFixedCells, (part + 1) kFixedCells) (an int64 cell takes twice the bytes).
    const int s = blockIdx.x / parts, part = blockIdx.x % parts, t = threadIdx.x;
    const uint32_t b0 = static_cast<uint32_t>(s) << sb_log2;
    const uint32_t nb = min(1u << sb_log2, B - b0);
    const uint32_t nf_slice = nb * static_cast<uint32_t>(d);
    const uint32_t lo = FIXED ? static_cast<uint32_t>(part) * kFixedCells : 0u;
    const uint32_t nf = FIXED ? (nf_slice > lo ? min(nf_slice - lo, kFixedCells) : 0u) : nf_slice;
    float *dst = SX + static_cast<size_t>(b0) * d + lo;
    const bool vec = (nf & 3u) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    pdl_wait();  // pass 1 wrote the streams (and the max-|x| pass maxbits)
    const int F = FIXED ? fixed_point_exponent(*maxbits, nnz) : 0;
    const int cnt = min(__ldg(cursor + s), scap);
    const long long at = static_cast<long long>(s) * scap;  // 16-byte aligned: scap is a multiple of 8
    const uint16_t *keys = rkeys + at;
    const float *vs = rvals + at;
    if (t == 0 && cnt > 0) {
        prefetch_l2(keys, keys + cnt);
        prefetch_l2(vs, vs + cnt);
    }
    if (FIXED) {
        for (uint32_t i = t; i < nf; i += kReduceThreads) slice64[i] = 0ull;
    } else if (vec) {
        for (uint32_t i = t; i < (nf >> 2); i += kReduceThreads)
            reinterpret_cast<float4 *>(slice)[i] =
                accumulate ? reinterpret_cast<const float4 *>(dst)[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        for (uint32_t i = t; i < nf; i += kReduceThreads) slice[i] = accumulate ? dst[i] : 0.0f;
    }
    __syncthreads();
    auto add = [&](uint32_t k, float v) {
        if (FIXED)
            atomicAdd(slice64 + k, to_fixed(v, F));
        else
            atomicAdd(slice + k, v);
    };
    const uint64_t pol = l2_evict_first_policy();
    const int n8 = cnt >> 3;
    constexpr int kIn = 2;  // groups of eight records in flight per thread
    for (int q0 = 0; q0 < n8; q0 += kReduceThreads * kIn) {
        uint4 k8[kIn];
        float4 v0[kIn], v1[kIn];
#pragma unroll
        for (int u = 0; u < kIn; ++u) {
            const int q = q0 + u * kReduceThreads + t;
            if (q < n8) {
                asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                             : "=r"(k8[u].x), "=r"(k8[u].y), "=r"(k8[u].z), "=r"(k8[u].w)
                             : "l"(keys + 8 * q), "l"(pol));
                asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                             : "=f"(v0[u].x), "=f"(v0[u].y), "=f"(v0[u].z), "=f"(v0[u].w)
                             : "l"(vs + 8 * q), "l"(pol));
                asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                             : "=f"(v1[u].x), "=f"(v1[u].y), "=f"(v1[u].z), "=f"(v1[u].w)
                             : "l"(vs + 8 * q + 4), "l"(pol));
            }
        }
#pragma unroll
        for (int u = 0; u < kIn; ++u) {
            if (q0 + u * kReduceThreads + t >= n8) break;
            const uint32_t kk[8] = {k8[u].x & 0xFFFFu, k8[u].x >> 16, k8[u].y & 0xFFFFu, k8[u].y >> 16,
                                    k8[u].z & 0xFFFFu, k8[u].z >> 16, k8[u].w & 0xFFFFu, k8[u].w >> 16};
            const float vv[8] = {v0[u].x, v0[u].y, v0[u].z, v0[u].w, v1[u].x, v1[u].y, v1[u].z, v1[u].w};
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (kk[e] - lo < nf) add(kk[e] - lo, vv[e]);
        }
    }
    for (int i = (n8 << 3) + t; i < cnt; i += kReduceThreads) {
        const uint32_t k = keys[i];
        if (k - lo < nf) add(k - lo, vs[i]);
    }
    if (FIXED) {
        // the overflow records of this slice (pass 1 finished: their count is final)
        const int no = min(__ldg(cursor + P), ocap);
        const uint32_t c0 = b0 * static_cast<uint32_t>(d) + lo;
        for (int i = t; i < no; i += kReduceThreads) {
            const uint2 r = __ldg(orec + i);
            if (r.x >= c0 && r.x - c0 < nf) add(r.x - c0, __uint_as_float(r.y));
        }
        __syncthreads();
        for (uint32_t i = t; i < nf; i += kReduceThreads)
            dst[i] = ldexpf(__ll2float_rn(static_cast<long long>(slice64[i])), -F);
        return;
    }
    __syncthreads();
    if (vec) {
        for (uint32_t i = t; i < (nf >> 2); i += kReduceThreads)
            reinterpret_cast<float4 *>(dst)[i] = reinterpret_cast<const float4 *>(slice)[i];
    } else {
        for (uint32_t i = t; i < nf; i += kReduceThreads) dst[i] = slice[i];
    }
    // the last CTA adds the overflow records once every slice is written
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(cursor + P + 1, 1) == static_cast<int>(gridDim.x) - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int no = min(*reinterpret_cast<volatile int *>(cursor + P), ocap);
    const uint32_t cells = B * static_cast<uint32_t>(d);
    for (int i = t; i < no; i += kReduceThreads) {
        const uint2 r = orec[i];
        if (r.x < cells) atomicAdd(SX + r.x, __uint_as_float(r.y));
    }
}

// Rows per lane per tile: the most (a power of two, at most 16) whose tiles hold at most
// 95 % of the staging buffer's records on average; a tile past the buffer is rare and
// takes the slower path.
int rows_per_lane(int64_t n, int64_t nnz, int T) {
    const double per_row = n > 0 ? static_cast<double>(nnz) / static_cast<double>(n) : 1.0;
    const double want = 0.95 * T / (kBinThreads * (per_row > 1.0 / 16 ? per_row : 1.0 / 16));
    int r = 1;
    while (r < 16 && 2 * r <= want) r *= 2;
    return r;
}

// log2 of the buckets per slice: the largest power of two SB with SB d <= kSliceFloats.
// The fixed-point form bins by the same slices (fewer slices keep pass 1's runs long) and
// sums each in kFixedCells parts.
int slice_log2(int d) {
    int l = 0;
    while ((2LL << l) * d <= kSliceFloats) ++l;
    return l;
}

struct BinPlan {
    int sb_log2 = 0, P = 0, G = 0, RPL = 1, rows_per_cta = 0, T = kStageRecords, scap = 0;
    size_t keys_off = 0, vals_off = 0, cursor_off = 0, orec_off = 0, maxbits_off = 0, bytes = 0;
};

BinPlan bin_plan(int64_t n, int d, int64_t B, int64_t nnz, int ctas, bool fixed = false) {
    BinPlan L;
    L.sb_log2 = slice_log2(d);
    L.P = static_cast<int>((B + (1LL << L.sb_log2) - 1) >> L.sb_log2);
    const int sms = num_sms() > 0 ? num_sms() : 148;
    const int G = ctas > 0 ? ctas : 2 * sms;
    L.RPL = rows_per_lane(n, nnz, L.T);
    const int64_t TR = static_cast<int64_t>(kBinThreads) * L.RPL;
    const int64_t per = (n + G - 1) / G;
    L.rows_per_cta = static_cast<int>(std::max<int64_t>(TR, (per + TR - 1) / TR * TR));
    L.G = static_cast<int>(std::max<int64_t>(1, (n + L.rows_per_cta - 1) / L.rows_per_cta));
    // stream capacity: the even share of the nonzeros plus 1/16 and 1024, in whole
    // groups of eight records (so that every stream starts 16-byte aligned)
    const int64_t share = (nnz + L.P - 1) / L.P;
    L.scap = static_cast<int>(((share + share / 16 + 1024) + 7) / 8 * 8);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t records = static_cast<size_t>(L.P) * static_cast<size_t>(L.scap);
    L.keys_off = take(records * sizeof(uint16_t));
    L.vals_off = take(records * sizeof(float));
    L.cursor_off = take((static_cast<size_t>(L.P) + 2) * sizeof(int));
    L.orec_off = take(static_cast<size_t>(std::max<int64_t>(nnz, 1)) * sizeof(uint2));
    L.maxbits_off = take(fixed ? 2 * sizeof(int) : 0);
    L.bytes = off;
    return L;
}

size_t bin_smem(const BinPlan &L) {
    return static_cast<size_t>(L.T) * 14 + (static_cast<size_t>(kBinThreads) * L.RPL + 1) * 4 +
           static_cast<size_t>(L.P) * 12;
}

template <int RPL>
cudaError_t launch_bin_pass(const BinPlan &L, const BinArgs &a, cudaStream_t stream) {
    const size_t smem = bin_smem(L);
    cudaError_t e = cudaFuncSetAttribute(bin_pass_kernel<RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    bin_pass_kernel<RPL><<<L.G, kBinThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool binned_supported(int64_t n, int d, int64_t B, bool fixed) {
    (void)fixed;
    if (d > kSliceFloats || n <= 0) return false;
    const int l = slice_log2(d);
    const int64_t P = (B + (1LL << l) - 1) >> l;
    return P <= kMaxSlices && static_cast<uint64_t>(P << l) * static_cast<uint64_t>(d) < (1ull << 32);
}

size_t sketch_binned_scratch_bytes(int64_t n, int d, int64_t B, int64_t nnz, int ctas, bool fixed) {
    return bin_plan(n, d, B, nnz, ctas, fixed).bytes;
}

cudaError_t launch_sketch_csr_binned(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                     uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, int *status,
                                     void *scratch, int ctas, const EventPair *ev, cudaStream_t stream, bool clear,
                                     bool prefetch, bool fixed) {
    const BinPlan L = bin_plan(n, d, B, nnz, ctas, fixed);
    char *base = static_cast<char *>(scratch);
    BinArgs a;
    a.row_ptr = row_ptr;
    a.col_idx = col_idx;
    a.vals = vals;
    a.n = n;
    a.nnz = nnz;
    a.d = d;
    a.B = B;
    a.key = key;
    a.row_offset = row_offset;
    a.sb_log2 = L.sb_log2;
    a.P = L.P;
    a.rows_per_cta = L.rows_per_cta;
    a.T = L.T;
    a.prefetch = prefetch ? 1 : 0;
    a.scap = L.scap;
    a.rkeys = reinterpret_cast<uint16_t *>(base + L.keys_off);
    a.rvals = reinterpret_cast<float *>(base + L.vals_off);
    a.cursor = reinterpret_cast<int *>(base + L.cursor_off);
    a.orec = reinterpret_cast<uint2 *>(base + L.orec_off);
    a.ocap = std::max(nnz, 1);
    a.status = status;
    int *maxbits = fixed ? reinterpret_cast<int *>(base + L.maxbits_off) : nullptr;
    cudaError_t e = cudaMemsetAsync(a.cursor, 0, (static_cast<size_t>(L.P) + 2) * sizeof(int), stream);
    if (e == cudaSuccess && fixed) e = cudaMemsetAsync(maxbits, 0, 2 * sizeof(int), stream);
    if (e != cudaSuccess) return e;
    record(ev, true, stream);
    if (fixed && (e = launch_absmax(vals, nnz, maxbits, stream)) != cudaSuccess) return e;
    switch (L.RPL) {
        case 1: e = launch_bin_pass<1>(L, a, stream); break;
        case 2: e = launch_bin_pass<2>(L, a, stream); break;
        case 4: e = launch_bin_pass<4>(L, a, stream); break;
        case 8: e = launch_bin_pass<8>(L, a, stream); break;
        default: e = launch_bin_pass<16>(L, a, stream); break;
    }
    if (e != cudaSuccess) return e;
    const size_t slice_cells = (static_cast<size_t>(1) << L.sb_log2) * d;
    const int parts = fixed ? static_cast<int>((slice_cells + kFixedCells - 1) / kFixedCells) : 1;
    const size_t smem2 = fixed ? std::min<size_t>(slice_cells, kFixedCells) * sizeof(unsigned long long)
                               : slice_cells * sizeof(float);
    auto reduce = fixed ? bin_reduce_kernel<true> : bin_reduce_kernel<false>;
    if ((e = cudaFuncSetAttribute(reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem2))) !=
        cudaSuccess)
        return e;
    e = launch_after_previous(reduce, dim3(L.P * parts), dim3(kReduceThreads), smem2, stream,
                              static_cast<const uint16_t *>(a.rkeys), static_cast<const float *>(a.rvals), a.cursor,
                              L.P, L.scap, L.sb_log2, d, B, SX, clear ? 0 : 1, a.ocap,
                              static_cast<const uint2 *>(a.orec), static_cast<const int *>(maxbits), nnz, parts);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && fixed)
        e = launch_add_nonfinite(row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset, maxbits, SX, stream);
    record(ev, false, stream);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace cg

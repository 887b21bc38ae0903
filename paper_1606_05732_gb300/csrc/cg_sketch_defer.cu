// cg_sketch_defer.cu -- SX = S.X (Section 1.1, the O(nnz(X)) stage) for an SX too large
// for the L2 to hold, in one pass over the CSR plus one pass over records.
//
// One fp32 reduction per nonzero runs at the L2's atomic rate only while the reduced
// array stays in L2; past that (on GB300 from about 100 MB on) most reductions miss and
// the rate falls several-fold.  So SX is split at bucket bsplit (B/2, or more so that the
// lower part fills about 0.62 of the L2; deferred_split):
//   pass 1  streams the CSR once, hashes every row once, reduces the nonzeros of rows
//           with h < bsplit into SX at once, and writes those of the other rows as
//           8-byte records (h d + j, sigma x) into its CTA's region of a records buffer
//           (regions follow the nonzero order: CTA c owns rows [c R, (c+1) R) and the
//           record slots of their nonzeros; one shared atomic per warp and 128 nonzeros
//           hands out slots, so records are written compactly and coalesced);
//   pass 2  streams each region's records and reduces them into the upper part of SX,
//           which is then the one in L2.
// Each part of SX stays within the L2 (for an SX up to about 1.1 times its size), and the
// extra traffic is the records, 16 bytes per deferred nonzero (written once, read once,
// with an evict-first L2 policy).  Sums are fp32 in an order that depends on timing, as
// with the atomic scatter.  Both passes are
// templated on the type of the row offsets: int, or long long for matrices of 2^31
// nonzeros or more (warp chunks rebased to their first nonzero, 64-bit record indices
// and per-CTA counts).
#include <algorithm>

#include "cg_internal.cuh"
#include "cg_scatter.cuh"
#include "cg_tc.cuh"

namespace cg {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ void st_stream_u2(uint2 *p, uint2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ uint2 ld_stream_u2(const uint2 *p, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}

// Reductions into SX carry an evict-last L2 priority: each pass reduces into a part of SX
// that fits the L2 while hundreds of MB of CSR and records stream past it (evict-first),
// and without the hint the L2 still wrote the reduced lines back to DRAM several times
// over (at the 2^26 x 128 ladder shape pass 1 wrote 845 MB per launch, 464 MB with the
// hint; the replay 307 MB, 1 MB with it; sketch 0.774 -> 0.708 ms).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void red_add_last(float *a, float v, uint64_t pol) {
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}

// The same reduction, or nothing where p is false (a predicated instruction, no branch).
__device__ __forceinline__ void red_add_last_if(bool p, float *a, float v, uint64_t pol) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q red.global.add.L2::cache_hint.f32 [%0], %1, %3;\n\t}" ::"l"(a),
        "f"(v), "r"(static_cast<int>(p)), "l"(pol)
        : "memory");
}

// A record store with the evict-first hint, or nothing where p is false.
__device__ __forceinline__ void st_stream_u2_if(bool p, uint2 *a, uint2 v, uint64_t pol) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %4;\n\t}" ::"l"(a),
        "r"(v.x), "r"(v.y), "r"(static_cast<int>(p)), "l"(pol)
        : "memory");
}

// Shared-memory counter of a CTA's records: returns the old value.
__device__ __forceinline__ int add_count(int *c, int v) { return atomicAdd(c, v); }
__device__ __forceinline__ long long add_count(long long *c, int v) {
    return static_cast<long long>(atomicAdd(reinterpret_cast<unsigned long long *>(c), static_cast<unsigned long long>(v)));
}

// Rows [first, min(first + ROWS, n)) staged as in scatter_chunk: lane l loads the
// row_ptr entries of rows first + l + 32 r and hashes those rows into s_rp[ROWS + 1],
// s_h[ROWS], s_sg[ROWS].  RP is the type of the row offsets: int, or long long for
// matrices of 2^31 nonzeros or more, whose chunk offsets are rebased to the chunk's first
// nonzero `base` (so s_rp holds 32-bit offsets; a chunk of more than kMaxChunkNnz
// nonzeros is malformed); with int, base = 0.  Returns the chunk's nonzero range
// [beg, end) relative to base, or false (setting `bad`) if the offsets leave [0, nnz] or
// are out of order.  All lanes of the warp take part.
template <int ROWS, typename RP>
__device__ __forceinline__ bool stage_chunk(const RP *__restrict__ row_ptr, int first, int n, RP nnz, uint32_t B,
                                            Key key, int64_t row_offset, int *s_rp, uint32_t *s_h, float *s_sg,
                                            uint64_t pol, int &beg, int &end, RP &base, int &bad) {
    static_assert(ROWS == 32 || ROWS == 64 || ROWS == 128 || ROWS == 256, "chunk height");
    constexpr int R = ROWS / 32;
    const int lane = threadIdx.x & 31;
    const int last = min(first + ROWS, n);
    int rp[R];
    bool malformed = false;
    if constexpr (sizeof(RP) == 4) {
        base = 0;
        end = __ldg(row_ptr + last);
#pragma unroll
        for (int r = 0; r < R; ++r) {  // all row_ptr loads in flight before the hashing
            const int i = first + r * 32 + lane;
            rp[r] = i < n ? ld_stream_i32(row_ptr + i, pol) : end;
        }
        malformed = end > nnz;
    } else {
        const long long end64 = __ldg(row_ptr + last);
        long long rp64[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = first + r * 32 + lane;
            rp64[r] = i < n ? ld_stream_i64(row_ptr + i, pol) : end64;
        }
        base = __shfl_sync(0xffffffffu, rp64[0], 0);  // row_ptr[first]
        malformed = base < 0 || end64 > nnz || end64 < base || end64 - base > kMaxChunkNnz;
        const long long span = malformed ? 0 : end64 - base;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long rel = rp64[r] - base;
            rp[r] = rel >= 0 && rel <= span ? static_cast<int>(rel) : -1;  // -1 breaks the order check
            malformed |= rel < 0 || rel > span;
        }
        malformed = __any_sync(0xffffffffu, malformed);
        end = static_cast<int>(span);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = first + r * 32 + lane;
        uint32_t h = 0;
        float sg = 0.0f;
        if (i < n) hash_sign(key, static_cast<uint64_t>(row_offset + i), B, h, sg);
        s_rp[r * 32 + lane] = rp[r];
        s_h[r * 32 + lane] = h;
        s_sg[r * 32 + lane] = sg;
    }
    if (lane == 0) s_rp[ROWS] = end;
    __syncwarp();
    beg = s_rp[0];
    bool ordered = true;
#pragma unroll
    for (int r = 0; r < R; ++r) ordered &= s_rp[r * 32 + lane] <= s_rp[r * 32 + lane + 1];
    if (malformed || beg < 0 || !__all_sync(0xffffffffu, ordered)) {  // malformed row_ptr: skip the chunk
        bad = 1;
        __syncwarp();
        return false;
    }
    return true;
}

// Rows of a chunk whose nonzeros number at most kMapCap find a nonzero's row in a
// per-warp map (one byte per nonzero, written by the row's lane: the rows are in order)
// instead of by binary search over the row offsets.
constexpr int kMapCap = 1024;

// The row map of a staged chunk (after stage_chunk, end - beg <= kMapCap): lane l writes,
// for each of its rows q = l + 32 r, q into s_map[k - beg] for the row's nonzeros k.
template <int ROWS>
__device__ __forceinline__ void map_rows(const int *s_rp, int beg, uint8_t *s_map) {
    constexpr int R = ROWS / 32;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int q = r * 32 + lane;
        const int a = s_rp[q], e = s_rp[q + 1];
        for (int k = a; k < e; ++k) s_map[k - beg] = static_cast<uint8_t>(q);
    }
    __syncwarp();
}

// Pass 1 on one staged chunk: nonzeros of rows with h < bsplit are reduced into SX;
// the others become records appended to the CTA's region region[0, cap) through
// *s_count (one shared atomic per warp and 32 kScatterUnroll nonzeros).  col_idx and
// vals point at the chunk's base nonzero, so nonzero k of [beg, end) is col_idx[k],
// vals[k].  The nonzeros are swept 32 x kScatterUnroll at a
// time with coalesced evict-first loads, each finding its row in the row map (s_map
// non-null) or by a log2(ROWS)-step binary search over s_rp.  Bad column indices, and
// records that would leave the region (only possible with malformed offsets), are
// dropped and reported through `bad`.
template <int ROWS, typename RP>
__device__ __forceinline__ void split_chunk(const int *__restrict__ col_idx, const float *__restrict__ vals, int beg,
                                            int end, int d, float *__restrict__ SX, uint32_t bsplit,
                                            uint2 *__restrict__ region, RP cap, RP *s_count, const int *s_rp,
                                            const uint32_t *s_h, const float *s_sg, const uint8_t *s_map,
                                            uint64_t pol, uint64_t pol_last, int &bad) {
    const int lane = threadIdx.x & 31;
    for (int k0 = beg; k0 < end; k0 += 32 * kScatterUnroll) {
        int col[kScatterUnroll];
        float v[kScatterUnroll];
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const int k = k0 + u * 32 + lane;
            col[u] = -1;
            v[u] = 0.0f;
            if (k0 + u * 32 < end && k < end) {  // first test warp-uniform: empty slots cost nothing
                col[u] = ld_stream_i32(col_idx + k, pol);
                v[u] = ld_stream_f32(vals + k, pol);
            }
        }
        // The kScatterUnroll nonzeros of each lane: reduce or keep as a record.
        bool dfr[kScatterUnroll];
        uint32_t cell[kScatterUnroll];
        float x[kScatterUnroll];
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const int k = k0 + u * 32 + lane;
            dfr[u] = false;
            cell[u] = 0;
            x[u] = 0.0f;
            if (k < end) {
                int lo = 0;
                if (s_map != nullptr) {
                    lo = s_map[k - beg];
                } else {
#pragma unroll
                    for (int step = ROWS / 2; step > 0; step >>= 1)
                        if (s_rp[lo + step] <= k) lo += step;
                }
                const int j = col[u];
                const uint32_t hb = s_h[lo];
                if (static_cast<unsigned>(j) < static_cast<unsigned>(d)) {
                    cell[u] = hb * static_cast<uint32_t>(d) + static_cast<uint32_t>(j);
                    x[u] = s_sg[lo] * v[u];
                    if (hb < bsplit)
                        red_add_last(SX + cell[u], x[u], pol_last);
                    else
                        dfr[u] = true;
                } else {
                    bad = 1;
                }
            }
        }
        // One shared-memory atomic hands out the slots of all the step's records (one per
        // slot of 32 nonzeros cost 9 % more instructions in this pass).
        unsigned mask[kScatterUnroll];
        int total = 0;
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            mask[u] = __ballot_sync(0xffffffffu, dfr[u]);
            total += __popc(mask[u]);
        }
        if (total == 0) continue;  // warp-uniform
        RP at0 = 0;
        if (lane == 0) at0 = add_count(s_count, total);
        at0 = __shfl_sync(0xffffffffu, at0, 0);
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            if (dfr[u]) {
                const RP at = at0 + __popc(mask[u] & below);
                if (at < cap)
                    st_stream_u2(region + at, make_uint2(cell[u], __float_as_uint(x[u])), pol);
                else
                    bad = 1;
            }
            at0 += __popc(mask[u]);
        }
    }
    __syncwarp();
}

// Pass 1: CTA c takes rows [c R, min((c+1) R, n)) (R a multiple of kWarps ROWS) and the
// record slots row_ptr[c R] .. row_ptr[min((c+1) R, n)] - 1; it writes how many records
// it made to counts[c] (0 for a CTA whose region offsets are malformed).  With int
// offsets, five CTAs per SM (at most 48 registers): the pass is issue-bound, and 40
// warps per SM hide its load latency better than 32 (the 256-row form at 63 registers
// took 1.02 ms at the 2^26-row ladder shape, 0.91 ms at 48; at 40 registers and six
// CTAs, 0.93 ms).  The long long form keeps four, which it needs to avoid spills.
template <int ROWS, typename RP>
__global__ void __launch_bounds__(kThreads, sizeof(RP) == 4 ? 5 : 4)
split_pass_kernel(const RP *__restrict__ row_ptr, const int *__restrict__ col_idx, const float *__restrict__ vals,
                  int n, int d, uint32_t B, RP nnz, Key key, int64_t row_offset, float *__restrict__ SX,
                  uint32_t bsplit, int rows_per_cta, uint2 *__restrict__ records, RP *__restrict__ counts,
                  int *__restrict__ status) {
    __shared__ int s_rp[kWarps][ROWS + 1];
    __shared__ uint32_t s_h[kWarps][ROWS];
    __shared__ float s_sg[kWarps][ROWS];
    __shared__ uint8_t s_map[kWarps][kMapCap];
    __shared__ RP s_count;
    const int w = threadIdx.x >> 5;
    const int r0 = static_cast<int>(min(static_cast<int64_t>(n), static_cast<int64_t>(blockIdx.x) * rows_per_cta));
    const int r1 = static_cast<int>(min(static_cast<int64_t>(n), static_cast<int64_t>(r0) + rows_per_cta));
    const RP rec_lo = __ldg(row_ptr + r0);
    const RP rec_hi = __ldg(row_ptr + r1);
    if (rec_lo < 0 || rec_hi > nnz || rec_lo > rec_hi) {  // uniform over the CTA
        if (threadIdx.x == 0) {
            counts[blockIdx.x] = 0;
            atomicOr(status, kStatusBounds);
        }
        return;
    }
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const uint64_t pol = l2_evict_first_policy();
    const uint64_t pol_last = l2_evict_last_policy();
    int bad = 0;
    for (int first = r0 + w * ROWS; first < r1; first += kWarps * ROWS) {
        int beg, end;
        RP base;
        if (stage_chunk<ROWS, RP>(row_ptr, first, r1, nnz, B, key, row_offset, s_rp[w], s_h[w], s_sg[w], pol, beg,
                                  end, base, bad)) {
            const bool mapped = end - beg <= kMapCap;  // warp-uniform
            if (mapped) map_rows<ROWS>(s_rp[w], beg, s_map[w]);
            split_chunk<ROWS, RP>(col_idx + base, vals + base, beg, end, d, SX, bsplit, records + rec_lo,
                                  rec_hi - rec_lo, &s_count, s_rp[w], s_h[w], s_sg[w], mapped ? s_map[w] : nullptr,
                                  pol, pol_last, bad);
        }
    }
    if (bad) atomicOr(status, kStatusBounds);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s_count;
}

// ---- pass 1 with each chunk's nonzeros staged in shared memory ----------------------
// The same pass for int offsets and device-resident, 16-byte aligned col_idx and vals
// (B d <= 2^31).  Once a warp has its chunk's row offsets, one lane starts two bulk
// copies (cp.async.bulk, completion on a per-warp mbarrier) of the chunk's col_idx and
// vals into shared memory, from the 16-byte boundary at or below the first nonzero up
// to the last boundary at or below the end (the ragged tail of at most three nonzeros
// is loaded by plain loads); while the copies are in flight the warp hashes its rows and
// builds the row map, so the hashing hides the load latency, and the sweep then reads
// its operands from shared memory.  Each lane hashes four consecutive rows with one
// Philox call (the words of a call serve four rows), and a row's bucket and sign are
// kept as one word, h d with the sign in bit 31.  Chunks of more than kStageCap nonzeros (past the 16-byte
// boundary below the first) read their nonzeros from global memory as in the plain pass.
constexpr int kStageCap = 384;
constexpr uint32_t kStageWaitPolls = 1u << 22;  // bounded wait for a chunk's copies

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bulk copy global -> this CTA's shared memory (dst, src 16-byte aligned, bytes a
// multiple of 16), completing `bytes` transactions on the mbarrier at `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint32_t bar,
                                              uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(tc::smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}

// The sweep of a chunk whose nonzeros are not staged: nonzero k's column and value from
// global memory, its row from the row map (MAPPED) or by binary search over the offsets
// in s_rp.  Reduction or record as in split_chunk.
template <int ROWS, bool MAPPED>
__device__ __forceinline__ void split_sweep(const int *__restrict__ col_idx, const float *__restrict__ vals, int beg,
                                            int end, int d, float *__restrict__ SX, uint32_t lo_cell,
                                            uint2 *__restrict__ region, int cap, int *s_count, const uint32_t *s_hw,
                                            const uint8_t *s_map, const int *s_rp, uint64_t pol, uint64_t pol_last,
                                            int &bad) {
    const int lane = threadIdx.x & 31;
    for (int k0 = beg; k0 < end; k0 += 32 * kScatterUnroll) {
        int col[kScatterUnroll];
        float v[kScatterUnroll];
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const int k = k0 + u * 32 + lane;
            col[u] = -1;
            v[u] = 0.0f;
            if (k0 + u * 32 < end && k < end) {  // first test warp-uniform
                col[u] = ld_stream_i32(col_idx + k, pol);
                v[u] = ld_stream_f32(vals + k, pol);
            }
        }
        bool dfr[kScatterUnroll];
        uint32_t cell[kScatterUnroll];
        float x[kScatterUnroll];
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const int k = k0 + u * 32 + lane;
            dfr[u] = false;
            cell[u] = 0;
            x[u] = 0.0f;
            if (k < end) {
                int lo = 0;
                if constexpr (MAPPED) {
                    lo = s_map[k - beg];
                } else {
#pragma unroll
                    for (int step = ROWS / 2; step > 0; step >>= 1)
                        if (s_rp[lo + step] <= k) lo += step;
                }
                const int j = col[u];
                const uint32_t hw = s_hw[lo];
                if (static_cast<unsigned>(j) < static_cast<unsigned>(d)) {
                    const uint32_t base = hw & 0x7fffffffu;
                    cell[u] = base + static_cast<uint32_t>(j);
                    x[u] = __uint_as_float(__float_as_uint(v[u]) ^ (hw & 0x80000000u));  // sigma x, exactly
                    if (base < lo_cell)
                        red_add_last(SX + cell[u], x[u], pol_last);
                    else
                        dfr[u] = true;
                } else {
                    bad = 1;
                }
            }
        }
        unsigned mask[kScatterUnroll];
        int total = 0;
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            mask[u] = __ballot_sync(0xffffffffu, dfr[u]);
            total += __popc(mask[u]);
        }
        if (total == 0) continue;  // warp-uniform
        int at0 = 0;
        if (lane == 0) at0 = atomicAdd(s_count, total);
        at0 = __shfl_sync(0xffffffffu, at0, 0);
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            if (dfr[u]) {
                const int at = at0 + __popc(mask[u] & below);
                if (at < cap)
                    st_stream_u2(region + at, make_uint2(cell[u], __float_as_uint(x[u])), pol);
                else
                    bad = 1;
            }
            at0 += __popc(mask[u]);
        }
    }
    __syncwarp();
}

// The sweep of a staged chunk: nonzero k's column and value at s_col / s_val [k - kbase],
// its row from the row map.  Without branches: a slot past the chunk's end reads the last
// nonzero, and the reduction and the record store are predicated instructions (with
// branches around them the pass ran 15 % more instructions).
__device__ __forceinline__ void split_sweep_staged(const int *s_col, const int *s_val, int kbase, int beg, int end,
                                                   int d, float *__restrict__ SX, uint32_t lo_cell,
                                                   uint2 *__restrict__ region, int cap, int *s_count,
                                                   const uint32_t *s_hw, const uint8_t *s_map, uint64_t pol,
                                                   uint64_t pol_last, int &bad) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    for (int k0 = beg; k0 < end; k0 += 32 * kScatterUnroll) {
        bool dfr[kScatterUnroll];
        uint32_t cell[kScatterUnroll];
        float x[kScatterUnroll];
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const int k = k0 + u * 32 + lane;
            const bool live = k < end;
            const int kk = live ? k : end - 1;  // end > k0 >= beg
            const int j = s_col[kk - kbase];
            const float v = __int_as_float(s_val[kk - kbase]);
            const uint32_t hw = s_hw[s_map[kk - beg]];
            const bool ok = static_cast<unsigned>(j) < static_cast<unsigned>(d);
            bad |= (live && !ok) ? 1 : 0;
            const uint32_t base = hw & 0x7fffffffu;
            cell[u] = base + static_cast<uint32_t>(j);
            x[u] = __uint_as_float(__float_as_uint(v) ^ (hw & 0x80000000u));  // sigma x, exactly
            dfr[u] = live && ok && base >= lo_cell;
            red_add_last_if(live && ok && base < lo_cell, SX + cell[u], x[u], pol_last);
        }
        unsigned mask[kScatterUnroll];
        int total = 0;
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            mask[u] = __ballot_sync(0xffffffffu, dfr[u]);
            total += __popc(mask[u]);
        }
        if (total == 0) continue;  // warp-uniform
        int at0 = 0;
        if (lane == 0) at0 = atomicAdd(s_count, total);
        at0 = __shfl_sync(0xffffffffu, at0, 0);
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const int at = at0 + __popc(mask[u] & below);
            st_stream_u2_if(dfr[u] && at < cap, region + at, make_uint2(cell[u], __float_as_uint(x[u])), pol);
            bad |= (dfr[u] && at >= cap) ? 1 : 0;
            at0 += __popc(mask[u]);
        }
    }
    __syncwarp();
}

template <int ROWS>
__global__ void __launch_bounds__(kThreads, 5)
split_pass_staged_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col_idx,
                         const float *__restrict__ vals, int n, int d, uint32_t B, int nnz, Key key,
                         int64_t row_offset, float *__restrict__ SX, uint32_t lo_cell, int rows_per_cta,
                         uint2 *__restrict__ records, int *__restrict__ counts, int *__restrict__ status) {
    constexpr int R = ROWS / 32;
    static_assert(ROWS + 1 <= 2 * kStageCap && ROWS <= 256, "row offsets fit the staging area; rows fit a byte");
    __shared__ __align__(16) int s_stage[kWarps][2 * kStageCap];  // col_idx | vals, or the row offsets
    __shared__ uint32_t s_hw[kWarps][ROWS];
    __shared__ __align__(16) uint8_t s_map[kWarps][kMapCap];
    __shared__ __align__(8) uint64_t s_bar[kWarps];
    __shared__ int s_count;
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int r0 = static_cast<int>(min(static_cast<int64_t>(n), static_cast<int64_t>(blockIdx.x) * rows_per_cta));
    const int r1 = static_cast<int>(min(static_cast<int64_t>(n), static_cast<int64_t>(r0) + rows_per_cta));
    const int rec_lo = __ldg(row_ptr + r0);
    const int rec_hi = __ldg(row_ptr + r1);
    if (rec_lo < 0 || rec_hi > nnz || rec_lo > rec_hi) {  // uniform over the CTA
        if (threadIdx.x == 0) {
            counts[blockIdx.x] = 0;
            atomicOr(status, kStatusBounds);
        }
        return;
    }
    const uint32_t bar = tc::smem_u32(&s_bar[w]);
    if (lane == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const uint64_t pol = l2_evict_first_policy();
    uint2 *region = records + rec_lo;
    const int cap = rec_hi - rec_lo;
    const uint64_t pol_last = l2_evict_last_policy();
    uint32_t phase = 0;
    int bad = 0, late = 0;
    for (int first = r0 + w * ROWS; first < r1; first += kWarps * ROWS) {
        if (first != r0 + w * ROWS) {  // the previous chunk's shared-memory accesses before new copies
            tc::fence_proxy_async_smem();
            __syncwarp();
        }
        const int last = min(first + ROWS, r1);
        const int end = __ldg(row_ptr + last);
        int rp[R], nx[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = first + r * 32 + lane;
            rp[r] = i < last ? ld_stream_i32(row_ptr + i, pol) : end;
        }
        bool ordered = true;
#pragma unroll
        for (int r = 0; r < R; ++r) {  // nx[r]: the offset after row r*32 + lane
            const int up = __shfl_sync(0xffffffffu, r + 1 < R ? rp[r + 1 < R ? r + 1 : r] : end, 0);
            const int dn = __shfl_down_sync(0xffffffffu, rp[r], 1);
            nx[r] = lane == 31 ? up : dn;
            ordered &= rp[r] <= nx[r];
        }
        const int beg = __shfl_sync(0xffffffffu, rp[0], 0);
        if (end > nnz || beg < 0 || !__all_sync(0xffffffffu, ordered)) {  // malformed offsets: skip the chunk
            bad = 1;
            continue;
        }
        const int kbase = beg & ~3;
        const bool staged = end - kbase <= kStageCap;  // warp-uniform
        const bool mapped = end - beg <= kMapCap;
        int nb = 0;
        if (staged) {
            const int end_lo = end & ~3;
            nb = end_lo > kbase ? end_lo - kbase : 0;
            if (nb > 0 && lane == 0) {
                mbar_expect_tx(bar, 8u * static_cast<uint32_t>(nb));
                bulk_copy_g2s(&s_stage[w][0], col_idx + kbase, 4u * nb, bar, pol);
                bulk_copy_g2s(&s_stage[w][kStageCap], vals + kbase, 4u * nb, bar, pol);
            }
            const int k = max(kbase + nb, beg) + lane;  // the ragged tail: at most three nonzeros
            if (k < end) {
                s_stage[w][k - kbase] = ld_stream_i32(col_idx + k, pol);
                s_stage[w][kStageCap + k - kbase] = __float_as_int(ld_stream_f32(vals + k, pol));
            }
        } else if (!mapped) {  // row offsets for the binary search, in the unused staging area
#pragma unroll
            for (int r = 0; r < R; ++r) s_stage[w][r * 32 + lane] = rp[r];
            if (lane == 0) s_stage[w][ROWS] = end;
        }
        {  // while the copies are in flight: one Philox call per lane hashes four rows
            const int64_t g0 = row_offset + first;   // global row of chunk row 0
            const int64_t c0 = g0 >> 2;                // its call
            const int calls = static_cast<int>(((g0 + (last - first) - 1) >> 2) - c0 + 1);
#pragma unroll
            for (int t = 0; t < (ROWS + 127) / 128 + 1; ++t) {  // the last round only where g0 % 4 != 0
                const int c = t * 32 + lane;
                if (t * 32 < calls && c < calls) {
                    const uint4 wd = stream_words(key, static_cast<uint64_t>(c0 + c), kTagHash);
                    const int q0 = static_cast<int>(4 * (c0 + c) - g0);  // chunk row of the call's word 0
                    const uint32_t ws[4] = {wd.x, wd.y, wd.z, wd.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (q0 + j >= 0 && q0 + j < last - first)
                            s_hw[w][q0 + j] = __umulhi(ws[j], B) * static_cast<uint32_t>(d) | (ws[j] << 31);
                }
            }
        }
        if (mapped) {  // the row map: row starts marked, then a forward max-fill over the chunk
            const int cnt = end - beg;
            uint32_t *map32 = reinterpret_cast<uint32_t *>(s_map[w]);
            for (int q = lane; 4 * q < cnt; q += 32) map32[q] = 0u;
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; ++r)  // a non-empty row's start is no other non-empty row's
                if (rp[r] < nx[r]) s_map[w][rp[r] - beg] = static_cast<uint8_t>(r * 32 + lane);
            __syncwarp();
            const int span = (cnt + 31) >> 5;  // positions per lane
            const int p0 = lane * span;
            int run = 0;
            for (int i = 0; i < span; ++i)
                if (p0 + i < cnt) run = max(run, static_cast<int>(s_map[w][p0 + i]));
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {  // inclusive max-scan of the lanes' maxima
                const int y = __shfl_up_sync(0xffffffffu, run, o);
                if (lane >= o) run = max(run, y);
            }
            run = __shfl_up_sync(0xffffffffu, run, 1);
            if (lane == 0) run = 0;
            for (int i = 0; i < span; ++i)
                if (p0 + i < cnt) {
                    run = max(run, static_cast<int>(s_map[w][p0 + i]));
                    s_map[w][p0 + i] = static_cast<uint8_t>(run);
                }
        }
        __syncwarp();
        if (nb > 0) {
            if (!__all_sync(0xffffffffu, tc::mbar_wait_bounded(bar, phase, kStageWaitPolls))) {
                late = 1;  // give up on this warp's rows; let the copies land before the CTA ends
                tc::mbar_wait_bounded(bar, phase, kStageWaitPolls);
                break;
            }
            phase ^= 1u;
        }
        if (staged)
            split_sweep_staged(s_stage[w], s_stage[w] + kStageCap, kbase, beg, end, d, SX, lo_cell, region, cap,
                               &s_count, s_hw[w], s_map[w], pol, pol_last, bad);
        else if (mapped)
            split_sweep<ROWS, true>(col_idx, vals, beg, end, d, SX, lo_cell, region, cap, &s_count, s_hw[w], s_map[w],
                                    nullptr, pol, pol_last, bad);
        else
            split_sweep<ROWS, false>(col_idx, vals, beg, end, d, SX, lo_cell, region, cap, &s_count, s_hw[w], nullptr,
                                     s_stage[w], pol, pol_last, bad);
    }
    if (bad) atomicOr(status, kStatusBounds);
    if (late) atomicOr(status, kStatusTimeout);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s_count;
}

// Pass 2: CTA c reduces the counts[c] records of its region into SX.  First each CTA asks
// for its share of the upper half of SX (cells [lo_cell, cells)) to be brought into L2,
// where pass 1 left the lower half (a small gain: at the ladder size the pass is bound by
// the issue of its random reductions, not by their L2 misses).
template <typename RP>
__global__ void __launch_bounds__(kThreads)
replay_records_kernel(const RP *__restrict__ row_ptr, int n, int rows_per_cta, const uint2 *__restrict__ records,
                      const RP *__restrict__ counts, uint32_t lo_cell, uint32_t cells, float *__restrict__ SX) {
    if (threadIdx.x == 0 && cells > lo_cell) {
        const uint64_t share = (static_cast<uint64_t>(cells - lo_cell) + gridDim.x - 1) / gridDim.x;
        const uint64_t c0 = lo_cell + share * blockIdx.x;
        const uint64_t c1 = c0 + share < cells ? c0 + share : cells;
        if (c0 < c1) {
            const uintptr_t a = (reinterpret_cast<uintptr_t>(SX + c0) + 15) & ~static_cast<uintptr_t>(15);
            const uintptr_t e = reinterpret_cast<uintptr_t>(SX + c1) & ~static_cast<uintptr_t>(15);
            for (uintptr_t q = a; q < e; q += (1u << 20)) {  // at most 1 MB per hint
                const uint32_t len = static_cast<uint32_t>(e - q < (1u << 20) ? e - q : (1u << 20));
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(len) : "memory");
            }
        }
    }
    const int r0 = static_cast<int>(min(static_cast<int64_t>(n), static_cast<int64_t>(blockIdx.x) * rows_per_cta));
    const int r1 = static_cast<int>(min(static_cast<int64_t>(n), static_cast<int64_t>(r0) + rows_per_cta));
    const RP start = __ldg(row_ptr + r0);
    // records were written only inside [row_ptr[r0], row_ptr[r1]) (pass 1 set counts to 0
    // where these offsets were malformed)
    const RP cnt = min(counts[blockIdx.x], __ldg(row_ptr + r1) - start);
    if (cnt <= 0) return;
    const uint64_t pol = l2_evict_first_policy();
    const uint64_t pol_last = l2_evict_last_policy();
    constexpr int kInFlight = 4;  // record loads in flight per thread before their reductions
    RP i = threadIdx.x;
    for (; i + (kInFlight - 1) * kThreads < cnt; i += kInFlight * kThreads) {
        uint2 r[kInFlight];
#pragma unroll
        for (int u = 0; u < kInFlight; ++u) r[u] = ld_stream_u2(records + start + i + u * kThreads, pol);
#pragma unroll
        for (int u = 0; u < kInFlight; ++u)
            if (r[u].x < cells) red_add_last(SX + r[u].x, __uint_as_float(r[u].y), pol_last);
    }
    for (; i < cnt; i += kThreads) {
        const uint2 r = ld_stream_u2(records + start + i, pol);
        if (r.x < cells) red_add_last(SX + r.x, __uint_as_float(r.y), pol_last);
    }
}

// Chunk height of pass 1: as for the one-pass scatter (about 96 nonzeros per chunk), but
// 256 rows for rows of under 1.5 nonzeros: eight independent hashes per lane and fewer
// chunk boundaries (at 1.28 nonzeros per row, 0.976 ms against 1.010 ms with 128 rows).
int staged_rows(int n, int64_t nnz, int forced) {
    if (forced == 32 || forced == 64 || forced == 128 || forced == 256) return forced;
    const double per_row = n > 0 ? static_cast<double>(nnz) / n : 0.0;
    if (per_row * 32 >= 96.0) return 32;
    if (per_row * 64 >= 96.0) return 64;
    if (per_row >= 1.5) return 128;
    return 256;
}

// The bucket below which pass 1 reduces at once: for an SX past 60 % of the L2 (where the
// automatic choice takes this scatter), the largest that keeps that part of SX at 0.62 of
// the L2 (about 82 MB on GB300), and at least B/2 so that the part the records fill is no
// larger; for a smaller SX (the scatter forced) B/2.  Past that point the lower part's
// reductions leave the L2, short of it the records cost more than the direct reductions
// they replace.  Sketch times (memset and both passes) against the split, 2^26 rows at
// 1.28 nonzeros per row, with the evict-last reductions: 2^18 x 128 (134 MB of SX) 0.46 B
// 0.722 ms, 0.50 B 0.711, 0.54 B 0.696, 0.58 B 0.680, 0.62 B 0.681; 2^18 x 96 (101 MB)
// 0.60 B 0.565, 0.68 B 0.541, 0.76 B 0.516, 0.84 B 0.505.  The optimum's lower part is
// 80-85 MB in both (before the evict-last hint it was 67-70 MB: 0.50-0.52 B and 0.68 B).
uint32_t deferred_split(uint32_t B, int d) {
    const uint32_t half = B / 2;
    const int l2 = l2_bytes();
    const double sx = static_cast<double>(B) * d * sizeof(float);
    if (l2 <= 0 || d <= 0 || sx <= 0.6 * l2) return half;
    const uint64_t fit = static_cast<uint64_t>(0.62 * l2) / (static_cast<uint64_t>(d) * sizeof(float));
    return static_cast<uint32_t>(std::min<uint64_t>(B, std::max<uint64_t>(half, fit)));
}

}  // namespace

bool deferred_supported(int64_t B, int d) { return static_cast<uint64_t>(B) * static_cast<uint64_t>(d) < (1ull << 32); }

size_t sketch_deferred_scratch_bytes(int64_t nnz, int ctas) {
    return align256(static_cast<size_t>(nnz) * sizeof(uint2)) + align256(static_cast<size_t>(ctas) * sizeof(long long));
}

// CTAs of both passes: `ctas` when given, else one per sweep of the CTA's warps (kWarps
// chunks of H rows; at least the one-pass scatter's grid).  Regions are whole sweeps
// because a CTA lasts as long as its busiest warp, and many small CTAs leave no partial
// last wave (760 are resident at once): at the 2^26-row ladder shape the pair takes
// 0.916 ms with 1216 CTAs (1.6 waves), 0.898 ms with 10486 CTAs of 25 chunks (one warp
// with four, the others three), 0.842 ms with 32768 CTAs of one sweep and 0.840 ms with
// 16384 of two; at a quarter of its rows, 0.257 ms with 2048 CTAs of four sweeps and
// 0.246 ms with 8192 of one.
int sketch_deferred_ctas(int ctas, int64_t n, int64_t nnz, int rows) {
    if (ctas > 0) return ctas;
    const int64_t sweep = static_cast<int64_t>(kWarps) * staged_rows(static_cast<int>(n), nnz, rows);
    const int64_t g = std::max<int64_t>(sketch_default_ctas(), (n + sweep - 1) / sweep);
    return static_cast<int>(std::min<int64_t>(g, 1 << 26));
}

namespace {

// The staged pass 1 needs five CTAs' 41 KB of shared memory on an SM: ask for the
// largest shared-memory carveout.
template <int ROWS>
void launch_staged(int grid, const int *row_ptr, const int *col_idx, const float *vals, int n, int d, uint32_t B,
                   int nnz, Key key, int64_t row_offset, float *SX, uint32_t lo_cell, int rows_per_cta,
                   uint2 *records, int *counts, int *status, cudaStream_t stream) {
    static const cudaError_t attr = cudaFuncSetAttribute(
        split_pass_staged_kernel<ROWS>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    (void)attr;  // a preference only
    split_pass_staged_kernel<ROWS><<<grid, kThreads, 0, stream>>>(row_ptr, col_idx, vals, n, d, B, nnz, key,
                                                                  row_offset, SX, lo_cell, rows_per_cta, records,
                                                                  counts, status);
}

template <typename RP>
cudaError_t sketch_deferred(const RP *row_ptr, const int *col_idx, const float *vals, int n, int d, uint32_t B,
                            RP nnz, Key key, int64_t row_offset, float *SX, int *status, void *scratch, int ctas,
                            int rows, const EventPair *ev, cudaStream_t stream, bool clear, bool staged_ok) {
    cudaError_t e = clear ? cudaMemsetAsync(SX, 0, static_cast<size_t>(B) * d * sizeof(float), stream) : cudaSuccess;
    if (e != cudaSuccess || n == 0) return e;
    const int G = sketch_deferred_ctas(ctas, n, nnz, rows);
    const int H = staged_rows(n, nnz, rows);
    // whole sweeps of the CTA's warps (kWarps chunks of H rows each): a CTA lasts as long
    // as its busiest warp
    const int per = (n + G - 1) / G;
    const int sweep = kWarps * H;
    const int rows_per_cta = static_cast<int>((static_cast<int64_t>(per) + sweep - 1) / sweep * sweep);
    const int used = (n + rows_per_cta - 1) / rows_per_cta;
    uint2 *records = static_cast<uint2 *>(scratch);
    RP *counts = reinterpret_cast<RP *>(static_cast<char *>(scratch) + align256(static_cast<size_t>(nnz) * sizeof(uint2)));
    const uint32_t bsplit = deferred_split(B, d);
    record(ev, true, stream);
    if constexpr (sizeof(RP) == 4) {
        if (staged_ok && ((reinterpret_cast<uintptr_t>(col_idx) | reinterpret_cast<uintptr_t>(vals)) & 15u) == 0 &&
            static_cast<uint64_t>(B) * static_cast<uint64_t>(d) <= (1ull << 31)) {
            const uint32_t lo_cell = bsplit * static_cast<uint32_t>(d);
            switch (H) {
                case 256:
                    launch_staged<256>(used, row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset, SX, lo_cell,
                                       rows_per_cta, records, counts, status, stream);
                    break;
                case 128:
                    launch_staged<128>(used, row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset, SX, lo_cell,
                                       rows_per_cta, records, counts, status, stream);
                    break;
                case 64:
                    launch_staged<64>(used, row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset, SX, lo_cell,
                                      rows_per_cta, records, counts, status, stream);
                    break;
                default:
                    launch_staged<32>(used, row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset, SX, lo_cell,
                                      rows_per_cta, records, counts, status, stream);
                    break;
            }
            replay_records_kernel<RP><<<used, kThreads, 0, stream>>>(row_ptr, n, rows_per_cta, records, counts,
                                                                     lo_cell, B * static_cast<uint32_t>(d), SX);
            record(ev, false, stream);
            return cudaGetLastError();
        }
    }
    switch (H) {
        case 256:
            split_pass_kernel<256, RP><<<used, kThreads, 0, stream>>>(row_ptr, col_idx, vals, n, d, B, nnz, key,
                                                                      row_offset, SX, bsplit, rows_per_cta, records,
                                                                      counts, status);
            break;
        case 128:
            split_pass_kernel<128, RP><<<used, kThreads, 0, stream>>>(row_ptr, col_idx, vals, n, d, B, nnz, key,
                                                                      row_offset, SX, bsplit, rows_per_cta, records,
                                                                      counts, status);
            break;
        case 64:
            split_pass_kernel<64, RP><<<used, kThreads, 0, stream>>>(row_ptr, col_idx, vals, n, d, B, nnz, key,
                                                                     row_offset, SX, bsplit, rows_per_cta, records,
                                                                     counts, status);
            break;
        default:
            split_pass_kernel<32, RP><<<used, kThreads, 0, stream>>>(row_ptr, col_idx, vals, n, d, B, nnz, key,
                                                                     row_offset, SX, bsplit, rows_per_cta, records,
                                                                     counts, status);
            break;
    }
    replay_records_kernel<RP><<<used, kThreads, 0, stream>>>(row_ptr, n, rows_per_cta, records, counts,
                                                             bsplit * static_cast<uint32_t>(d),
                                                             B * static_cast<uint32_t>(d), SX);
    record(ev, false, stream);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sketch_csr_deferred(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                       uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, int *status,
                                       void *scratch, int ctas, int rows, const EventPair *ev, cudaStream_t stream,
                                       bool clear, bool staged_ok) {
    return sketch_deferred<int>(row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset, SX, status, scratch, ctas, rows,
                                ev, stream, clear, staged_ok);
}

cudaError_t launch_sketch_csr_deferred_i64(const long long *row_ptr, const int *col_idx, const float *vals, int n,
                                           int d, uint32_t B, long long nnz, Key key, int64_t row_offset, float *SX,
                                           int *status, void *scratch, int ctas, int rows, const EventPair *ev,
                                           cudaStream_t stream, bool clear) {
    return sketch_deferred<long long>(row_ptr, col_idx, vals, n, d, B, nnz, key, row_offset, SX, status, scratch, ctas,
                                      rows, ev, stream, clear, false);
}

}  // namespace cg

// cg_sketch_part.cu -- SX = S.X for CSR X by partitioning nonzeros by bucket range
// (Section 1.1: the O(nnz(X)) stage), for GPUs whose L2 reduction rate, not HBM
// bandwidth, limits a one-reduction-per-nonzero scatter.
//
// The B buckets are cut into P ranges ("slices") of SB buckets, SB = floor(32768 / d), so
// that one slice of SX (SB x d fp32 <= 128 KB) fits in shared memory.
//
// Pass 1 (partition): a CTA takes a tile of rows, hashes them once (h, sigma, slice),
//   and sweeps the tile's nonzeros in batches of up to kBatch.  For each batch it
//   histograms the records (slice, offset-in-slice = (h mod SB) d + j, sigma x) by
//   slice in shared memory, reserves one run per slice with a single global atomic,
//   sorts the batch by slice in shared memory and copies each run out contiguously:
//   one global atomic per (batch, slice) instead of one reduction per nonzero.
//   Records beyond a slice's capacity go to an overflow list.
// Pass 2 (accumulate): one CTA per slice zeroes the slice in shared memory, adds its
//   records with shared-memory atomics and writes the slice to SX once.
// Pass 3: the overflow list (normally empty) is reduced into SX with global atomics.
//
// Record order inside a slice depends on timing, so SX is reproducible only up to
// fp32 rounding order (as with the atomic scatter).
#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 1024;        // rows per tile
constexpr int kBatch = 4096;       // nonzeros per batch
constexpr int kPerThread = kBatch / kThreads;
constexpr int kAccThreads = 512;
constexpr int kSliceFloats = 32768;  // 128 KB

struct PartParams {
    int n, d, nnz;
    uint32_t B;
    int SB;        // buckets per slice
    int P;         // slices
    int64_t cap;   // records per slice region
    Key key;
    int64_t row_offset;
};

__global__ void __launch_bounds__(kThreads)
partition_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col_idx, const float *__restrict__ vals,
                 PartParams pp, int *__restrict__ fills, uint16_t *__restrict__ rkeys, float *__restrict__ rvals,
                 int *__restrict__ ocount, uint32_t *__restrict__ okeys, float *__restrict__ ovals,
                 float *__restrict__ cta_amax, int *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem[];
    int *s_rp = reinterpret_cast<int *>(smem);                    // kRows + 1
    uint32_t *s_meta = reinterpret_cast<uint32_t *>(s_rp + kRows + 4);  // kRows: base | sign<<15 | slice<<16
    int *s_cnt = reinterpret_cast<int *>(s_meta + kRows);          // P: records of the batch per slice
    int *s_off = s_cnt + pp.P;                                     // P: batch offset of each slice
    int *s_gpos = s_off + pp.P;                                    // P: region fill before the batch
    int *s_fill = s_gpos + pp.P;                                   // P: region fill so far
    uint16_t *s_rowid = reinterpret_cast<uint16_t *>(s_fill + pp.P);  // kBatch
    uint16_t *s_skey = s_rowid + kBatch;                           // kBatch
    uint16_t *s_spart = s_skey + kBatch;                           // kBatch
    float *s_sval = reinterpret_cast<float *>(s_spart + kBatch);   // kBatch
    __shared__ int s_warp_sum[kThreads / 32];
    __shared__ float s_warp_max[kThreads / 32];

    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    const int ntiles = (pp.n + kRows - 1) / kRows;
    int bad = 0;
    float amax = 0.0f;  // largest |x| this CTA saw (fixes the fixed-point scale of pass 2)

    for (int i = t; i < pp.P; i += kThreads) {
        s_cnt[i] = 0;
        s_fill[i] = 0;
    }

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int r0 = tile * kRows;
        const int nr = min(kRows, pp.n - r0);
        __syncthreads();  // previous tile's readers of s_rp / s_meta are done
        for (int r = t; r <= nr; r += kThreads) s_rp[r] = __ldg(row_ptr + r0 + r);
        for (int r = t; r < nr; r += kThreads) {
            uint32_t h;
            float sg;
            hash_sign(pp.key, static_cast<uint64_t>(pp.row_offset + r0 + r), pp.B, h, sg);
            const uint32_t sl = h / static_cast<uint32_t>(pp.SB);
            const uint32_t base = (h - sl * static_cast<uint32_t>(pp.SB)) * static_cast<uint32_t>(pp.d);
            s_meta[r] = base | (sg < 0.0f ? 0x8000u : 0u) | (sl << 16);
        }
        __syncthreads();
        const int kbeg = s_rp[0];
        const int kend = s_rp[nr];
        if (kbeg < 0 || kend > pp.nnz || kbeg > kend) {  // malformed row_ptr: skip the tile
            bad = 1;
            continue;
        }
        for (int kb = kbeg; kb < kend; kb += kBatch) {
            const int ke = min(kend, kb + kBatch);
            const int nb = ke - kb;
            // nonzero -> row index within the tile
            for (int r = t; r < nr; r += kThreads) {
                const int a = max(s_rp[r], kb), e = min(s_rp[r + 1], ke);
                for (int k = a; k < e; ++k) s_rowid[k - kb] = static_cast<uint16_t>(r);
            }
            __syncthreads();
            uint16_t mkey[kPerThread], mpart[kPerThread], mrank[kPerThread];
            float mval[kPerThread];
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) {
                const int idx = t + j * kThreads;
                mpart[j] = 0xFFFFu;
                if (idx < nb) {
                    const int k = kb + idx;
                    const int col = __ldg(col_idx + k);
                    const float v = __ldg(vals + k);
                    const uint32_t meta = s_meta[min(static_cast<int>(s_rowid[idx]), nr - 1)];
                    if (static_cast<unsigned>(col) < static_cast<unsigned>(pp.d)) {
                        const uint32_t sl = meta >> 16;
                        mkey[j] = static_cast<uint16_t>((meta & 0x7FFFu) + static_cast<uint32_t>(col));
                        mval[j] = (meta & 0x8000u) ? -v : v;
                        amax = fmaxf(amax, fabsf(v));
                        mpart[j] = static_cast<uint16_t>(sl);
                        mrank[j] = static_cast<uint16_t>(atomicAdd(&s_cnt[sl], 1));
                    } else {
                        bad = 1;
                    }
                }
            }
            __syncthreads();
            // exclusive scan of the slice counts; reserve one run per non-empty slice
            {
                const int per = (pp.P + kThreads - 1) / kThreads;
                const int i0 = t * per, i1 = min(pp.P, i0 + per);
                int sum = 0;
                for (int i = i0; i < i1; ++i) sum += s_cnt[i];
                int incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane == 31) s_warp_sum[warp] = incl;
                __syncthreads();
                int wbase = 0;
                for (int w = 0; w < warp; ++w) wbase += s_warp_sum[w];
                int run = wbase + incl - sum;
                for (int i = i0; i < i1; ++i) {
                    const int c = s_cnt[i];
                    s_off[i] = run;
                    s_gpos[i] = s_fill[i];  // this CTA's own region of slice i: no global atomics
                    s_fill[i] += c;
                    run += c;
                }
            }
            __syncthreads();
            // sort the batch by slice in shared memory
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) {
                if (mpart[j] != 0xFFFFu) {
                    const int pos = s_off[mpart[j]] + mrank[j];
                    s_skey[pos] = mkey[j];
                    s_sval[pos] = mval[j];
                    s_spart[pos] = mpart[j];
                }
            }
            __syncthreads();
            // copy out the runs (consecutive records of a slice go to consecutive slots)
            const int nvalid = s_off[pp.P - 1] + s_cnt[pp.P - 1];
            for (int i = t; i < nvalid; i += kThreads) {
                const int sl = s_spart[i];
                const int64_t dst = static_cast<int64_t>(s_gpos[sl]) + (i - s_off[sl]);
                if (dst < pp.cap) {
                    const int64_t at = (static_cast<int64_t>(blockIdx.x) * pp.P + sl) * pp.cap + dst;
                    rkeys[at] = s_skey[i];
                    rvals[at] = s_sval[i];
                } else {
                    const int o = atomicAdd(ocount, 1);
                    okeys[o] = static_cast<uint32_t>(sl) * static_cast<uint32_t>(pp.SB) * static_cast<uint32_t>(pp.d) +
                               s_skey[i];
                    ovals[o] = s_sval[i];
                }
            }
            __syncthreads();
            for (int i = t; i < pp.P; i += kThreads) s_cnt[i] = 0;
        }
    }
    __syncthreads();
    for (int i = t; i < pp.P; i += kThreads) fills[static_cast<int64_t>(blockIdx.x) * pp.P + i] = s_fill[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) s_warp_max[warp] = amax;
    __syncthreads();
    if (t == 0) {
        float mx = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, s_warp_max[w]);
        cta_amax[blockIdx.x] = mx;
    }
    if (bad) atomicOr(status, kStatusBounds);
}

// One CTA per slice: gather the slice's records from every pass-1 CTA's region,
// accumulate them in shared memory, write the slice once.
__global__ void __launch_bounds__(kAccThreads)
accumulate_kernel(PartParams pp, int nregions, const int *__restrict__ fills, const uint16_t *__restrict__ rkeys,
                  const float *__restrict__ rvals, float *__restrict__ SX, bool vec_out) {
    extern __shared__ __align__(16) float slice[];
    const int sl = blockIdx.x;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    const int b0 = sl * pp.SB;
    const int nbk = min(pp.SB, static_cast<int>(pp.B) - b0);
    const int nf = nbk * pp.d;
    for (int i = t; i < nf; i += kAccThreads) slice[i] = 0.0f;
    __syncthreads();
    // warp w takes regions c = w, w + 16, ...; 4 records per lane-step (regions start
    // at multiples of 8 records, so uint2 / float4 loads are aligned)
    for (int c = warp; c < nregions; c += kAccThreads / 32) {
        const int64_t reg = static_cast<int64_t>(c) * pp.P + sl;
        const int64_t n = min(static_cast<int64_t>(__ldg(fills + reg)), pp.cap);
        const uint16_t *keys = rkeys + reg * pp.cap;
        const float *vs = rvals + reg * pp.cap;
        const int64_t n4 = n >> 2;
        for (int64_t q = lane; q < n4; q += 32) {
            const uint2 k4 = __ldg(reinterpret_cast<const uint2 *>(keys) + q);
            const float4 v4 = __ldg(reinterpret_cast<const float4 *>(vs) + q);
            atomicAdd(&slice[k4.x & 0xFFFFu], v4.x);
            atomicAdd(&slice[k4.x >> 16], v4.y);
            atomicAdd(&slice[k4.y & 0xFFFFu], v4.z);
            atomicAdd(&slice[k4.y >> 16], v4.w);
        }
        for (int64_t i = (n4 << 2) + lane; i < n; i += 32) atomicAdd(&slice[keys[i]], vs[i]);
    }
    __syncthreads();
    float *dst = SX + static_cast<size_t>(b0) * pp.d;
    if (vec_out) {
        for (int i = t; i < (nf >> 2); i += kAccThreads)
            reinterpret_cast<float4 *>(dst)[i] = reinterpret_cast<const float4 *>(slice)[i];
    } else {
        for (int i = t; i < nf; i += kAccThreads) dst[i] = slice[i];
    }
}

// Deterministic variant of pass 2.  Every record value v is mapped to the integer
// q = round(v 2^F) and summed with 64-bit integer atomics, which are associative, so
// the integer sum is the same whatever order the records arrive in; SX is the single
// rounding (float)(sum 2^-F).  F = 62 - L - e with 2^e > max|x| (from pass 1) and
// 2^L > nnz, so no partial sum can leave the int64 range; each term is resolved to
// 2^(L+e-62) absolute (about 1e-11 of max|x| at nnz ~ 5e7), far finer than fp32
// accumulation.  Records of this slice that overflowed their region are read from
// the overflow list here as well.  Inputs must be finite.
__global__ void __launch_bounds__(kAccThreads)
accumulate_fixed_kernel(PartParams pp, int nregions, const int *__restrict__ fills,
                        const uint16_t *__restrict__ rkeys, const float *__restrict__ rvals,
                        const float *__restrict__ cta_amax, const int *__restrict__ ocount,
                        const uint32_t *__restrict__ okeys, const float *__restrict__ ovals, float *__restrict__ SX) {
    extern __shared__ __align__(16) unsigned long long acc[];
    __shared__ float s_max[kAccThreads / 32];
    const int sl = blockIdx.x;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    const int b0 = sl * pp.SB;
    const int nbk = min(pp.SB, static_cast<int>(pp.B) - b0);
    const int nf = nbk * pp.d;
    for (int i = t; i < nf; i += kAccThreads) acc[i] = 0ull;
    float mx = 0.0f;
    for (int c = t; c < nregions; c += kAccThreads) mx = fmaxf(mx, __ldg(cta_amax + c));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_max[warp] = mx;
    __syncthreads();
    mx = 0.0f;
    for (int w = 0; w < kAccThreads / 32; ++w) mx = fmaxf(mx, s_max[w]);
    int e = 0;
    if (mx > 0.0f) frexpf(mx, &e);  // mx < 2^e
    int L = 1;
    while ((1LL << L) <= static_cast<int64_t>(pp.nnz)) ++L;  // nnz < 2^L
    const int F = 62 - L - e;
    auto fixed = [&](float v) {
        return static_cast<unsigned long long>(__double2ll_rn(ldexp(static_cast<double>(v), F)));
    };
    for (int c = warp; c < nregions; c += kAccThreads / 32) {
        const int64_t reg = static_cast<int64_t>(c) * pp.P + sl;
        const int64_t n = min(static_cast<int64_t>(__ldg(fills + reg)), pp.cap);
        const uint16_t *keys = rkeys + reg * pp.cap;
        const float *vs = rvals + reg * pp.cap;
        for (int64_t i = lane; i < n; i += 32) atomicAdd(&acc[keys[i]], fixed(vs[i]));
    }
    const int no = *ocount;
    const uint32_t lo = static_cast<uint32_t>(b0) * static_cast<uint32_t>(pp.d);
    for (int i = t; i < no; i += kAccThreads) {
        const uint32_t k = okeys[i];
        if (k >= lo && k < lo + static_cast<uint32_t>(nf)) atomicAdd(&acc[k - lo], fixed(ovals[i]));
    }
    __syncthreads();
    float *dst = SX + static_cast<size_t>(b0) * pp.d;
    for (int i = t; i < nf; i += kAccThreads)
        dst[i] = __double2float_rn(ldexp(static_cast<double>(static_cast<long long>(acc[i])), -F));
}

__global__ void overflow_kernel(const int *__restrict__ ocount, const uint32_t *__restrict__ okeys,
                                const float *__restrict__ ovals, float *__restrict__ SX) {
    const int n = *ocount;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(SX + okeys[i], ovals[i]);
}

}  // namespace

// ---- host side --------------------------------------------------------------------

namespace {
int slice_floats(bool det) { return det ? kSliceFloats / 2 : kSliceFloats; }  // int64 slices are twice as wide
}  // namespace

bool partition_supported(const cg_plan &p) {
    const bool det = p.deterministic != 0;
    if (p.d > slice_floats(det)) return false;
    const int64_t SB = slice_floats(det) / p.d;
    const int64_t P = (p.B + SB - 1) / SB;
    return P <= 4096 && p.B * static_cast<int64_t>(p.d) < (1LL << 32) && p.n < (1LL << 31) - 1;
}

size_t partition_smem(int P) {
    return static_cast<size_t>(kRows + 4) * 4 + kRows * 4 + 4 * static_cast<size_t>(P) * 4 +
           static_cast<size_t>(kBatch) * (2 + 2 + 2 + 4);
}

PartLayout partition_layout(const cg_plan &p, int64_t nnz) {
    PartLayout L{};
    L.det = p.deterministic != 0;
    L.SB = slice_floats(L.det) / p.d;
    L.P = static_cast<int>((p.B + L.SB - 1) / L.SB);
    const int sms = num_sms() > 0 ? num_sms() : 148;
    int per_sm = static_cast<int>((200 * 1024) / (partition_smem(L.P) + 2048));
    per_sm = per_sm < 1 ? 1 : (per_sm > 2 ? 2 : per_sm);
    const int64_t ntiles = (p.n + kRows - 1) / kRows;
    L.G = static_cast<int>(ntiles < sms * per_sm ? (ntiles > 0 ? ntiles : 1) : sms * per_sm);
    // one region per (pass-1 CTA, slice); records beyond a region go to the overflow list
    const int64_t expect = (nnz + static_cast<int64_t>(L.P) * L.G - 1) / (static_cast<int64_t>(L.P) * L.G);
    L.cap = ((expect + expect / 4 + 64 + 7) / 8) * 8;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    L.gcount_off = take((static_cast<size_t>(L.G) * L.P + 1) * sizeof(int));  // fills + overflow counter
    L.amax_off = take(static_cast<size_t>(L.G) * sizeof(float));
    L.rkeys_off = take(static_cast<size_t>(L.G) * L.P * L.cap * sizeof(uint16_t));
    L.rvals_off = take(static_cast<size_t>(L.G) * L.P * L.cap * sizeof(float));
    L.okeys_off = take(static_cast<size_t>(nnz) * sizeof(uint32_t));
    L.ovals_off = take(static_cast<size_t>(nnz) * sizeof(float));
    L.bytes = off;
    return L;
}

cudaError_t launch_sketch_csr_partitioned(const int *row_ptr, const int *col_idx, const float *vals, int n, int d,
                                          uint32_t B, int nnz, Key key, int64_t row_offset, float *SX, int *status,
                                          void *scratch, const PartLayout &L, const EventPair *ev,
                                          cudaStream_t stream) {
    char *base = static_cast<char *>(scratch);
    int *fills = reinterpret_cast<int *>(base + L.gcount_off);
    int *ocount = fills + static_cast<size_t>(L.G) * L.P;
    float *amax = reinterpret_cast<float *>(base + L.amax_off);
    uint16_t *rkeys = reinterpret_cast<uint16_t *>(base + L.rkeys_off);
    float *rvals = reinterpret_cast<float *>(base + L.rvals_off);
    uint32_t *okeys = reinterpret_cast<uint32_t *>(base + L.okeys_off);
    float *ovals = reinterpret_cast<float *>(base + L.ovals_off);

    PartParams pp{n, d, nnz, B, L.SB, L.P, L.cap, key, row_offset};
    cudaError_t e = cudaMemsetAsync(ocount, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    const int sms = num_sms() > 0 ? num_sms() : 148;
    const size_t smem1 = partition_smem(L.P);
    if ((e = cudaFuncSetAttribute(partition_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem1))) != cudaSuccess)
        return e;
    const size_t smem2 = static_cast<size_t>(L.SB) * d * (L.det ? sizeof(unsigned long long) : sizeof(float));
    if (L.det) {
        if ((e = cudaFuncSetAttribute(accumulate_fixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem2))) != cudaSuccess)
            return e;
    } else if ((e = cudaFuncSetAttribute(accumulate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem2))) != cudaSuccess) {
        return e;
    }
    const bool vec_out = d % 4 == 0 && (reinterpret_cast<uintptr_t>(SX) & 15) == 0;
    record(ev, true, stream);
    // every pass-1 CTA runs (even without tiles) so that all region fills are written
    partition_kernel<<<L.G, kThreads, smem1, stream>>>(row_ptr, col_idx, vals, pp, fills, rkeys, rvals, ocount, okeys,
                                                       ovals, amax, status);
    if (L.det) {
        accumulate_fixed_kernel<<<L.P, kAccThreads, smem2, stream>>>(pp, L.G, fills, rkeys, rvals, amax, ocount,
                                                                     okeys, ovals, SX);
        record(ev, false, stream);
    } else {
        accumulate_kernel<<<L.P, kAccThreads, smem2, stream>>>(pp, L.G, fills, rkeys, rvals, SX, vec_out);
        record(ev, false, stream);
        overflow_kernel<<<sms, 256, 0, stream>>>(ocount, okeys, ovals, SX);
    }
    return cudaGetLastError();
}

}  // namespace cg

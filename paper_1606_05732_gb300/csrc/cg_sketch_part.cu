// cg_sketch_part.cu -- SX = S.X for CSR X by partitioning nonzeros by bucket range
// (Section 1.1: the O(nnz(X)) stage), for GPUs whose L2 reduction rate, not HBM
// bandwidth, limits a one-reduction-per-nonzero scatter.
//
// The B buckets are cut into P ranges ("slices") of SB buckets, SB = floor(32768 / d), so
// that one slice of SX (SB x d fp32 <= 128 KB) fits in shared memory.
//
// Pass 1 (partition): a persistent CTA takes tiles of rows, hashes each row once
//   (h, sigma, slice), and sorts each batch of the tile's records (slice,
//   offset-in-slice = (h mod SB) d + j, sigma x) by slice in shared memory -- one
//   shared-memory atomic per row reserves the row's run -- then appends each slice's
//   run to its own region of that slice: no global atomics, coalesced copies.
//   Records beyond a region's capacity go to an overflow list.
// Pass 2 (accumulate): one CTA per slice zeroes the slice in shared memory, gathers
//   the slice's records from every pass-1 CTA's region, adds them with shared-memory
//   atomics and writes the slice to SX once.
// Pass 3: the overflow list (normally empty) is reduced into SX with global atomics.
//
// Record order inside a slice depends on timing, so SX is reproducible only up to
// fp32 rounding order (as with the atomic scatter).
#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 1024;          // rows per tile
constexpr int kBatch = 4096;         // records per batch (a row never exceeds it: d <= kBatch)
constexpr int kAccThreads = 1024;
constexpr int kAccUnroll = 4;        // 16-byte loads in flight per lane in pass 2
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

// Pass 1.  Per tile of kRows rows: hash every row once.  Then per batch of rows whose
// nonzeros fit in kBatch: (A) each row reserves its run inside its slice with one
// shared-memory atomic (its length), (B) the slice counts are scanned into batch
// offsets and this CTA's region fills, (C) every nonzero is written, coalesced, to its
// sorted slot: the row's slot plus its position in the row, (D) the runs are copied
// to this CTA's region of each slice.
__global__ void __launch_bounds__(kThreads)
partition_kernel(const int *__restrict__ row_ptr, const int *__restrict__ col_idx, const float *__restrict__ vals,
                 PartParams pp, int *__restrict__ fills, uint16_t *__restrict__ rkeys, float *__restrict__ rvals,
                 int *__restrict__ ocount, uint32_t *__restrict__ okeys, float *__restrict__ ovals,
                 float *__restrict__ cta_amax, int *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem[];
    int *s_rp = reinterpret_cast<int *>(smem);                          // kRows + 1
    uint32_t *s_meta = reinterpret_cast<uint32_t *>(s_rp + kRows + 4);  // base | sign << 15 | slice << 16
    int *s_rdst = reinterpret_cast<int *>(s_meta + kRows);              // row's first slot in the batch
    int *s_cnt = s_rdst + kRows;                                        // P: records of the batch per slice
    int *s_sbase = s_cnt + pp.P;                                        // P: batch offset of each slice
    int *s_gpos = s_sbase + pp.P;                                       // P: region fill before the batch
    int *s_fill = s_gpos + pp.P;                                        // P: region fill so far
    uint16_t *s_rowid = reinterpret_cast<uint16_t *>(s_fill + pp.P);    // kBatch
    uint16_t *s_key = s_rowid + kBatch;                                 // kBatch
    uint16_t *s_part = s_key + kBatch;                                  // kBatch
    float *s_val = reinterpret_cast<float *>(s_part + kBatch);          // kBatch
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
        __syncthreads();  // the previous tile is finished with s_rp / s_meta
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
        if (s_rp[0] < 0 || s_rp[nr] > pp.nnz || s_rp[0] > s_rp[nr]) {  // malformed row_ptr: skip the tile
            bad = 1;
            continue;
        }
        int r = 0;
        while (r < nr) {
            // largest re with rp[re] - rp[r] <= kBatch (at least one row)
            int lo = r + 1, hi = nr;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_rp[mid] - s_rp[r] <= kBatch) lo = mid; else hi = mid - 1;
            }
            const int re = lo;
            const int kb = s_rp[r];
            const int ke = min(s_rp[re], kb + kBatch);
            const int nb = max(0, ke - kb);
            // (A) one run per row inside its slice
            for (int i = r + t; i < re; i += kThreads) {
                const int a = max(s_rp[i], kb), e = min(s_rp[i + 1], ke);
                if (s_rp[i + 1] < s_rp[i]) bad = 1;
                s_rdst[i] = atomicAdd(&s_cnt[s_meta[i] >> 16], max(0, e - a));
            }
            __syncthreads();
            // (B) batch offsets of the slices, region fills of this CTA
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
                int run = incl - sum;
                for (int w = 0; w < warp; ++w) run += s_warp_sum[w];
                for (int i = i0; i < i1; ++i) {
                    const int c = s_cnt[i];
                    s_sbase[i] = run;
                    s_gpos[i] = s_fill[i];
                    s_fill[i] += c;
                    s_cnt[i] = 0;
                    run += c;
                }
            }
            __syncthreads();
            // rows: absolute first slot; nonzero -> row map
            for (int i = r + t; i < re; i += kThreads) {
                s_rdst[i] += s_sbase[s_meta[i] >> 16];
                const int a = max(s_rp[i], kb), e = min(s_rp[i + 1], ke);
                for (int k = a; k < e; ++k) s_rowid[k - kb] = static_cast<uint16_t>(i);
            }
            __syncthreads();
            // (C) every nonzero to its sorted slot (coalesced loads)
            for (int idx = t; idx < nb; idx += kThreads) {
                const int k = kb + idx;
                const int i = min(max(static_cast<int>(s_rowid[idx]), r), re - 1);
                const uint32_t meta = s_meta[i];
                const int col = __ldg(col_idx + k);
                const float v = __ldg(vals + k);
                const int pos = s_rdst[i] + (k - max(s_rp[i], kb));
                if (static_cast<unsigned>(pos) >= static_cast<unsigned>(nb)) {
                    bad = 1;
                    continue;
                }
                if (static_cast<unsigned>(col) < static_cast<unsigned>(pp.d)) {
                    s_key[pos] = static_cast<uint16_t>((meta & 0x7FFFu) + static_cast<uint32_t>(col));
                    s_val[pos] = (meta & 0x8000u) ? -v : v;
                    amax = fmaxf(amax, fabsf(v));
                } else {  // a harmless record keeps every reserved slot written
                    bad = 1;
                    s_key[pos] = 0;
                    s_val[pos] = 0.0f;
                }
                s_part[pos] = static_cast<uint16_t>(meta >> 16);
            }
            __syncthreads();
            // (D) the runs, contiguous per slice, to this CTA's regions
            for (int i = t; i < nb; i += kThreads) {
                const int sl = min(static_cast<int>(s_part[i]), pp.P - 1);
                const int64_t dst = static_cast<int64_t>(s_gpos[sl]) + (i - s_sbase[sl]);
                if (dst >= 0 && dst < pp.cap) {
                    const int64_t at = (static_cast<int64_t>(blockIdx.x) * pp.P + sl) * pp.cap + dst;
                    rkeys[at] = s_key[i];
                    rvals[at] = s_val[i];
                } else {
                    const int o = atomicAdd(ocount, 1);
                    if (o < pp.nnz) {
                        okeys[o] = static_cast<uint32_t>(sl) * static_cast<uint32_t>(pp.SB) *
                                       static_cast<uint32_t>(pp.d) + s_key[i];
                        ovals[o] = s_val[i];
                    }
                }
            }
            __syncthreads();
            r = re;
        }
    }
    __syncthreads();
    // region fills, clamped to the capacity (the rest went to the overflow list)
    for (int i = t; i < pp.P; i += kThreads)
        fills[static_cast<int64_t>(blockIdx.x) * pp.P + i] =
            static_cast<int>(static_cast<int64_t>(s_fill[i]) < pp.cap ? static_cast<int64_t>(s_fill[i]) : pp.cap);
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

// Pass 2: one CTA per slice gathers the slice's records from every pass-1 CTA's
// region (warp per region, kAccUnroll 16-byte loads in flight per lane), adds them
// into the slice in shared memory and writes the slice to SX once.
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
    const unsigned nf = static_cast<unsigned>(nbk * pp.d);
    for (unsigned i = t; i < nf; i += kAccThreads) slice[i] = 0.0f;
    __syncthreads();
    for (int c = warp; c < nregions; c += kAccThreads / 32) {
        const int64_t reg = static_cast<int64_t>(c) * pp.P + sl;
        const int64_t n = min(static_cast<int64_t>(__ldg(fills + reg)), pp.cap);
        const uint16_t *keys = rkeys + reg * pp.cap;
        const float *vs = rvals + reg * pp.cap;
        const int64_t n4 = n >> 2;
        for (int64_t q0 = lane; q0 < n4; q0 += 32 * kAccUnroll) {
            uint2 k4[kAccUnroll];
            float4 v4[kAccUnroll];
#pragma unroll
            for (int u = 0; u < kAccUnroll; ++u) {
                const int64_t q = q0 + 32 * u;
                if (q < n4) {
                    k4[u] = __ldg(reinterpret_cast<const uint2 *>(keys) + q);
                    v4[u] = __ldg(reinterpret_cast<const float4 *>(vs) + q);
                }
            }
#pragma unroll
            for (int u = 0; u < kAccUnroll; ++u) {
                if (q0 + 32 * u < n4) {
                    const unsigned k0 = k4[u].x & 0xFFFFu, k1 = k4[u].x >> 16;
                    const unsigned k2 = k4[u].y & 0xFFFFu, k3 = k4[u].y >> 16;
                    if (k0 < nf) atomicAdd(&slice[k0], v4[u].x);
                    if (k1 < nf) atomicAdd(&slice[k1], v4[u].y);
                    if (k2 < nf) atomicAdd(&slice[k2], v4[u].z);
                    if (k3 < nf) atomicAdd(&slice[k3], v4[u].w);
                }
            }
        }
        for (int64_t i = (n4 << 2) + lane; i < n; i += 32) {
            const unsigned k = keys[i];
            if (k < nf) atomicAdd(&slice[k], vs[i]);
        }
    }
    __syncthreads();
    float *dst = SX + static_cast<size_t>(b0) * pp.d;
    if (vec_out) {
        for (unsigned i = t; i < (nf >> 2); i += kAccThreads)
            reinterpret_cast<float4 *>(dst)[i] = reinterpret_cast<const float4 *>(slice)[i];
    } else {
        for (unsigned i = t; i < nf; i += kAccThreads) dst[i] = slice[i];
    }
}

__global__ void overflow_kernel(const int *__restrict__ ocount, const uint32_t *__restrict__ okeys,
                                const float *__restrict__ ovals, float *__restrict__ SX) {
    const int n = *ocount;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(SX + okeys[i], ovals[i]);
}

}  // namespace

// ---- host side --------------------------------------------------------------------

bool partition_supported(const cg_plan &p) {
    if (p.d > kBatch) return false;
    const int64_t SB = kSliceFloats / p.d;
    const int64_t P = (p.B + SB - 1) / SB;
    return P <= 4096 && p.B * static_cast<int64_t>(p.d) < (1LL << 32) && p.n < (1LL << 31) - 1;
}

size_t partition_smem(int P) {
    return static_cast<size_t>(kRows + 4) * 4 + 2 * kRows * 4 + 4 * static_cast<size_t>(P) * 4 +
           static_cast<size_t>(kBatch) * (2 + 2 + 2 + 4);
}

PartLayout partition_layout(const cg_plan &p, int64_t nnz) {
    PartLayout L{};
    L.SB = kSliceFloats / p.d;
    L.P = static_cast<int>((p.B + L.SB - 1) / L.SB);
    const int sms = num_sms() > 0 ? num_sms() : 148;
    int per_sm = static_cast<int>((200 * 1024) / (partition_smem(L.P) + 2048));
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
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
    const size_t smem2 = static_cast<size_t>(L.SB) * d * sizeof(float);
    if ((e = cudaFuncSetAttribute(accumulate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem2))) != cudaSuccess)
        return e;
    const bool vec_out = d % 4 == 0 && (reinterpret_cast<uintptr_t>(SX) & 15) == 0;
    record(ev, true, stream);
    // every pass-1 CTA runs (even without tiles) so that all region fills are written
    partition_kernel<<<L.G, kThreads, smem1, stream>>>(row_ptr, col_idx, vals, pp, fills, rkeys, rvals, ocount, okeys,
                                                       ovals, amax, status);
    accumulate_kernel<<<L.P, kAccThreads, smem2, stream>>>(pp, L.G, fills, rkeys, rvals, SX, vec_out);
    record(ev, false, stream);
    overflow_kernel<<<sms, 256, 0, stream>>>(ocount, okeys, ovals, SX);
    return cudaGetLastError();
}

}  // namespace cg

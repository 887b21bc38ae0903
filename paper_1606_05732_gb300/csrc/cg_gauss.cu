// cg_gauss.cu -- stage 2 of the transform: Y = G.SX with G (m x B, i.i.d. N(0,1),
// Theorem 1) generated tile by tile in shared memory and never written to HBM
// (Section 1.1, the cost of G.(S.X), independent of n).
//
// FP32 FFMA path.  The contraction dimension B is split over the grid ("split-K"):
// CTA (s, bm, bn) owns a contiguous range of 32-column slabs of G, output rows
// [64 bm, 64 bm + 64) and output columns [BN bn, BN bn + BN).  Per slab it draws the
// 64 x 32 tile of G (one Philox call per 4 x 1 quad), stages the 32 x BN tile of
// SX, and accumulates a 4 x TN register tile per thread.  When the output block is
// smaller than 256 thread tiles, the surplus threads take interleaved k-indices of
// the slab and are summed in a fixed order at the end.  Each CTA writes one m x d
// partial; a second kernel sums the partials in a fixed order, so Y is
// bit-reproducible for a given grid.
#include <algorithm>

#include "cg_ffma.cuh"
#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr int kThreads = 256;
constexpr int kBM = 64;
constexpr int kKT = 32;

template <int TN>
__global__ void __launch_bounds__(kThreads)
contract_ffma_kernel(const float *__restrict__ SX, int m, int d, int64_t B, Key key, int64_t slabs_per_split,
                     bool vec_x, float *__restrict__ part) {
    __shared__ __align__(16) float raw[FfmaShape<TN>::kRawFloats];
    pdl_wait();  // SX comes from the scatter launched before
    const int64_t nslabs = (B + kKT - 1) / kKT;
    const int64_t s_begin = static_cast<int64_t>(blockIdx.x) * slabs_per_split;
    const int64_t s_end = min(nslabs, s_begin + slabs_per_split);
    ffma_block<TN, false>(SX, m, d, B, key, s_begin, s_end, blockIdx.y * kBM, blockIdx.z * 16 * TN, vec_x,
                          part + static_cast<size_t>(blockIdx.x) * m * d, raw);
}

// Y[o] = sum over s of part[s][o], for groups of 32 consecutive outputs (the lanes of a
// warp, coalesced).  W warps share a group: warp w sums the partials s = w, w + W, ...
// in increasing s, then the W warp sums are added in increasing w -- a fixed order for
// a given (nsplit, W), so Y is reproducible.  W follows nsplit (about four partials per
// warp), so that few splits over many outputs do not leave most warps idle.  CTAs hold
// 256 threads (8 / W groups) for W <= 8 and one group of W warps otherwise.  With
// tr_cols > 0 the rows x tr_cols result is stored transposed: output o = q tr_cols + j
// goes to Y[j (total / tr_cols) + q].
template <int W>
constexpr int red_threads() { return W >= 8 ? W * 32 : 256; }

template <int W>
__global__ void __launch_bounds__(red_threads<W>())
reduce_splits_kernel(const float *__restrict__ part, int nsplit, int64_t total, int tr_cols, float *__restrict__ Y) {
    pdl_wait();  // the partials come from the kernel launched before
    constexpr int kGroups = red_threads<W>() / (32 * W);
    __shared__ float red[W > 1 ? red_threads<W>() / 32 : 1][33];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = warp / W;
    const int sl = warp % W;
    const int64_t o = (static_cast<int64_t>(blockIdx.x) * kGroups + grp) * 32 + lane;
    float acc = 0.0f;
    if (o < total) {
        int s = sl;
        for (; s + 3 * W < nsplit; s += 4 * W) {
            const float a0 = __ldg(part + static_cast<size_t>(s) * total + o);
            const float a1 = __ldg(part + static_cast<size_t>(s + W) * total + o);
            const float a2 = __ldg(part + static_cast<size_t>(s + 2 * W) * total + o);
            const float a3 = __ldg(part + static_cast<size_t>(s + 3 * W) * total + o);
            acc += a0;
            acc += a1;
            acc += a2;
            acc += a3;
        }
        for (; s < nsplit; s += W) acc += __ldg(part + static_cast<size_t>(s) * total + o);
    }
    float r = acc;
    if (W > 1) {
        red[warp][lane] = acc;
        __syncthreads();
        if (sl != 0) return;
        r = red[grp * W][lane];
#pragma unroll
        for (int q = 1; q < W; ++q) r += red[grp * W + q][lane];
    }
    if (o < total) {
        if (tr_cols > 0)
            Y[(o % tr_cols) * (total / tr_cols) + o / tr_cols] = r;
        else
            Y[o] = r;
    }
}

// The split-K sum fused with Algorithm 1 step 3: CTA r owns row r of Y (m x d) and sums
// its splits in a fixed order -- the row's columns in chunks of 32 (one lane each), W
// warps per chunk with warp w taking partials s = w, w + W, ... in increasing s, the W
// sums then added in increasing w -- writes the row, and takes its argmax and argmin in
// the same pass, ties to the lowest column (strict comparisons in increasing column
// order, lowest index between equal values in the reductions).  A NaN is never chosen;
// a row with no ordered value reports column 0.
constexpr int kRowThreads = 1024;

__global__ void __launch_bounds__(kRowThreads)
reduce_rows_anchors_kernel(const float *__restrict__ part, int nsplit, int m, int d, float *__restrict__ Y,
                           int32_t *__restrict__ imax, int32_t *__restrict__ imin) {
    pdl_wait();  // the partials come from the kernel launched before
    constexpr int kWarps = kRowThreads / 32;
    __shared__ float red[kWarps][33];
    __shared__ float s_v[2][kWarps];
    __shared__ int s_j[2][kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x;
    const int64_t total = static_cast<int64_t>(m) * d;
    const int chunks = (d + 31) / 32;
    const int per_round = chunks < kWarps ? chunks : kWarps;  // chunks summed at once
    const int W = kWarps / per_round;                         // warps per chunk
    const int ci = warp / W, slot = warp % W;
    float vmax = -INFINITY, vmin = INFINITY;
    int jmax = d, jmin = d;
    for (int c0 = 0; c0 < chunks; c0 += per_round) {
        const int c = c0 + ci;
        const int j = c * 32 + lane;
        const bool live = ci < per_round && c < chunks && j < d;
        float acc = 0.0f;
        if (live) {
            const float *p = part + static_cast<int64_t>(r) * d + j;
            int s = slot;
            for (; s + 3 * W < nsplit; s += 4 * W) {
                const float a0 = __ldg(p + static_cast<int64_t>(s) * total);
                const float a1 = __ldg(p + static_cast<int64_t>(s + W) * total);
                const float a2 = __ldg(p + static_cast<int64_t>(s + 2 * W) * total);
                const float a3 = __ldg(p + static_cast<int64_t>(s + 3 * W) * total);
                acc += a0;
                acc += a1;
                acc += a2;
                acc += a3;
            }
            for (; s < nsplit; s += W) acc += __ldg(p + static_cast<int64_t>(s) * total);
        }
        red[warp][lane] = acc;
        __syncthreads();
        if (slot == 0 && live) {
            float y = red[warp][lane];
            for (int q = 1; q < W; ++q) y += red[warp + q][lane];
            Y[static_cast<int64_t>(r) * d + j] = y;
            if (y > vmax) {  // columns reach a lane in increasing order: the first wins ties
                vmax = y;
                jmax = j;
            }
            if (y < vmin) {
                vmin = y;
                jmin = j;
            }
        }
        __syncthreads();
    }
    // lanes, then warps: the larger (smaller) value, the lower column between equal ones
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float omax = __shfl_xor_sync(0xffffffffu, vmax, o);
        const int ojmax = __shfl_xor_sync(0xffffffffu, jmax, o);
        const float omin = __shfl_xor_sync(0xffffffffu, vmin, o);
        const int ojmin = __shfl_xor_sync(0xffffffffu, jmin, o);
        if (omax > vmax || (omax == vmax && ojmax < jmax)) {
            vmax = omax;
            jmax = ojmax;
        }
        if (omin < vmin || (omin == vmin && ojmin < jmin)) {
            vmin = omin;
            jmin = ojmin;
        }
    }
    if (lane == 0) {
        s_v[0][warp] = vmax;
        s_j[0][warp] = jmax;
        s_v[1][warp] = vmin;
        s_j[1][warp] = jmin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kWarps; ++w) {
            if (s_v[0][w] > vmax || (s_v[0][w] == vmax && s_j[0][w] < jmax)) {
                vmax = s_v[0][w];
                jmax = s_j[0][w];
            }
            if (s_v[1][w] < vmin || (s_v[1][w] == vmin && s_j[1][w] < jmin)) {
                vmin = s_v[1][w];
                jmin = s_j[1][w];
            }
        }
        imax[r] = jmax < d ? jmax : 0;
        imin[r] = jmin < d ? jmin : 0;
    }
}

template <int W>
cudaError_t launch_reduce_w(const float *partials, int nsplit, int64_t total, float *Y, cudaStream_t stream,
                            int tr_cols) {
    constexpr int kGroups = red_threads<W>() / (32 * W);
    const int64_t groups = (total + 31) / 32;
    const int64_t grid = (groups + kGroups - 1) / kGroups;
    const cudaError_t e = launch_after_previous(reduce_splits_kernel<W>, dim3(static_cast<unsigned>(grid)),
                                                dim3(red_threads<W>()), 0, stream, partials, nsplit, total, tr_cols, Y);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

int contract_splits(const cg_plan &p) {
    const int64_t nslabs = (p.B + kKT - 1) / kKT;
    if (p.ksplit > 0) return static_cast<int>(std::min<int64_t>(p.ksplit, nslabs));
    const int TN = p.d > 64 ? 8 : 4;
    const int64_t blocks = static_cast<int64_t>((p.m + kBM - 1) / kBM) * ((p.d + 16 * TN - 1) / (16 * TN));
    const int sms = num_sms() > 0 ? num_sms() : 148;
    // whole waves: as many CTAs as fit the GPU at once, never a partial second wave
    int per_sm = 3;
    if (num_sms() > 0) {
        static int resident[2] = {0, 0};
        int &r = resident[TN == 8 ? 1 : 0];
        if (r == 0)
            r = TN == 8 ? resident_ctas_per_sm(reinterpret_cast<const void *>(contract_ffma_kernel<8>), kThreads, 0, 0)
                        : resident_ctas_per_sm(reinterpret_cast<const void *>(contract_ffma_kernel<4>), kThreads, 0, 0);
        per_sm = r;
    }
    const int64_t target = static_cast<int64_t>(per_sm) * sms;
    int64_t s = target / blocks;
    s = std::max<int64_t>(1, std::min<int64_t>(s, nslabs));
    return static_cast<int>(s);
}

size_t contract_partials_bytes(const cg_plan &p) {
    const int splits = p.precision == CG_PREC_FP32 ? contract_splits(p) : contract_tc_splits(p);
    return static_cast<size_t>(splits) * p.m * p.d * sizeof(float);
}

cudaError_t launch_reduce_rows_anchors(const float *partials, int nsplit, int m, int d, float *Y, int32_t *imax,
                                      int32_t *imin, cudaStream_t stream) {
    if (m == 0) return cudaSuccess;
    const cudaError_t e = launch_after_previous(reduce_rows_anchors_kernel, dim3(static_cast<unsigned>(m)),
                                                dim3(kRowThreads), 0, stream, partials, nsplit, m, d, Y, imax, imin);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_reduce_splits(const float *partials, int nsplit, int64_t total, float *Y, cudaStream_t stream,
                                 int tr_cols) {
    if (total == 0) return cudaSuccess;
    const int per_warp = (nsplit + 3) / 4;  // warps per group: about four partials each
    if (per_warp <= 1) return launch_reduce_w<1>(partials, nsplit, total, Y, stream, tr_cols);
    if (per_warp <= 2) return launch_reduce_w<2>(partials, nsplit, total, Y, stream, tr_cols);
    if (per_warp <= 4) return launch_reduce_w<4>(partials, nsplit, total, Y, stream, tr_cols);
    if (per_warp <= 8) return launch_reduce_w<8>(partials, nsplit, total, Y, stream, tr_cols);
    if (per_warp <= 16) return launch_reduce_w<16>(partials, nsplit, total, Y, stream, tr_cols);
    return launch_reduce_w<32>(partials, nsplit, total, Y, stream, tr_cols);
}

cudaError_t launch_contract_ffma(const float *SX, int m, int d, int64_t B, Key key, int nsplit, float *partials,
                                 float *Y, const EventPair *ev, cudaStream_t stream, bool transpose, int32_t *imax,
                                 int32_t *imin) {
    const int64_t nslabs = (B + kKT - 1) / kKT;
    const int64_t per = (nslabs + nsplit - 1) / nsplit;
    const int used = static_cast<int>((nslabs + per - 1) / per);
    const int gm = (m + kBM - 1) / kBM;
    const bool vec_x = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(SX) & 15) == 0);
    record(ev, true, stream);
    cudaError_t e;
    if (d > 64) {
        const int gn = (d + 127) / 128;
        e = launch_after_previous(contract_ffma_kernel<8>, dim3(used, gm, gn), dim3(kThreads), 0, stream, SX, m, d, B, key,
                                  per, vec_x, partials);
    } else {
        const int gn = (d + 63) / 64;
        e = launch_after_previous(contract_ffma_kernel<4>, dim3(used, gm, gn), dim3(kThreads), 0, stream, SX, m, d, B, key,
                                  per, vec_x, partials);
    }
    record(ev, false, stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (imax != nullptr) return launch_reduce_rows_anchors(partials, used, m, d, Y, imax, imin, stream);
    return launch_reduce_splits(partials, used, static_cast<int64_t>(m) * d, Y, stream, transpose ? d : 0);
}

}  // namespace cg

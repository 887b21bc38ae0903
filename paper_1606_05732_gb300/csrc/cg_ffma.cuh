// cg_ffma.cuh -- the FP32 FFMA contraction of one output block over a range of K
// slabs (G generated tile by tile in shared memory, never stored), shared by the
// split-K contraction kernel and the batched persistent kernel.
#pragma once
#include "cg_internal.cuh"

namespace cg {

constexpr int kFfmaThreads = 256;
constexpr int kFfmaBM = 64;
constexpr int kFfmaKT = 32;

template <int TN>
struct FfmaShape {
    static constexpr int BN = 16 * TN;
    static constexpr int kMainFloats = kFfmaKT * (kFfmaBM + BN);
    static constexpr int kRedFloats = kFfmaThreads * 4 * TN;
    static constexpr int kRawFloats = kMainFloats > kRedFloats ? kMainFloats : kRedFloats;
};

template <bool COHERENT>
__device__ __forceinline__ float4 load4(const float4 *p) {
    if (COHERENT) return __ldcg(p);
    return __ldg(p);
}
template <bool COHERENT>
__device__ __forceinline__ float load1(const float *p) {
    if (COHERENT) return __ldcg(p);
    return __ldg(p);
}

// Partial contraction of one output block over a range of K slabs:
//   out[r, c] = sum over b in slabs [s_begin, s_end) x 32 of G[r, b] SX[b, c]
// for r in [m0, m0 + 64), c in [n0, n0 + 16 TN), written (not accumulated) into the
// m x d row-major array `out`.  Called by all 256 threads of a CTA; `raw` is the
// CTA's shared buffer of FfmaShape<TN>::kRawFloats floats.  With COHERENT the SX
// loads bypass the non-coherent read-only path (SX written earlier in the same launch).
template <int TN, bool COHERENT>
__device__ __forceinline__ void ffma_block(const float *__restrict__ SX, int m, int d, int64_t B, Key key,
                                           int64_t s_begin, int64_t s_end, int m0, int n0, bool vec_x,
                                           float *__restrict__ out, float *raw) {
    constexpr int BN = 16 * TN;
    constexpr int kRawFloats = FfmaShape<TN>::kRawFloats;
    (void)kRawFloats;
    float(*sG)[kFfmaBM] = reinterpret_cast<float(*)[kFfmaBM]>(raw);                // [kFfmaKT][kFfmaBM]
    float(*sX)[BN] = reinterpret_cast<float(*)[BN]>(raw + kFfmaKT * kFfmaBM);      // [kFfmaKT][BN]

    const int bm = min(kFfmaBM, m - m0);
    const int bn = min(BN, d - n0);
    const int mt = (bm + 3) >> 2;
    const int nt = (bn + TN - 1) / TN;
    const int tiles = mt * nt;
    const int kg = max(1, kFfmaThreads / tiles);
    const int t = threadIdx.x;
    const int tile = t % tiles;
    const int grp = t / tiles;
    const bool active = grp < kg;
    const int ti = tile % mt;
    const int tj = tile / mt;
    const uint64_t groups = static_cast<uint64_t>((m + 3) >> 2);
    const int g0 = m0 >> 2;

    float acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;


    for (int64_t sl = s_begin; sl < s_end; ++sl) {
        const int64_t b0 = sl * kFfmaKT;
        // G[m0 .. m0+4mt, b0 .. b0+kFfmaKT): quads of four rows of one column.
        for (int q = t; q < mt * kFfmaKT; q += kFfmaThreads) {
            const int gl = q % mt;
            const int kk = q / mt;
            const int64_t b = b0 + kk;
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (b < B) z = gauss_quad(key, kTagG, groups, static_cast<uint64_t>(b), static_cast<uint64_t>(g0 + gl));
            *reinterpret_cast<float4 *>(&sG[kk][4 * gl]) = z;
        }
        // SX[b0 .. b0+kFfmaKT, n0 .. n0+bn)
        if (vec_x) {
            constexpr int BQ = BN / 4;
            for (int q = t; q < kFfmaKT * BQ; q += kFfmaThreads) {
                const int kk = q / BQ;
                const int cq = q % BQ;
                const int64_t b = b0 + kk;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (b < B && 4 * cq < bn) x = load4<COHERENT>(reinterpret_cast<const float4 *>(SX + b * d + n0) + cq);
                *reinterpret_cast<float4 *>(&sX[kk][4 * cq]) = x;
            }
        } else {
            for (int q = t; q < kFfmaKT * BN; q += kFfmaThreads) {
                const int kk = q / BN;
                const int cc = q % BN;
                const int64_t b = b0 + kk;
                sX[kk][cc] = (b < B && cc < bn) ? load1<COHERENT>(SX + b * d + n0 + cc) : 0.0f;
            }
        }
        __syncthreads();
        if (active) {
            for (int kk = grp; kk < kFfmaKT; kk += kg) {
                const float4 a = *reinterpret_cast<const float4 *>(&sG[kk][4 * ti]);
                float bv[TN];
#pragma unroll
                for (int j4 = 0; j4 < TN / 4; ++j4) {
                    const float4 x = *reinterpret_cast<const float4 *>(&sX[kk][TN * tj + 4 * j4]);
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
        }
        __syncthreads();
    }

    // Sum the k-groups in a fixed order (group 0 + group 1 + ...).
    if (kg > 1) {
        float *red = raw;
        if (active && grp > 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) red[((grp - 1) * tiles + tile) * 4 * TN + i * TN + j] = acc[i][j];
        }
        __syncthreads();
        if (grp == 0) {
            for (int g = 1; g < kg; ++g)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] += red[((g - 1) * tiles + tile) * 4 * TN + i * TN + j];
        }
    }
    if (grp == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = m0 + 4 * ti + i;
            if (r >= m) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int c = n0 + TN * tj + j;
                if (TN * tj + j < bn) out[static_cast<size_t>(r) * d + c] = acc[i][j];
            }
        }
    }
}

}  // namespace cg

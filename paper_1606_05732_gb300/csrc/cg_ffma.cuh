// cg_ffma.cuh -- the FP32 FFMA contraction of one output block over a range of K
// slabs (G generated tile by tile in shared memory, never stored), shared by the
// split-K contraction kernel and the batched persistent kernel.  It computes the
// second factor of T.X = G.(S.X): Y = G.SX with G the m x B matrix of i.i.d. N(0,1)
// entries (Section 2, Theorem 1; Algorithm 1 step 2).
#pragma once
#include "cg_internal.cuh"

namespace cg {

constexpr int kFfmaThreads = 256;
constexpr int kFfmaBM = 64;
constexpr int kFfmaKT = 32;

template <int TN>
struct FfmaShape {
    static constexpr int BN = 16 * TN;
    static constexpr int kMainFloats = kFfmaKT * (kFfmaBM + 2 * BN);  // G tile + two SX tiles
    static constexpr int kRedFloats = kFfmaThreads * 4 * TN;
    static constexpr int kRawFloats = kMainFloats > kRedFloats ? kMainFloats : kRedFloats;
};

// 16-byte asynchronous copy global -> shared through L2 (coherent with writes made
// earlier in the same launch); `bytes` = 0 fills the 16 bytes with zeros instead.
__device__ __forceinline__ void cp_async16(float *dst, const float *src, int bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <bool COHERENT>
__device__ __forceinline__ float load1(const float *p) {
    if (COHERENT) return __ldcg(p);
    return __ldg(p);
}

// Partial contraction of one output block over a range of K slabs:
//   out[r, c] = sum over b in slabs [s_begin, s_end) x 32 of G[r, b] SX[b, c]
// for r in [m0, m0 + 64), c in [n0, n0 + 16 TN), written (not accumulated) into the
// m x d row-major array `out`.  Called by all 256 threads of a CTA; `raw` is the
// CTA's shared buffer of FfmaShape<TN>::kRawFloats floats (16-byte aligned).  With
// vec_x (d % 4 == 0, SX 16-byte aligned) the SX tile of slab s + 1 is copied with
// cp.async into the second buffer while slab s's G tile is drawn and multiplied;
// otherwise it is loaded synchronously (with COHERENT through L2, for SX written
// earlier in the same launch).
// UNROLLED: when one or two k-groups cover the block (256 or 128 thread tiles), the kk
// loop runs with constant bounds and fully unrolled (shared-memory offsets become
// immediates; the FP32 contraction at m = d = 128 went from 0.276 to 0.252 ms, the
// 96-instance batch from 1.367 to 1.338 ms although its 64-register budget spills 4 bytes).
template <int TN, bool COHERENT, bool UNROLLED = true>
__device__ __forceinline__ void ffma_block(const float *__restrict__ SX, int m, int d, int64_t B, Key key,
                                           int64_t s_begin, int64_t s_end, int m0, int n0, bool vec_x,
                                           float *__restrict__ out, float *raw) {
    constexpr int BN = 16 * TN;
    constexpr int BQ = BN / 4;
    float(*sG)[kFfmaBM] = reinterpret_cast<float(*)[kFfmaBM]>(raw);  // [kFfmaKT][kFfmaBM]
    float *sXb = raw + kFfmaKT * kFfmaBM;                              // two [kFfmaKT][BN] tiles

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
    const int gquads = mt * kFfmaKT;

    // SX[b0 .. b0+kFfmaKT, n0 .. n0+bn) of slab sl into tile `buf`, asynchronously.
    auto stage_x_async = [&](int64_t sl, int buf) {
        float(*dst)[BN] = reinterpret_cast<float(*)[BN]>(sXb + buf * kFfmaKT * BN);
        const int64_t b0 = sl * kFfmaKT;
        for (int q = t; q < kFfmaKT * BQ; q += kFfmaThreads) {
            const int kk = q / BQ;
            const int cq = q % BQ;
            const int64_t b = b0 + kk;
            const bool in = b < B && 4 * cq < bn;
            cp_async16(&dst[kk][4 * cq], in ? SX + b * d + n0 + 4 * cq : SX, in ? 16 : 0);
        }
        cp_async_commit();
    };

    float acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;

    if (vec_x && s_begin < s_end) stage_x_async(s_begin, 0);
    int buf = 0;
    for (int64_t sl = s_begin; sl < s_end; ++sl, buf ^= 1) {
        const int64_t b0 = sl * kFfmaKT;
        // The other tile was read in the previous slab, before its closing barrier.
        if (vec_x && sl + 1 < s_end) stage_x_async(sl + 1, buf ^ 1);
        // G[m0 .. m0+4mt, b0 .. b0+kFfmaKT): quads of four rows of one column, two
        // independent quads per step.
        for (int q0 = t; q0 < gquads; q0 += 2 * kFfmaThreads) {
            const int q1 = q0 + kFfmaThreads;
            const int kk0 = q0 / mt, kk1 = q1 / mt;
            const int gl0 = q0 - kk0 * mt, gl1 = q1 - kk1 * mt;
            float4 z0 = make_float4(0.f, 0.f, 0.f, 0.f), z1 = z0;
            if (b0 + kk0 < B)
                z0 = gauss_quad(key, kTagG, groups, static_cast<uint64_t>(b0 + kk0), static_cast<uint64_t>(g0 + gl0));
            if (q1 < gquads && b0 + kk1 < B)
                z1 = gauss_quad(key, kTagG, groups, static_cast<uint64_t>(b0 + kk1), static_cast<uint64_t>(g0 + gl1));
            *reinterpret_cast<float4 *>(&sG[kk0][4 * gl0]) = z0;
            if (q1 < gquads) *reinterpret_cast<float4 *>(&sG[kk1][4 * gl1]) = z1;
        }
        float(*sX)[BN] = reinterpret_cast<float(*)[BN]>(sXb + buf * kFfmaKT * BN);
        if (vec_x) {
            if (sl + 1 < s_end)
                cp_async_wait<1>();  // this slab's tile has landed (the next may be in flight)
            else
                cp_async_wait<0>();
        } else {
            for (int q = t; q < kFfmaKT * BN; q += kFfmaThreads) {
                const int kk = q / BN;
                const int cc = q % BN;
                const int64_t b = b0 + kk;
                sX[kk][cc] = (b < B && cc < bn) ? load1<COHERENT>(SX + b * d + n0 + cc) : 0.0f;
            }
        }
        __syncthreads();
        // acc += G[4 ti .. 4 ti + 4, kk] x SX[kk, TN tj .. TN tj + TN)
        auto step = [&](int kk) {
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
        };
        // Threads past the last k-group (grp >= kg: the block has fewer than 256 tiles and
        // 256 is not a multiple of their count) own no k-index and take no step.
        if (active) {
            if (UNROLLED && kg == 1) {  // one k-group: every k-index of the slab
#pragma unroll
                for (int kk = 0; kk < kFfmaKT; ++kk) step(kk);
            } else if (UNROLLED && kg == 2) {  // two k-groups: k-indices grp, grp + 2, ...
#pragma unroll
                for (int i = 0; i < kFfmaKT / 2; ++i) step(grp + 2 * i);
            } else {
                for (int kk = grp; kk < kFfmaKT; kk += kg) step(kk);
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
        // 16-byte stores where the thread's TN columns are all in range and rows of `out`
        // start 16-byte aligned
        const bool vec = TN * tj + TN <= bn && (d & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(out) | ((n0 + TN * tj) * 4u)) & 15) == 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = m0 + 4 * ti + i;
            if (r >= m) continue;
            float *o = out + static_cast<size_t>(r) * d + n0 + TN * tj;
            if (vec) {
#pragma unroll
                for (int j = 0; j < TN; j += 4)
                    *reinterpret_cast<float4 *>(o + j) = make_float4(acc[i][j], acc[i][j + 1], acc[i][j + 2], acc[i][j + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    if (TN * tj + j < bn) o[j] = acc[i][j];
            }
        }
    }
}

}  // namespace cg

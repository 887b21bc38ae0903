// cg_rng.cuh -- device-side random streams of the CountGauss transform.
//
// The paper asks for independent uniform buckets and fair signs for the CountSketch
// S (Section 1.1; Section 7) and i.i.d. unit-variance Gaussians for G and G~
// (Section 2, Theorem 1).  Here they are pure functions of (seed, index), so no
// random matrix is ever stored:
//   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key (lo32(seed), hi32(seed)),
//   counter (lo32(idx), hi32(idx), tag, 0).
//   tag 0, idx = floor(i / 4) for global row i, w = word i mod 4 of the call:
//     h(i) = floor(w * B / 2^32),  sigma(i) = bit0(w) ? -1 : +1  (four rows per call).
//   uniform u(w) = (2 (w >> 9) + 1) 2^-24, exact in fp32, never 0 or 1.
//   Box-Muller quadruple of one call: sqrt(-2 ln u0) (cos, sin)(2 pi u1),
//                                     sqrt(-2 ln u2) (cos, sin)(2 pi u3).
//   Entry (r, c) of an R x C Gaussian with tag t: lane r%4 of the call at
//   idx = c * ceil(R/4) + r/4 (tag 1: G, m x B; tag 2: G~, m x n).
// The fp32 Box-Muller calls CUDA's logf, sqrtf and sincospif (exact argument
// reduction of 2u); nothing here is compiled with fast-math.
#pragma once
#include <cstdint>

namespace cg {

constexpr uint32_t kTagHash = 0u;
constexpr uint32_t kTagG = 1u;
constexpr uint32_t kTagGTilde = 2u;

struct Key {
    uint32_t k0, k1;
};

__host__ __device__ __forceinline__ Key make_key(uint64_t seed) {
    return Key{static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)};
}

// Ten Philox4x32 rounds: two 32x32->64 products per round (multipliers
// 0xD2511F53, 0xCD9E8D57), key bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85.
__device__ __forceinline__ uint4 philox10(uint4 c, Key k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        // one 32x32->64 product per multiplier: high and low halves from the same product
        const uint64_t pa = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t pb = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        c = make_uint4(static_cast<uint32_t>(pb >> 32) ^ c.y ^ k.k0, static_cast<uint32_t>(pb),
                       static_cast<uint32_t>(pa >> 32) ^ c.w ^ k.k1, static_cast<uint32_t>(pa));
        k.k0 += 0x9E3779B9u;
        k.k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 stream_words(Key k, uint64_t idx, uint32_t tag) {
    return philox10(make_uint4(static_cast<uint32_t>(idx), static_cast<uint32_t>(idx >> 32), tag, 0u), k);
}

// Word q of the ten-round output: nine full rounds, then of the last round only the
// product and mix that word q takes (words 0 and 1 from the product of c.z, 2 and 3 from
// that of c.x), so one output word costs one product less and keeps fewer registers.
__device__ __forceinline__ uint32_t philox10_word(uint4 c, Key k, uint32_t q) {
#pragma unroll
    for (int round = 0; round < 9; ++round) {
        const uint64_t pa = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t pb = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        c = make_uint4(static_cast<uint32_t>(pb >> 32) ^ c.y ^ k.k0, static_cast<uint32_t>(pb),
                       static_cast<uint32_t>(pa >> 32) ^ c.w ^ k.k1, static_cast<uint32_t>(pa));
        k.k0 += 0x9E3779B9u;
        k.k1 += 0xBB67AE85u;
    }
    const bool upper = q >= 2u;
    const uint64_t p = static_cast<uint64_t>(upper ? 0xD2511F53u : 0xCD9E8D57u) * (upper ? c.x : c.z);
    const uint32_t mix = upper ? (c.w ^ k.k1) : (c.y ^ k.k0);
    return (q & 1u) ? static_cast<uint32_t>(p) : (static_cast<uint32_t>(p >> 32) ^ mix);
}

// The hash word of global row i: word i mod 4 of the tag-0 call at floor(i / 4).
__device__ __forceinline__ uint32_t hash_word(Key k, uint64_t row) {
    const uint64_t g = row >> 2;
    return philox10_word(make_uint4(static_cast<uint32_t>(g), static_cast<uint32_t>(g >> 32), kTagHash, 0u), k,
                         static_cast<uint32_t>(row) & 3u);
}

// Bucket and sign of global row i for a sketch with B rows (B < 2^32).
__device__ __forceinline__ void hash_sign(Key k, uint64_t row, uint32_t B, uint32_t &h, float &s) {
    const uint32_t w = hash_word(k, row);
    h = __umulhi(w, B);
    s = (w & 1u) ? -1.0f : 1.0f;
}

// u(w) = (2 (w >> 9) + 1) 2^-24, formed without an integer-to-float conversion: the float
// with exponent 0 and mantissa w >> 9 is 1 + (w >> 9) 2^-23 exactly, and subtracting
// 1 - 2^-24 is exact (the operands are within a factor of two), leaving (2 (w >> 9) + 1) 2^-24.
__device__ __forceinline__ float uniform24(uint32_t w) {
    return __uint_as_float(0x3F800000u | (w >> 9)) - 0.999999940395355224609375f;  // 1 - 2^-24
}

__device__ __forceinline__ float4 box_muller4(uint4 w) {
    const float u0 = uniform24(w.x), u1 = uniform24(w.y);
    const float u2 = uniform24(w.z), u3 = uniform24(w.w);
    const float r01 = sqrtf(-2.0f * logf(u0));
    const float r23 = sqrtf(-2.0f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s3, &c3);
    return make_float4(r01 * c1, r01 * s1, r23 * c3, r23 * s3);
}

// The same quadruple with CUDA's fast intrinsics, for Gaussians that are rounded to bf16
// or e4m3 right away: __logf, rsqrtf, and __sincosf of 2 pi (u - 1/2), which stays in
// [-pi, pi] where __sincosf is accurate (cos and sin of 2 pi u are the negated values).
// Relative error about 1e-6, far below a bf16 or e4m3 rounding.
__device__ __forceinline__ float4 box_muller4_fast(uint4 w) {
    const float u0 = uniform24(w.x), u1 = uniform24(w.y);
    const float u2 = uniform24(w.z), u3 = uniform24(w.w);
    const float q01 = -2.0f * __logf(u0), q23 = -2.0f * __logf(u2);  // > 0: u < 1
    const float r01 = q01 * rsqrtf(q01), r23 = q23 * rsqrtf(q23);
    float s1, c1, s3, c3;
    __sincosf(6.28318530717958647692f * (u1 - 0.5f), &s1, &c1);
    __sincosf(6.28318530717958647692f * (u3 - 0.5f), &s3, &c3);
    return make_float4(-r01 * c1, -r01 * s1, -r23 * c3, -r23 * s3);
}

// The four Gaussian entries (4g .. 4g+3, c) of an R x C Gaussian, groups = ceil(R/4);
// with FAST the fast-intrinsic quadruple of the same words.
template <bool FAST = false>
__device__ __forceinline__ float4 gauss_quad(Key k, uint32_t tag, uint64_t groups, uint64_t c, uint64_t g) {
    const uint4 w = stream_words(k, c * groups + g, tag);
    return FAST ? box_muller4_fast(w) : box_muller4(w);
}

}  // namespace cg

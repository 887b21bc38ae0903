// cg_gauss_tc.cu -- stage 2 of the transform, Y = G.SX, on the 5th-generation tensor
// cores: G (i.i.d. N(0,1), Theorem 1) is drawn by Box-Muller straight into shared
// memory in the MMA operand layout and never touches HBM; SX is staged through
// registers (fp32 -> bf16); tcgen05.mma accumulates in fp32 in tensor memory.
//
// Precisions (the "precision ladder"):
//   bf16     Y ~= hi(G) . hi(SX)
//   bf16x3   Y ~= hi(G).hi(SX) + hi(G).lo(SX) + lo(G).hi(SX), with lo(x) = bf16(x - hi(x));
//            the dropped lo.lo term is about 2^-16 of each product.
//
// Tile: M = 128 rows of G (zero rows past m), N = NT columns of SX (64/128/256, zero
// columns past d), K = 64 per slab (one 128-byte swizzle atom of bf16).  The CTA owns a
// contiguous range of slabs of B (split-K); 2-stage ring: while the tensor core runs the
// MMAs of slab i, the 256 threads draw G and convert SX for slab i+1.  Completion of a
// stage's MMAs is signalled by tcgen05.commit on that stage's mbarrier.  The epilogue
// reads the 128 x NT accumulator from TMEM and writes one fp32 partial per CTA; the
// partials are summed in a fixed order by reduce_splits_kernel.
//
// Every wait is bounded (about two seconds of SM clock); on expiry the kernel sets
// the timeout bit of the status word, stops issuing, waits (bounded) for MMAs in
// flight, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "cg_internal.cuh"
#include "cg_tc.cuh"

namespace cg {

namespace {

constexpr int kThreads = 256;
constexpr int kM = 128;
constexpr int kBK = 64;
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ bool wait_stage(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void split_bf16(float x, float &hi, float &lo) {
    hi = __bfloat162float(__float2bfloat16_rn(x));
    lo = x - hi;
}

// L2 prefetch of rows [r0, r0 + rows) of the row-major B x d fp32 SX (clipped to B):
// one contiguous range, trimmed to whole 16-byte units and to 1 MB; skipped if SX is not
// 16-byte aligned.
__device__ __forceinline__ void prefetch_rows(const float *SX, int64_t r0, int rows, int64_t B, int d) {
    if (r0 >= B || (reinterpret_cast<uintptr_t>(SX) & 15) != 0) return;
    const int64_t r1 = r0 + rows < B ? r0 + rows : B;
    const uint64_t first = static_cast<uint64_t>(r0) * d * sizeof(float);
    const uint64_t last = static_cast<uint64_t>(r1) * d * sizeof(float);
    const uint64_t a = (first + 15) & ~15ull;
    uint64_t b = last & ~15ull;
    if (b > a + (1ull << 20)) b = a + (1ull << 20);  // at most 1 MB per hint
    if (b > a) tc::prefetch_l2_bulk(reinterpret_cast<const char *>(SX) + a, static_cast<uint32_t>(b - a));
}

template <int NT, bool SPLIT3>
struct Cfg {
    static constexpr uint32_t kA = kM * kBK * 2;  // 16 KB
    static constexpr uint32_t kB = NT * kBK * 2;  // NT x 128 B
    static constexpr uint32_t kStage = SPLIT3 ? 2 * (kA + kB) : (kA + kB);
    static constexpr uint32_t kSmem = 2 * kStage + 1024;
    static constexpr uint32_t kTmemCols = NT < 32 ? 32 : NT;
};

// Threads of the bf16 kernel: 512 for the split form with N tiles of 128 or more (its two
// operand sets leave room for one CTA per SM, so the Gaussians are drawn by 16 warps),
// else 256 (several CTAs per SM).
template <int NT, bool SPLIT3>
constexpr int bf16_threads() { return SPLIT3 && NT >= 128 ? 512 : 256; }

// Resident CTAs per SM the register budget is sized for: three for the single-bf16 form
// with N tiles of at most 128 (its stages fit three times in shared memory), else one.
template <int NT, bool SPLIT3>
constexpr int bf16_min_ctas() { return !SPLIT3 && NT <= 128 ? 3 : 1; }

template <int NT, bool SPLIT3>
__global__ void __launch_bounds__(bf16_threads<NT, SPLIT3>(), bf16_min_ctas<NT, SPLIT3>())
contract_tc_bf16_kernel(const float *__restrict__ SX, int m, int d, int64_t B, Key key, int64_t slabs_per_cta,
                        float *__restrict__ part, int *__restrict__ status) {
    pdl_wait();  // SX comes from the scatter launched before
    using C = Cfg<NT, SPLIT3>;
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int t = threadIdx.x;
    const int warp = t >> 5;
    const int lane = t & 31;
    const uint32_t raw = tc::smem_u32(dsmem);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *gbase = dsmem + (sbase - raw);

    const int m0 = blockIdx.z * kM;
    const int n0 = blockIdx.y * NT;
    const int bn = min(NT, d - n0);
    const uint64_t groups = static_cast<uint64_t>((m + 3) >> 2);
    const int64_t nslabs = (B + kBK - 1) / kBK;
    const int64_t s_begin = static_cast<int64_t>(blockIdx.x) * slabs_per_cta;
    const int64_t s_end = min(nslabs, s_begin + slabs_per_cta);
    const int nmine = s_end > s_begin ? static_cast<int>(s_end - s_begin) : 0;

    if (t == 0) {
        tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
        tc::mbar_init(tc::smem_u32(&mbar[1]), 1);
        tc::fence_mbar_init();
        abort_flag = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), C::kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kM, NT);

    int issued = 0;  // slabs whose MMAs were issued (thread 0's view == everyone's)
    for (int it = 0; it < nmine; ++it) {
        const int s = it & 1;
        const int64_t k0 = (s_begin + it) * kBK;
        // the SX rows of the next slab into L2 while this slab's G tile is drawn
        if (t == 0 && it + 1 < nmine) prefetch_rows(SX, k0 + kBK, kBK, B, d);
        if (it >= 2 && !wait_stage(tc::smem_u32(&mbar[s]), static_cast<uint32_t>(((it >> 1) - 1) & 1))) {
            atomicOr(status, kStatusTimeout);
            abort_flag = 1;
        }
        uint8_t *stage = gbase + s * C::kStage;
        uint8_t *a_hi = stage;
        uint8_t *b_hi = stage + C::kA;
        uint8_t *a_lo = stage + C::kA + C::kB;
        uint8_t *b_lo = a_lo + C::kA;

        // B^T = SX[k0 .. k0+64, n0 .. n0+NT) stored [n][k]: its loads are issued first, so
        // that they are in flight while the G tile is drawn, and stored after it.
        constexpr int kThr = bf16_threads<NT, SPLIT3>();
        constexpr int kBq = (NT * (kBK / 4) + kThr - 1) / kThr;  // quads of SX per thread
        float xs[kBq][4];
#pragma unroll
        for (int j = 0; j < kBq; ++j) {
            const int q = t + j * kThr;
            const int nl = q % NT;
            const int kq = q / NT;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t krow = k0 + 4 * kq + c;
                xs[j][c] = (q < NT * (kBK / 4) && krow < B && nl < bn) ? __ldg(SX + krow * d + n0 + nl) : 0.0f;
            }
        }
        // A = G[m0 .. m0+128, k0 .. k0+64): blocks of 4 rows (one Philox call) x 4 columns.
        for (int q = t; q < (kM / 4) * (kBK / 4); q += bf16_threads<NT, SPLIT3>()) {
            const int gl = q >> 4;
            const int kq = q & 15;
            const uint64_t g = static_cast<uint64_t>((m0 >> 2) + gl);
            float z[4][4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t col = k0 + 4 * kq + c;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                // one bf16 per entry: G drawn with the fast intrinsics; the split form keeps the
                // fp32-accurate G its two bf16 terms resolve
                if (g < groups && col < B) v = gauss_quad<!SPLIT3>(key, kTagG, groups, static_cast<uint64_t>(col), g);
                z[c][0] = v.x;
                z[c][1] = v.y;
                z[c][2] = v.z;
                z[c][3] = v.w;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = 4 * gl + r;
                const bool live = m0 + row < m;
                float h[4], l[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) split_bf16(live ? z[c][r] : 0.0f, h[c], l[c]);
                const uint32_t off = tc::sw128_bf16(row, 4 * kq);
                *reinterpret_cast<uint2 *>(a_hi + off) = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
                if (SPLIT3)
                    *reinterpret_cast<uint2 *>(a_lo + off) =
                        make_uint2(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]));
            }
        }
#pragma unroll
        for (int j = 0; j < kBq; ++j) {
            const int q = t + j * kThr;
            if (q >= NT * (kBK / 4)) break;
            const int nl = q % NT;
            const int kq = q / NT;
            float h[4], l[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) split_bf16(xs[j][c], h[c], l[c]);
            const uint32_t off = tc::sw128_bf16(nl, 4 * kq);
            *reinterpret_cast<uint2 *>(b_hi + off) = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
            if (SPLIT3)
                *reinterpret_cast<uint2 *>(b_lo + off) = make_uint2(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]));
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (abort_flag) break;
        if (t == 0) {
            tc::fence_after_sync();
            const uint32_t sa_hi = sbase + s * C::kStage;
            const uint32_t sb_hi = sa_hi + C::kA;
            const uint32_t sa_lo = sa_hi + C::kA + C::kB;
            const uint32_t sb_lo = sa_lo + C::kA;
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks) {
                const uint32_t koff = 32u * ks;  // 16 bf16 of K = 32 bytes inside the swizzle atom
                const uint64_t ad = tc::smem_desc_sw128(sa_hi + koff, 16, 1024);
                const uint64_t bd = tc::smem_desc_sw128(sb_hi + koff, 16, 1024);
                tc::mma_bf16(tmem, ad, bd, kIdesc, (it > 0 || ks > 0) ? 1u : 0u);
                if (SPLIT3) {
                    tc::mma_bf16(tmem, ad, tc::smem_desc_sw128(sb_lo + koff, 16, 1024), kIdesc, 1u);
                    tc::mma_bf16(tmem, tc::smem_desc_sw128(sa_lo + koff, 16, 1024), bd, kIdesc, 1u);
                }
            }
            tc::mma_commit(tc::smem_u32(&mbar[s]));
        }
        issued = it + 1;
    }

    // Wait for the last committed stage (commits complete in order).
    bool ok = !abort_flag;
    if (issued > 0) {
        const int last = issued - 1;
        if (!wait_stage(tc::smem_u32(&mbar[last & 1]), static_cast<uint32_t>((last >> 1) & 1))) {
            atomicOr(status, kStatusTimeout);
            ok = false;
        }
    }
    tc::fence_after_sync();
    __syncthreads();

    // Epilogue: warps w, w+4, w+8, ... share TMEM lanes 32(w%4) .. +32 and split the
    // columns (at least 32 each: bf16_threads gives 512 threads only for NT >= 128).
    constexpr int kGroups = bf16_threads<NT, SPLIT3>() / 128;
    constexpr int kCols = NT / kGroups;
    static_assert(kCols % 32 == 0, "epilogue column split");
    const int quad = warp & 3;
    const int grp = warp >> 2;
    const int row = quad * 32 + lane;
    const int grow = m0 + row;
    float *out = part + static_cast<size_t>(blockIdx.x) * m * d;
    // whole 16-byte groups of a row when the tile is full and rows start 16-byte aligned
    const bool vec = bn == NT && (d & 3) == 0 && ((reinterpret_cast<uintptr_t>(out) | (n0 * 4u)) & 15) == 0;
    for (int c0 = grp * kCols; c0 < (grp + 1) * kCols; c0 += 32) {
        uint32_t r[32];
        tc::tmem_ld_32x32b_x32(tmem + (static_cast<uint32_t>(quad * 32) << 16) + static_cast<uint32_t>(c0), r);
        tc::tmem_ld_wait();
        if (grow < m) {
            float *o = out + static_cast<size_t>(grow) * d + n0 + c0;
            const bool good = ok && issued > 0;
            if (vec) {
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    *reinterpret_cast<float4 *>(o + j) =
                        good ? make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                           __uint_as_float(r[j + 3]))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < bn) o[j] = good ? __uint_as_float(r[j]) : 0.0f;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, C::kTmemCols);
}

template <int NT, bool SPLIT3>
cudaError_t launch_tc(const float *SX, int m, int d, int64_t B, Key key, int nsplit, float *partials, int *status,
                      const EventPair *ev, cudaStream_t stream) {
    using C = Cfg<NT, SPLIT3>;
    const int64_t nslabs = (B + kBK - 1) / kBK;
    const int64_t per = (nslabs + nsplit - 1) / nsplit;
    const int used = static_cast<int>((nslabs + per - 1) / per);
    const uint32_t smem = C::kSmem;
    cudaError_t e = cudaFuncSetAttribute(contract_tc_bf16_kernel<NT, SPLIT3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    dim3 grid(used, (d + NT - 1) / NT, (m + kM - 1) / kM);
    record(ev, true, stream);
    e = launch_after_previous(contract_tc_bf16_kernel<NT, SPLIT3>, grid, dim3(bf16_threads<NT, SPLIT3>()), smem, stream,
                              SX, m, d, B, key, per, partials, status);
    record(ev, false, stream);
    return e != cudaSuccess ? e : cudaGetLastError();
}

int tc_nt(int d) { return d <= 64 ? 64 : (d <= 128 ? 128 : 256); }

// ---- FP8-E4M3 with per-tile scales -------------------------------------------------
// K slab = one 128-byte swizzle atom of e4m3 = 128 columns of G / rows of SX.  Each
// slab t is its own scaled tile: G is quantised as e4m3(64 z) (|64 z| <= 369 < 448,
// exact power-of-two scale), the slab of SX as e4m3(x / s_t) with s_t = absmax / 448
// over the 128 x NT tile.  Slab t's MMAs write a fresh fp32 tile D_t into TMEM buffer
// t % 2; the epilogue warps then add D_t * s_t / 64 into registers while the tensor
// core runs slab t + 1.  With SPLIT3 each operand is also split, x = hi + lo with
// hi = e4m3(x), lo = e4m3(x - hi), and hi.hi + hi.lo + lo.hi is accumulated.
constexpr int kBK8 = 128;
constexpr float kGScale = 64.0f;
constexpr float kE4M3Max = 448.0f;

__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float e) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, e), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

__device__ __forceinline__ void split_e4m3(float x, float &hi, float &lo) {
    const __nv_fp8_e4m3 h(x);
    hi = static_cast<float>(h);
    lo = x - hi;
}

template <int NT, bool SPLIT3>
struct Cfg8 {
    static constexpr uint32_t kA = kM * kBK8;   // 16 KB
    static constexpr uint32_t kB = NT * kBK8;   // NT x 128 B
    static constexpr uint32_t kStage = SPLIT3 ? 2 * (kA + kB) : (kA + kB);
    static constexpr uint32_t kSmem = 2 * kStage + 1024;
    static constexpr uint32_t kTmemCols = 2 * NT;  // two fp32 tiles
    static constexpr int kQuadsPerThread = NT * (kBK8 / 4) / kThreads;
};

template <int NT, bool SPLIT3>
__global__ void __launch_bounds__(kThreads, 1)
contract_tc_fp8_kernel(const float *__restrict__ SX, int m, int d, int64_t B, Key key, int64_t slabs_per_cta,
                       float *__restrict__ part, int *__restrict__ status) {
    pdl_wait();  // SX comes from the scatter launched before
    using C = Cfg8<NT, SPLIT3>;
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ float warp_max[kThreads / 32];
    __shared__ float tile_scale[2];

    const int t = threadIdx.x;
    const int warp = t >> 5;
    const int lane = t & 31;
    const uint32_t raw = tc::smem_u32(dsmem);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *gbase = dsmem + (sbase - raw);

    const int m0 = blockIdx.z * kM;
    const int n0 = blockIdx.y * NT;
    const int bn = min(NT, d - n0);
    const uint64_t groups = static_cast<uint64_t>((m + 3) >> 2);
    const int64_t nslabs = (B + kBK8 - 1) / kBK8;
    const int64_t s_begin = static_cast<int64_t>(blockIdx.x) * slabs_per_cta;
    const int64_t s_end = min(nslabs, s_begin + slabs_per_cta);
    const int nmine = s_end > s_begin ? static_cast<int>(s_end - s_begin) : 0;

    if (t == 0) {
        tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
        tc::mbar_init(tc::smem_u32(&mbar[1]), 1);
        tc::fence_mbar_init();
        abort_flag = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), C::kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t kIdesc = tc::idesc_e4m3_f32(kM, NT);

    const int quad = warp & 3;
    const int half = warp >> 2;
    const int row = quad * 32 + lane;
    float acc[NT / 2];
#pragma unroll
    for (int j = 0; j < NT / 2; ++j) acc[j] = 0.0f;

    // Add tile `tile` (TMEM buffer tile % 2) times its scale into acc.
    auto drain = [&](int tile) {
        const int b = tile & 1;
        // warp-uniform outcome: tcgen05.ld below is .sync.aligned
        const bool good = __all_sync(0xffffffffu, wait_stage(tc::smem_u32(&mbar[b]),
                                                              static_cast<uint32_t>((tile >> 1) & 1)));
        if (!good) {
            if (lane == 0) atomicOr(status, kStatusTimeout);
            abort_flag = 1;
            return;
        }
        tc::fence_after_sync();
        const float sc = tile_scale[b] * (1.0f / kGScale);
#pragma unroll
        for (int c = 0; c < NT / 2; c += 32) {
            uint32_t r[32];
            tc::tmem_ld_32x32b_x32(tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                                       static_cast<uint32_t>(b * NT + half * (NT / 2) + c),
                                   r);
            tc::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[c + j] = fmaf(__uint_as_float(r[j]), sc, acc[c + j]);
        }
    };

    int issued = 0;
    for (int it = 0; it < nmine; ++it) {
        const int s = it & 1;
        const int64_t k0 = (s_begin + it) * kBK8;
        // the SX rows of the next slab into L2 while this slab's G tile is drawn
        if (t == 0 && it + 1 < nmine) prefetch_rows(SX, k0 + kBK8, kBK8, B, d);
        uint8_t *stage = gbase + s * C::kStage;
        uint8_t *a_hi = stage;
        uint8_t *b_hi = stage + C::kA;
        uint8_t *a_lo = stage + C::kA + C::kB;
        uint8_t *b_lo = a_lo + C::kA;

        // SX slab into registers and its absmax.
        float xb[C::kQuadsPerThread][4];
        float amax = 0.0f;
#pragma unroll
        for (int j = 0; j < C::kQuadsPerThread; ++j) {
            const int q = t + j * kThreads;
            const int nl = q % NT;
            const int kq = q / NT;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t krow = k0 + 4 * kq + c;
                const float x = (krow < B && nl < bn) ? __ldg(SX + krow * d + n0 + nl) : 0.0f;
                xb[j][c] = x;
                amax = fmaxf(amax, fabsf(x));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        if (lane == 0) warp_max[warp] = amax;

        // G slab: blocks of 4 rows (one Philox call) x 4 columns, quantised e4m3(64 z).
        for (int q = t; q < (kM / 4) * (kBK8 / 4); q += kThreads) {
            const int gl = q >> 5;
            const int kq = q & 31;
            const uint64_t g = static_cast<uint64_t>((m0 >> 2) + gl);
            float z[4][4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t col = k0 + 4 * kq + c;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                // e4m3 keeps 3 mantissa bits (x3: about 7): G drawn with the fast intrinsics
                if (g < groups && col < B) v = gauss_quad<true>(key, kTagG, groups, static_cast<uint64_t>(col), g);
                z[c][0] = v.x;
                z[c][1] = v.y;
                z[c][2] = v.z;
                z[c][3] = v.w;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int rr = 4 * gl + r;
                const bool live = m0 + rr < m;
                float h[4], l[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) split_e4m3(live ? kGScale * z[c][r] : 0.0f, h[c], l[c]);
                const uint32_t off = tc::sw128_b8(rr, 4 * kq);
                *reinterpret_cast<uint32_t *>(a_hi + off) = pack_e4m3x4(h[0], h[1], h[2], h[3]);
                if (SPLIT3) *reinterpret_cast<uint32_t *>(a_lo + off) = pack_e4m3x4(l[0], l[1], l[2], l[3]);
            }
        }
        __syncthreads();  // warp_max complete; also: every thread finished draining tile it-2
        float tmax = 0.0f;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) tmax = fmaxf(tmax, warp_max[w]);
        const float scale = tmax > 0.0f ? tmax / kE4M3Max : 1.0f;
        const float inv = 1.0f / scale;
        if (t == 0) tile_scale[s] = scale;
#pragma unroll
        for (int j = 0; j < C::kQuadsPerThread; ++j) {
            const int q = t + j * kThreads;
            const int nl = q % NT;
            const int kq = q / NT;
            float h[4], l[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) split_e4m3(xb[j][c] * inv, h[c], l[c]);
            const uint32_t off = tc::sw128_b8(nl, 4 * kq);
            *reinterpret_cast<uint32_t *>(b_hi + off) = pack_e4m3x4(h[0], h[1], h[2], h[3]);
            if (SPLIT3) *reinterpret_cast<uint32_t *>(b_lo + off) = pack_e4m3x4(l[0], l[1], l[2], l[3]);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (abort_flag) break;
        if (t == 0) {
            tc::fence_after_sync();
            const uint32_t sa_hi = sbase + s * C::kStage;
            const uint32_t sb_hi = sa_hi + C::kA;
            const uint32_t sa_lo = sa_hi + C::kA + C::kB;
            const uint32_t sb_lo = sa_lo + C::kA;
            const uint32_t dst = tmem + static_cast<uint32_t>(s * NT);
#pragma unroll
            for (int ks = 0; ks < kBK8 / 32; ++ks) {
                const uint32_t koff = 32u * ks;  // 32 e4m3 of K = 32 bytes
                const uint64_t ad = tc::smem_desc_sw128(sa_hi + koff, 16, 1024);
                const uint64_t bd = tc::smem_desc_sw128(sb_hi + koff, 16, 1024);
                tc::mma_e4m3(dst, ad, bd, kIdesc, ks > 0 ? 1u : 0u);
                if (SPLIT3) {
                    tc::mma_e4m3(dst, ad, tc::smem_desc_sw128(sb_lo + koff, 16, 1024), kIdesc, 1u);
                    tc::mma_e4m3(dst, tc::smem_desc_sw128(sa_lo + koff, 16, 1024), bd, kIdesc, 1u);
                }
            }
            tc::mma_commit(tc::smem_u32(&mbar[s]));
        }
        issued = it + 1;
        if (it >= 1) drain(it - 1);
        tc::fence_before_sync();
    }
    __syncthreads();
    if (issued > 0 && !abort_flag) drain(issued - 1);
    __syncthreads();
    // A drained tile leaves no MMA in flight; after an abort wait (bounded) for the
    // last issued tile before TMEM is released.
    if (abort_flag && issued > 0) wait_stage(tc::smem_u32(&mbar[(issued - 1) & 1]), ((issued - 1) >> 1) & 1);
    const bool ok = !abort_flag;
    const int grow = m0 + row;
    float *out = part + static_cast<size_t>(blockIdx.x) * m * d;
    const bool vec = bn == NT && (d & 3) == 0 && ((reinterpret_cast<uintptr_t>(out) | (n0 * 4u)) & 15) == 0;
    if (grow < m) {
        float *o = out + static_cast<size_t>(grow) * d + n0 + half * (NT / 2);
        if (vec) {
#pragma unroll
            for (int j = 0; j < NT / 2; j += 4)
                *reinterpret_cast<float4 *>(o + j) = ok ? make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3])
                                                        : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
#pragma unroll
            for (int j = 0; j < NT / 2; ++j)
                if (half * (NT / 2) + j < bn) o[j] = ok ? acc[j] : 0.0f;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, C::kTmemCols);
}

template <int NT, bool SPLIT3>
cudaError_t launch_tc8(const float *SX, int m, int d, int64_t B, Key key, int nsplit, float *partials, int *status,
                       const EventPair *ev, cudaStream_t stream) {
    using C = Cfg8<NT, SPLIT3>;
    const int64_t nslabs = (B + kBK8 - 1) / kBK8;
    const int64_t per = (nslabs + nsplit - 1) / nsplit;
    const int used = static_cast<int>((nslabs + per - 1) / per);
    const uint32_t smem = C::kSmem;
    cudaError_t e = cudaFuncSetAttribute(contract_tc_fp8_kernel<NT, SPLIT3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    dim3 grid(used, (d + NT - 1) / NT, (m + kM - 1) / kM);
    record(ev, true, stream);
    e = launch_after_previous(contract_tc_fp8_kernel<NT, SPLIT3>, grid, dim3(kThreads), smem, stream, SX, m, d, B, key,
                              per, partials, status);
    record(ev, false, stream);
    return e != cudaSuccess ? e : cudaGetLastError();
}

int tc8_nt(int d) { return d <= 64 ? 64 : 128; }

// Resident CTAs per SM of each contraction kernel (from its registers, shared memory
// and TMEM columns; the same on every device of this architecture, so computed once).
template <int NT, bool SPLIT3>
int ctas_bf16() {
    using C = Cfg<NT, SPLIT3>;
    static int n = 0;
    if (n == 0)
        n = resident_ctas_per_sm(reinterpret_cast<const void *>(contract_tc_bf16_kernel<NT, SPLIT3>),
                                 bf16_threads<NT, SPLIT3>(),
                                 C::kSmem, static_cast<int>(C::kTmemCols));
    return n;
}

template <int NT, bool SPLIT3>
int ctas_fp8() {
    using C = Cfg8<NT, SPLIT3>;
    static int n = 0;
    if (n == 0)
        n = resident_ctas_per_sm(reinterpret_cast<const void *>(contract_tc_fp8_kernel<NT, SPLIT3>), kThreads,
                                 C::kSmem, static_cast<int>(C::kTmemCols));
    return n;
}

int tc_ctas_per_sm(int precision, int d) {
    const bool x3 = precision == CG_PREC_BF16X3 || precision == CG_PREC_FP8X3;
    if (precision == CG_PREC_FP8_E4M3 || precision == CG_PREC_FP8X3) {
        if (tc8_nt(d) == 64) return x3 ? ctas_fp8<64, true>() : ctas_fp8<64, false>();
        return x3 ? ctas_fp8<128, true>() : ctas_fp8<128, false>();
    }
    switch (tc_nt(d)) {
        case 64: return x3 ? ctas_bf16<64, true>() : ctas_bf16<64, false>();
        case 128: return x3 ? ctas_bf16<128, true>() : ctas_bf16<128, false>();
        default: return x3 ? ctas_bf16<256, true>() : ctas_bf16<256, false>();
    }
}

}  // namespace

int contract_tc_splits(const cg_plan &p) {
    const bool fp8 = p.precision == CG_PREC_FP8_E4M3 || p.precision == CG_PREC_FP8X3;
    const int64_t bk = fp8 ? kBK8 : kBK;
    const int64_t nslabs = (p.B + bk - 1) / bk;
    if (p.ksplit > 0) return static_cast<int>(p.ksplit < nslabs ? p.ksplit : nslabs);
    const int nt = fp8 ? tc8_nt(p.d) : tc_nt(p.d);
    const int64_t blocks = static_cast<int64_t>((p.m + kM - 1) / kM) * ((p.d + nt - 1) / nt);
    const int sms = num_sms() > 0 ? num_sms() : 148;
    // whole waves: as many CTAs as fit the GPU at once, never a partial second wave
    const int64_t target = static_cast<int64_t>(sms) * (num_sms() > 0 ? tc_ctas_per_sm(p.precision, p.d) : 1);
    int64_t s = target / blocks;
    if (s < 1) s = 1;
    if (s > nslabs) s = nslabs;
    return static_cast<int>(s);
}

cudaError_t launch_contract_tc(const float *SX, int m, int d, int64_t B, Key key, int precision, int nsplit,
                               float *partials, float *Y, int *status, const EventPair *ev, cudaStream_t stream,
                               bool transpose, int32_t *imax, int32_t *imin) {
    cudaError_t e;
    const bool fp8 = precision == CG_PREC_FP8_E4M3 || precision == CG_PREC_FP8X3;
    const int nt = fp8 ? tc8_nt(d) : tc_nt(d);
    const bool x3 = precision == CG_PREC_BF16X3 || precision == CG_PREC_FP8X3;
    if (fp8) {
        if (nt == 64)
            e = x3 ? launch_tc8<64, true>(SX, m, d, B, key, nsplit, partials, status, ev, stream)
                   : launch_tc8<64, false>(SX, m, d, B, key, nsplit, partials, status, ev, stream);
        else
            e = x3 ? launch_tc8<128, true>(SX, m, d, B, key, nsplit, partials, status, ev, stream)
                   : launch_tc8<128, false>(SX, m, d, B, key, nsplit, partials, status, ev, stream);
    } else if (nt == 64)
        e = x3 ? launch_tc<64, true>(SX, m, d, B, key, nsplit, partials, status, ev, stream)
               : launch_tc<64, false>(SX, m, d, B, key, nsplit, partials, status, ev, stream);
    else if (nt == 128)
        e = x3 ? launch_tc<128, true>(SX, m, d, B, key, nsplit, partials, status, ev, stream)
               : launch_tc<128, false>(SX, m, d, B, key, nsplit, partials, status, ev, stream);
    else
        e = x3 ? launch_tc<256, true>(SX, m, d, B, key, nsplit, partials, status, ev, stream)
               : launch_tc<256, false>(SX, m, d, B, key, nsplit, partials, status, ev, stream);
    if (e != cudaSuccess) return e;
    const int64_t bk = fp8 ? kBK8 : kBK;
    const int64_t nslabs = (B + bk - 1) / bk;
    const int64_t per = (nslabs + nsplit - 1) / nsplit;
    const int used = static_cast<int>((nslabs + per - 1) / per);
    if (imax != nullptr) return launch_reduce_rows_anchors(partials, used, m, d, Y, imax, imin, stream);
    return launch_reduce_splits(partials, used, static_cast<int64_t>(m) * d, Y, stream, transpose ? d : 0);
}

}  // namespace cg

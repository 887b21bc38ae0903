// cg_api.cu -- the C ABI of libcountgauss (declared in include/countgauss.h, where each
// entry point cites the passage of the paper it follows): plans, argument validation,
// workspace layout and dispatch to the kernels.
// Everything here is host code except the three generator-dump kernels.
#include <new>
#include <vector>

#include <algorithm>

#include "cg_internal.cuh"

namespace cg {

// Event pairs recorded per kernel kind; resolved and recycled by cg_plan_timing.
struct TimingState {
    std::vector<EventPair> pending[CG_KERNEL_COUNT];
    std::vector<EventPair> free_pairs;
    double carried_ms[CG_KERNEL_COUNT] = {0};
    int64_t carried_launches[CG_KERNEL_COUNT] = {0};
};

namespace {

constexpr size_t kMaxPendingPairs = 4096;

void resolve(TimingState *ts, int kernel) {
    for (EventPair &ev : ts->pending[kernel]) {
        float ms = 0.0f;
        if (cudaEventSynchronize(ev.stop) == cudaSuccess && cudaEventElapsedTime(&ms, ev.start, ev.stop) == cudaSuccess) {
            ts->carried_ms[kernel] += ms;
            ts->carried_launches[kernel] += 1;
        } else {
            cudaGetLastError();
        }
        ts->free_pairs.push_back(ev);
    }
    ts->pending[kernel].clear();
}

}  // namespace

const EventPair *timing_pair(cg_plan *p, int kernel) {
    if (p == nullptr || !p->timing || kernel < 0 || kernel >= CG_KERNEL_COUNT) return nullptr;
    TimingState *ts = static_cast<TimingState *>(p->timing_state);
    if (ts == nullptr) {
        ts = new (std::nothrow) TimingState;
        if (ts == nullptr) return nullptr;
        p->timing_state = ts;
    }
    if (ts->pending[kernel].size() >= kMaxPendingPairs) resolve(ts, kernel);
    EventPair ev;
    if (!ts->free_pairs.empty()) {
        ev = ts->free_pairs.back();
        ts->free_pairs.pop_back();
    } else if (cudaEventCreate(&ev.start) != cudaSuccess || cudaEventCreate(&ev.stop) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    ts->pending[kernel].push_back(ev);
    return &ts->pending[kernel].back();
}

namespace {

constexpr int kMaxDevices = 64;
int g_sms[kMaxDevices] = {0};

__global__ void generate_words_kernel(Key key, uint32_t tag, uint64_t idx0, int64_t count, uint32_t *words) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint4 w = stream_words(key, idx0 + static_cast<uint64_t>(t), tag);
        reinterpret_cast<uint4 *>(words)[t] = w;
    }
}

__global__ void generate_hash_sign_kernel(Key key, uint32_t B, int64_t row0, int64_t count, int32_t *h,
                                          int32_t *sigma) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint32_t hh;
        float s;
        hash_sign(key, static_cast<uint64_t>(row0 + t), B, hh, s);
        h[t] = static_cast<int32_t>(hh);
        sigma[t] = s < 0.0f ? -1 : 1;
    }
}

__global__ void generate_gaussian_kernel(Key key, uint32_t tag, int64_t R, int64_t r0, int64_t r1, int64_t c0,
                                         int64_t c1, float *out) {
    const int64_t rows = r1 - r0, cols = c1 - c0, total = rows * cols;
    const uint64_t groups = static_cast<uint64_t>((R + 3) / 4);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = r0 + t / cols;
        const int64_t c = c0 + t % cols;
        const float4 z = gauss_quad(key, tag, groups, static_cast<uint64_t>(c), static_cast<uint64_t>(r / 4));
        const int lane = static_cast<int>(r & 3);
        out[t] = lane == 0 ? z.x : lane == 1 ? z.y : lane == 2 ? z.z : z.w;
    }
}

// lowbias32 (C. Wellons): a 32-bit integer hash with good avalanche, used only to
// spread the diagnostic's reductions over the array.
__device__ __forceinline__ uint32_t lowbias32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// `count` reductions of 1.0f at lowbias32(k) mod cells, grid-stride over k, with the
// scatter kernel's block size (256) and grid.
__global__ void __launch_bounds__(256) random_reductions_kernel(float *__restrict__ a, uint32_t cells, uint32_t count) {
    for (uint32_t k = blockIdx.x * 256u + threadIdx.x; k < count; k += gridDim.x * 256u)
        atomicAdd(a + lowbias32(k) % cells, 1.0f);
}

unsigned dump_grid(int64_t count) {
    const int64_t g = (count + 255) / 256;
    return static_cast<unsigned>(g < 1 ? 1 : (g > 65536 ? 65536 : g));
}

}  // namespace

int num_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return 0;
    }
    if (dev < kMaxDevices && g_sms[dev] > 0) return g_sms[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (dev < kMaxDevices) g_sms[dev] = sms;
    return sms;
}

int l2_bytes() {
    static int cache[kMaxDevices] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return 0;
    }
    if (cache[dev] == 0 && cudaDeviceGetAttribute(&cache[dev], cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
        cudaGetLastError();
        cache[dev] = 0;
    }
    return cache[dev];
}

int resident_ctas_per_sm(const void *kernel, int threads, size_t dyn_smem, int tmem_cols) {
    int dev = 0, regs_sm = 0, smem_sm = 0, reserved = 0, threads_sm = 0, blocks_sm = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, kernel) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&blocks_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const int warps = (threads + 31) / 32;
    const int regs_warp = ((fa.numRegs > 0 ? fa.numRegs : 1) * 32 + 255) / 256 * 256;  // 256-register units
    int n = (regs_sm / regs_warp) / warps;
    const size_t smem_cta = fa.sharedSizeBytes + dyn_smem + static_cast<size_t>(reserved);
    if (smem_cta > 0) n = std::min<int>(n, static_cast<int>(static_cast<size_t>(smem_sm) / smem_cta));
    n = std::min(n, threads_sm / threads);
    n = std::min(n, blocks_sm);
    if (tmem_cols > 0) n = std::min(n, 512 / tmem_cols);
    return n < 1 ? 1 : n;
}

cudaError_t launch_generate_words(Key key, uint32_t tag, uint64_t idx0, int64_t count, uint32_t *words,
                                  cudaStream_t stream) {
    generate_words_kernel<<<dump_grid(count), 256, 0, stream>>>(key, tag, idx0, count, words);
    return cudaGetLastError();
}

cudaError_t launch_generate_hash_sign(Key key, uint32_t B, int64_t row0, int64_t count, int32_t *h, int32_t *sigma,
                                      cudaStream_t stream) {
    generate_hash_sign_kernel<<<dump_grid(count), 256, 0, stream>>>(key, B, row0, count, h, sigma);
    return cudaGetLastError();
}

cudaError_t launch_generate_gaussian(Key key, uint32_t tag, int64_t R, int64_t r0, int64_t r1, int64_t c0,
                                     int64_t c1, float *out, cudaStream_t stream) {
    generate_gaussian_kernel<<<dump_grid((r1 - r0) * (c1 - c0)), 256, 0, stream>>>(key, tag, R, r0, r1, c0, c1,
                                                                                  out);
    return cudaGetLastError();
}

// Rows per warp chunk of the one-pass scatter: as forced, else one row per lane for small
// inputs with under two nonzeros per row (there latency rules, and 32-row lane chunks give
// the most CTAs: 8.8 against 9.7 us per call at 2^16 x 16 with 0.8 nonzeros per row), else
// the kernel's own choice (staged chunks of about 96 nonzeros).
int one_pass_rows(const cg_plan &p, int64_t nnz) {
    if (p.scatter_rows != 0) return p.scatter_rows;
    if (p.n > 0 && p.n <= (1 << 18) && nnz < 2 * p.n) return 1;
    return 0;
}

}  // namespace cg

using namespace cg;

namespace {

constexpr int64_t kMaxB = (1LL << 31) - 1;

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

bool misaligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; }

cg_status from_cuda(cudaError_t e) { return e == cudaSuccess ? CG_OK : CG_ERR_CUDA; }

// Whether a CSR scatter through plan p uses the partitioned algorithm (on request
// only: the atomic scatter is faster at present).  Deterministic mode uses the
// fixed-point scatter instead.
bool use_partition(const cg_plan &p) {
    if (p.deterministic) return false;
    return p.scatter == 2 && partition_supported(p);
}

// Whether SX is larger than 60 % of the L2, where random reductions into it start to miss.
bool sx_past_l2(const cg_plan &p) {
    const double sx = static_cast<double>(p.B) * p.d * sizeof(float);
    const int l2 = l2_bytes();
    return l2 > 0 && sx > 0.6 * l2;
}

// Whether the deterministic mode bins the nonzeros by bucket slice and sums each slice in
// int64 fixed point in shared memory: when its int64 accumulator (8 B d bytes) would not
// fit the L2 (60 % of it), where the fixed-point reductions into global memory slow down
// several-fold; the sums are the same integers, so the result is bit-identical.
// CG_OPT_SCATTER = 4 asks for the slices, 1 for the global accumulator.
bool use_binned_fixed(const cg_plan &p) {
    if (!p.deterministic || !binned_supported(p.n, p.d, p.B, true)) return false;
    if (p.scatter == 4) return true;
    if (p.scatter == 1) return false;
    const double acc = 8.0 * static_cast<double>(p.B) * p.d;
    const int l2 = l2_bytes();
    return l2 > 0 && acc > 0.6 * l2;
}

// Whether a CSR scatter through plan p bins the nonzeros by bucket slice and sums each
// slice in shared memory: on request (CG_OPT_SCATTER = 4) only; on GB300 at the largest
// workload it measures slightly slower than the deferred scatter (0.98 against 0.93 ms).
bool use_binned(const cg_plan &p, int64_t nnz) {
    (void)nnz;
    return !p.deterministic && p.scatter == 4 && binned_supported(p.n, p.d, p.B);
}

// Whether a CSR scatter through plan p defers half of SX to a second pass: on request
// (CG_OPT_SCATTER = 3), or automatically for an SX past the L2 (and bucket-range passes
// not forced).
bool use_deferred(const cg_plan &p, int64_t nnz) {
    if (p.deterministic || use_partition(p) || use_binned(p, nnz) || !deferred_supported(p.B, p.d)) return false;
    if (p.scatter == 3) return true;
    if (p.scatter != 0 || p.scatter_passes > 0) return false;
    return sx_past_l2(p);
}

// Scratch bytes of the CSR scatter through plan p (region C).
size_t scatter_scratch(const cg_plan &p, int64_t nnz, PartLayout *part) {
    if (p.deterministic)
        return use_binned_fixed(p) ? sketch_binned_scratch_bytes(p.n, p.d, p.B, nnz, static_cast<int>(p.sketch_ctas), true)
                                   : sketch_fixed_scratch_bytes(p.B, p.d);
    if (use_partition(p)) {
        *part = partition_layout(p, nnz);
        return part->bytes;
    }
    if (use_binned(p, nnz)) return sketch_binned_scratch_bytes(p.n, p.d, p.B, nnz, static_cast<int>(p.sketch_ctas));
    if (use_deferred(p, nnz))
        return sketch_deferred_scratch_bytes(
            nnz, sketch_deferred_ctas(static_cast<int>(p.sketch_ctas), p.n, nnz, p.scatter_rows));
    return 0;
}

// Scratch bytes of the CSR scatter with int64 row offsets through plan p: the deferred
// scatter's records, or none for the one-pass scatter.
size_t scatter_scratch_i64(const cg_plan &p, int64_t nnz) {
    if (!use_deferred(p, nnz)) return 0;
    return sketch_deferred_scratch_bytes(
            nnz, sketch_deferred_ctas(static_cast<int>(p.sketch_ctas), p.n, nnz, p.scatter_rows));
}

// Workspace layout: [status 256 B][region A][region B][region C], each 256-aligned.
// A: SX or W;  B: split-K partials;  C: scratch of the partitioned scatter.
struct Layout {
    size_t a_off = kStatusBytes, a_bytes = 0;
    size_t b_off = 0, b_bytes = 0;
    size_t c_off = 0, c_bytes = 0;
    size_t total = 0;
    PartLayout part;
};

// Chunk sizes of cg_apply_csr_host and the bytes of one staging buffer (row offsets,
// column indices, values of one chunk, each 256-aligned).
struct HostCaps {
    int64_t nnz = 1, rows = 1;
    size_t rp_off = 0, ci_off = 0, v_off = 0, stage_bytes = 0;
};

HostCaps host_caps(const cg_plan &p, int64_t nnz) {
    HostCaps c;
    // automatic: about four chunks (copy of chunk c + 1 hides the scatter of chunk c), each
    // at least 2^20 and at most 2^24 nonzeros (per-copy overheads vs. pipeline fill)
    const int64_t chunk =
        p.host_chunk > 0 ? p.host_chunk : std::max<int64_t>(1LL << 20, std::min<int64_t>(1LL << 24, nnz / 4));
    c.nnz = std::max<int64_t>(1, std::min(nnz, chunk));
    c.rows = std::max<int64_t>(1, std::min(p.n, chunk));
    c.rp_off = 0;
    c.ci_off = align256(static_cast<size_t>(c.rows + 1) * sizeof(int32_t));
    c.v_off = c.ci_off + align256(static_cast<size_t>(c.nnz) * sizeof(int32_t));
    c.stage_bytes = c.v_off + align256(static_cast<size_t>(c.nnz) * sizeof(float));
    return c;
}

Layout layout_for(const cg_plan &p, int op, int64_t nnz) {
    Layout L;
    const size_t sx = static_cast<size_t>(p.B) * p.d * sizeof(float);
    switch (op) {
        case CG_OP_APPLY_CSR:
            L.a_bytes = sx;
            L.b_bytes = contract_partials_bytes(p);
            L.c_bytes = scatter_scratch(p, nnz, &L.part);
            break;
        case CG_OP_APPLY_DENSE:
            L.a_bytes = sx;
            L.b_bytes = contract_partials_bytes(p);
            break;
        case CG_OP_CONTRACT:
            L.b_bytes = contract_partials_bytes(p);
            break;
        case CG_OP_ADJOINT_DENSE:
        case CG_OP_ADJOINT_CSR:
            L.a_bytes = sx;
            break;
        case CG_OP_PLAIN_CSR:
            L.b_bytes = plain_partials_bytes(p.m, p.d);
            break;
        case CG_OP_SKETCH:
            L.c_bytes = scatter_scratch(p, nnz, &L.part);
            break;
        case CG_OP_APPLY_CSR_I64:
            L.a_bytes = sx;
            L.b_bytes = contract_partials_bytes(p);
            L.c_bytes = scatter_scratch_i64(p, nnz);
            break;
        case CG_OP_SKETCH_I64:
            L.c_bytes = scatter_scratch_i64(p, nnz);
            break;
        case CG_OP_APPLY_RIGHT_CSR:
            L.a_bytes = sx;
            L.b_bytes = contract_partials_bytes(p);
            L.c_bytes = right_scratch_bytes(p.n, nnz);
            break;
        case CG_OP_APPLY_CSR_HOST: {
            // [Y, m x d][two staging buffers (copied reads) or the scatter's scratch (direct reads)]
            const HostCaps c = host_caps(p, nnz);
            L.a_bytes = sx;
            L.b_bytes = contract_partials_bytes(p);
            L.c_bytes = align256(static_cast<size_t>(p.m) * p.d * sizeof(float)) +
                        std::max(2 * c.stage_bytes, scatter_scratch(p, nnz, &L.part));
            break;
        }
        default:
            break;
    }
    L.b_off = L.a_off + align256(L.a_bytes);
    L.c_off = L.b_off + align256(L.b_bytes);
    L.total = L.c_off + align256(L.c_bytes);
    return L;
}

cg_status check_ws(const cg_plan *p, int op, int64_t nnz, void *ws, size_t ws_bytes, Layout *L) {
    *L = layout_for(*p, op, nnz);
    if (ws == nullptr) return CG_ERR_INVALID_ARG;
    if (misaligned(ws, 256)) return CG_ERR_INVALID_ARG;
    if (ws_bytes < L->total) return CG_ERR_WORKSPACE;
    return CG_OK;
}

cg_status check_csr(const cg_plan *p, const int32_t *row_ptr, const int32_t *col_idx, const float *vals,
                    int64_t nnz, bool need_vals) {
    if (nnz < 0 || nnz > kMaxNnz) return CG_ERR_INVALID_ARG;
    if (row_ptr == nullptr) return CG_ERR_INVALID_ARG;
    if (nnz > 0 && (col_idx == nullptr || (need_vals && vals == nullptr))) return CG_ERR_INVALID_ARG;
    if (misaligned(row_ptr, 4) || misaligned(col_idx, 4) || misaligned(vals, 4)) return CG_ERR_INVALID_ARG;
    (void)p;
    return CG_OK;
}

int *status_word(void *ws) { return reinterpret_cast<int *>(ws); }
char *region(void *ws, size_t off) { return reinterpret_cast<char *>(ws) + off; }

// Y = G.SX (m x d), or with `transpose` its transpose (d x m); with imax / imin also the
// row argmax / argmin of Y, from the split-K sum itself (Algorithm 1 step 3).
cg_status run_contract(cg_plan *p, const float *SX, float *Y, void *ws, const Layout &L, cudaStream_t st,
                       bool transpose = false, int32_t *imax = nullptr, int32_t *imin = nullptr) {
    if (p->precision != CG_PREC_FP32)
        return from_cuda(launch_contract_tc(SX, p->m, p->d, p->B, make_key(p->seed), p->precision,
                                            contract_tc_splits(*p), reinterpret_cast<float *>(region(ws, L.b_off)),
                                            Y, status_word(ws), timing_pair(p, CG_KERNEL_CONTRACT), st, transpose,
                                            imax, imin));
    return from_cuda(launch_contract_ffma(SX, p->m, p->d, p->B, make_key(p->seed), contract_splits(*p),
                                          reinterpret_cast<float *>(region(ws, L.b_off)), Y,
                                          timing_pair(p, CG_KERNEL_CONTRACT), st, transpose, imax, imin));
}


// SX = S.X, or with clear = false SX += S.X (atomic and deferred scatters only).
// host_mapped: the CSR arrays are page-locked host memory read in place (no L2 prefetch
// of them).
cg_status run_sketch_csr(cg_plan *p, const int32_t *row_ptr, const int32_t *col_idx, const float *vals,
                         int64_t nnz, float *SX, void *ws, const Layout &L, cudaStream_t st, bool clear = true,
                         bool host_mapped = false) {
    if (p->deterministic && use_binned_fixed(*p))
        return from_cuda(launch_sketch_csr_binned(row_ptr, col_idx, vals, static_cast<int>(p->n), p->d,
                                                  static_cast<uint32_t>(p->B), static_cast<int>(nnz),
                                                  make_key(p->seed), p->row_offset, SX, status_word(ws),
                                                  region(ws, L.c_off), static_cast<int>(p->sketch_ctas),
                                                  timing_pair(p, CG_KERNEL_SKETCH), st, true, !host_mapped, true));
    if (p->deterministic)
        return from_cuda(launch_sketch_csr_fixed(row_ptr, col_idx, vals, static_cast<int>(p->n), p->d,
                                                 static_cast<uint32_t>(p->B), static_cast<int>(nnz), make_key(p->seed),
                                                 p->row_offset, SX, region(ws, L.c_off), status_word(ws),
                                                 static_cast<int>(p->sketch_ctas), p->scatter_rows,
                                                 timing_pair(p, CG_KERNEL_SKETCH), st));
    if (use_binned(*p, nnz))
        return from_cuda(launch_sketch_csr_binned(row_ptr, col_idx, vals, static_cast<int>(p->n), p->d,
                                                  static_cast<uint32_t>(p->B), static_cast<int>(nnz),
                                                  make_key(p->seed), p->row_offset, SX, status_word(ws),
                                                  region(ws, L.c_off), static_cast<int>(p->sketch_ctas),
                                                  timing_pair(p, CG_KERNEL_SKETCH), st, clear, !host_mapped));
    if (use_deferred(*p, nnz))
        return from_cuda(launch_sketch_csr_deferred(row_ptr, col_idx, vals, static_cast<int>(p->n), p->d,
                                                    static_cast<uint32_t>(p->B), static_cast<int>(nnz),
                                                    make_key(p->seed), p->row_offset, SX, status_word(ws),
                                                    region(ws, L.c_off), static_cast<int>(p->sketch_ctas),
                                                    p->scatter_rows, timing_pair(p, CG_KERNEL_SKETCH), st, clear,
                                                    !host_mapped));
    if (use_partition(*p))
        return from_cuda(launch_sketch_csr_partitioned(
            row_ptr, col_idx, vals, static_cast<int>(p->n), p->d, static_cast<uint32_t>(p->B), static_cast<int>(nnz),
            make_key(p->seed), p->row_offset, SX, status_word(ws), region(ws, L.c_off), L.part,
            timing_pair(p, CG_KERNEL_SKETCH), st));
    return from_cuda(launch_sketch_csr_atomic(row_ptr, col_idx, vals, static_cast<int>(p->n), p->d,
                                              static_cast<uint32_t>(p->B), static_cast<int>(nnz), make_key(p->seed),
                                              p->row_offset, SX, status_word(ws), static_cast<int>(p->sketch_ctas),
                                              p->scatter_passes, one_pass_rows(*p, nnz),
                                              timing_pair(p, CG_KERNEL_SKETCH), st, clear));
}

// Device address of the page-locked host range [p, p + bytes), or nullptr when the
// range is not page-locked memory mapped into the current device's address space.
const void *mapped_host(const void *p, size_t bytes) {
    if (p == nullptr || bytes == 0) return p;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return nullptr;
    cudaPointerAttributes b;  // the last byte must lie in the same mapped allocation
    if (cudaPointerGetAttributes(&b, static_cast<const char *>(p) + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (b.type != cudaMemoryTypeHost ||
        static_cast<const char *>(b.devicePointer) != static_cast<const char *>(a.devicePointer) + bytes - 1)
        return nullptr;
    return a.devicePointer;
}

// Direct reads for cg_apply_csr_host: on request (CG_OPT_HOST_READ = 2), and only when
// all three host arrays are mapped page-locked memory; then *drp, *dci, *dv receive their
// device addresses.  Not the default: on GB300 over NVLink-C2C the scatter reading host
// memory in place moves the CSR at about 177 GB/s, the copy engine at about 200 GB/s.
bool host_read_direct(const cg_plan &p, const int32_t *row_ptr, const int32_t *col_idx, const float *vals,
                      int64_t nnz, const int32_t **drp, const int32_t **dci, const float **dv) {
    if (p.host_read != 2) return false;
    const void *a = mapped_host(row_ptr, static_cast<size_t>(p.n + 1) * sizeof(int32_t));
    const void *b = mapped_host(col_idx, static_cast<size_t>(nnz) * sizeof(int32_t));
    const void *c = mapped_host(vals, static_cast<size_t>(nnz) * sizeof(float));
    if (a == nullptr || (nnz > 0 && (b == nullptr || c == nullptr))) return false;
    *drp = static_cast<const int32_t *>(a);
    *dci = static_cast<const int32_t *>(b);
    *dv = static_cast<const float *>(c);
    return true;
}

// Copy stream and events of cg_apply_csr_host, made on first use on a device and kept
// by the plan (remade if the plan is used on another device).
struct HostState {
    int device = -1;
    cudaStream_t copy = nullptr;
    cudaEvent_t start = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t consumed[2] = {nullptr, nullptr};
};

void destroy_host_state(cg_plan *p) {
    HostState *h = static_cast<HostState *>(p->host_state);
    if (h == nullptr) return;
    if (h->copy != nullptr) cudaStreamDestroy(h->copy);
    for (cudaEvent_t e : {h->start, h->copied[0], h->copied[1], h->consumed[0], h->consumed[1]})
        if (e != nullptr) cudaEventDestroy(e);
    delete h;
    p->host_state = nullptr;
}

HostState *host_state(cg_plan *p) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    HostState *h = static_cast<HostState *>(p->host_state);
    if (h != nullptr && h->device == dev) return h;
    destroy_host_state(p);
    h = new (std::nothrow) HostState;
    if (h == nullptr) return nullptr;
    h->device = dev;
    p->host_state = h;
    bool ok = cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&h->start, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaEventCreateWithFlags(&h->copied[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->consumed[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        destroy_host_state(p);
        return nullptr;
    }
    return h;
}

}  // namespace

extern "C" {

const char *cg_status_string(cg_status s) {
    switch (s) {
        case CG_OK: return "CG_OK";
        case CG_ERR_INVALID_ARG: return "CG_ERR_INVALID_ARG: invalid argument";
        case CG_ERR_UNSUPPORTED: return "CG_ERR_UNSUPPORTED: request not supported by the library";
        case CG_ERR_WORKSPACE: return "CG_ERR_WORKSPACE: workspace too small";
        case CG_ERR_CUDA: return "CG_ERR_CUDA: a CUDA call or kernel launch failed";
        case CG_ERR_TIMEOUT: return "CG_ERR_TIMEOUT: a bounded device wait gave up";
        case CG_ERR_DEVICE_BOUNDS: return "CG_ERR_DEVICE_BOUNDS: a kernel skipped an out-of-range index";
        case CG_ERR_NO_DEVICE: return "CG_ERR_NO_DEVICE: no usable CUDA device";
    }
    return "unknown cg_status";
}

cg_status cg_plan_create(int64_t n, int32_t d, int32_t m, int64_t B, uint64_t seed, cg_plan **out) {
    if (out == nullptr) return CG_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || n > kMaxRows || d < 1 || d > 65536 || m < 1 || m > 65536 || B < 1 || B > kMaxB)
        return CG_ERR_INVALID_ARG;
    if (B * static_cast<int64_t>(d) >= (1LL << 40)) return CG_ERR_INVALID_ARG;
    cg_plan *p = new (std::nothrow) cg_plan;
    if (p == nullptr) return CG_ERR_INVALID_ARG;
    p->n = n;
    p->d = d;
    p->m = m;
    p->B = B;
    p->seed = seed;
    p->precision = CG_PREC_FP32;
    p->deterministic = 0;
    p->row_offset = 0;
    p->ksplit = 0;
    p->sketch_ctas = 0;
    p->timing = 0;
    p->timing_state = nullptr;
    p->scatter = 0;
    p->scatter_passes = 0;
    p->scatter_rows = 0;
    p->host_chunk = 0;
    p->host_read = 0;
    p->accumulate = 0;
    p->host_state = nullptr;
    *out = p;
    return CG_OK;
}

cg_status cg_plan_destroy(cg_plan *plan) {
    if (plan == nullptr) return CG_OK;
    TimingState *ts = static_cast<TimingState *>(plan->timing_state);
    if (ts != nullptr) {
        for (int k = 0; k < CG_KERNEL_COUNT; ++k) {
            for (EventPair &ev : ts->pending[k]) ts->free_pairs.push_back(ev);
        }
        for (EventPair &ev : ts->free_pairs) {
            cudaEventDestroy(ev.start);
            cudaEventDestroy(ev.stop);
        }
        delete ts;
    }
    destroy_host_state(plan);
    delete plan;
    return CG_OK;
}

cg_status cg_plan_timing(cg_plan *p, int32_t kernel, double *total_ms, int64_t *launches) {
    if (p == nullptr || total_ms == nullptr || launches == nullptr || kernel < 0 || kernel >= CG_KERNEL_COUNT)
        return CG_ERR_INVALID_ARG;
    *total_ms = 0.0;
    *launches = 0;
    TimingState *ts = static_cast<TimingState *>(p->timing_state);
    if (ts == nullptr) return CG_OK;
    resolve(ts, kernel);
    *total_ms = ts->carried_ms[kernel];
    *launches = ts->carried_launches[kernel];
    ts->carried_ms[kernel] = 0.0;
    ts->carried_launches[kernel] = 0;
    return CG_OK;
}

cg_status cg_plan_set_option(cg_plan *p, int32_t option, int64_t value) {
    if (p == nullptr) return CG_ERR_INVALID_ARG;
    switch (option) {
        case CG_OPT_PRECISION:
            if (value < CG_PREC_FP32 || value > CG_PREC_FP8X3) return CG_ERR_INVALID_ARG;
            p->precision = static_cast<int32_t>(value);
            return CG_OK;
        case CG_OPT_DETERMINISTIC:
            if (value != 0 && value != 1) return CG_ERR_INVALID_ARG;
            p->deterministic = static_cast<int32_t>(value);
            return CG_OK;
        case CG_OPT_ROW_OFFSET:
            if (value < 0 || value > (1LL << 62)) return CG_ERR_INVALID_ARG;
            p->row_offset = value;
            return CG_OK;
        case CG_OPT_KSPLIT:
            if (value < 0 || value > (1 << 20)) return CG_ERR_INVALID_ARG;
            p->ksplit = value;
            return CG_OK;
        case CG_OPT_SKETCH_CTAS:
            if (value < 0 || value > (1 << 20)) return CG_ERR_INVALID_ARG;
            p->sketch_ctas = value;
            return CG_OK;
        case CG_OPT_TIMING:
            if (value != 0 && value != 1) return CG_ERR_INVALID_ARG;
            p->timing = static_cast<int32_t>(value);
            return CG_OK;
        case CG_OPT_SCATTER:
            if (value < 0 || value > 4) return CG_ERR_INVALID_ARG;
            p->scatter = static_cast<int32_t>(value);
            return CG_OK;
        case CG_OPT_SCATTER_PASSES:
            if (value < 0 || value > 16) return CG_ERR_INVALID_ARG;
            p->scatter_passes = static_cast<int32_t>(value);
            return CG_OK;
        case CG_OPT_SCATTER_ROWS:
            if (value != 0 && value != 1 && value != 32 && value != 64 && value != 128 && value != 256)
                return CG_ERR_INVALID_ARG;
            p->scatter_rows = static_cast<int32_t>(value);
            return CG_OK;
        case CG_OPT_HOST_CHUNK:
            if (value != 0 && (value < 32 || value > (1LL << 30))) return CG_ERR_INVALID_ARG;
            p->host_chunk = value;
            return CG_OK;
        case CG_OPT_HOST_READ:
            if (value < 0 || value > 2) return CG_ERR_INVALID_ARG;
            p->host_read = static_cast<int32_t>(value);
            return CG_OK;
        case CG_OPT_ACCUMULATE:
            if (value != 0 && value != 1) return CG_ERR_INVALID_ARG;
            p->accumulate = static_cast<int32_t>(value);
            return CG_OK;
        default:
            return CG_ERR_INVALID_ARG;
    }
}

cg_status cg_plan_get_option(const cg_plan *p, int32_t option, int64_t *value) {
    if (p == nullptr || value == nullptr) return CG_ERR_INVALID_ARG;
    switch (option) {
        case CG_OPT_PRECISION: *value = p->precision; return CG_OK;
        case CG_OPT_DETERMINISTIC: *value = p->deterministic; return CG_OK;
        case CG_OPT_ROW_OFFSET: *value = p->row_offset; return CG_OK;
        case CG_OPT_KSPLIT: *value = p->ksplit; return CG_OK;
        case CG_OPT_SKETCH_CTAS: *value = p->sketch_ctas; return CG_OK;
        case CG_OPT_TIMING: *value = p->timing; return CG_OK;
        case CG_OPT_SCATTER: *value = p->scatter; return CG_OK;
        case CG_OPT_SCATTER_PASSES: *value = p->scatter_passes; return CG_OK;
        case CG_OPT_SCATTER_ROWS: *value = p->scatter_rows; return CG_OK;
        case CG_OPT_HOST_CHUNK: *value = p->host_chunk; return CG_OK;
        case CG_OPT_HOST_READ: *value = p->host_read; return CG_OK;
        case CG_OPT_ACCUMULATE: *value = p->accumulate; return CG_OK;
        default: return CG_ERR_INVALID_ARG;
    }
}

cg_status cg_workspace_size(const cg_plan *p, int32_t op, int64_t nnz, size_t *bytes) {
    if (p == nullptr || bytes == nullptr || op < CG_OP_APPLY_CSR || op > CG_OP_SKETCH_I64) return CG_ERR_INVALID_ARG;
    *bytes = layout_for(*p, op, nnz).total;
    return CG_OK;
}

cg_status cg_plan_check(const cg_plan *p, void *ws, void *stream) {
    if (p == nullptr || ws == nullptr) return CG_ERR_INVALID_ARG;
    int h = 0;
    cudaStream_t st = as_stream(stream);
    if (cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CG_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CG_ERR_CUDA;
    if (h != 0) {
        if (cudaMemsetAsync(ws, 0, sizeof(int), st) != cudaSuccess) return CG_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return CG_ERR_CUDA;
    }
    if (h & kStatusTimeout) return CG_ERR_TIMEOUT;
    if (h & kStatusBounds) return CG_ERR_DEVICE_BOUNDS;
    return CG_OK;
}

cg_status cg_sketch_csr(cg_plan *p, const int32_t *row_ptr, const int32_t *col_idx, const float *vals, int64_t nnz,
                        float *SX, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_sketch_csr");
    if (p == nullptr || SX == nullptr || misaligned(SX, 16)) return CG_ERR_INVALID_ARG;
    cg_status s = check_csr(p, row_ptr, col_idx, vals, nnz, true);
    if (s != CG_OK) return s;
    Layout L;
    if ((s = check_ws(p, CG_OP_SKETCH, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    if (p->accumulate && (p->deterministic || use_partition(*p))) return CG_ERR_UNSUPPORTED;
    return run_sketch_csr(p, row_ptr, col_idx, vals, nnz, SX, ws, L, as_stream(stream), !p->accumulate);
}

cg_status cg_sketch_dense(cg_plan *p, const float *X, int64_t ldx, float *SX, void *ws, size_t ws_bytes,
                          void *stream) {
    cg::NvtxRange nvtx_range("cg_sketch_dense");
    if (p == nullptr || SX == nullptr || misaligned(SX, 16) || ldx < p->d) return CG_ERR_INVALID_ARG;
    if (p->n > 0 && (X == nullptr || misaligned(X, 4))) return CG_ERR_INVALID_ARG;
    cg_status s;
    Layout L;
    if ((s = check_ws(p, CG_OP_SKETCH, 0, ws, ws_bytes, &L)) != CG_OK) return s;
    if (p->deterministic) return CG_ERR_UNSUPPORTED;
    return from_cuda(launch_sketch_dense_atomic(X, ldx, static_cast<int>(p->n), p->d, static_cast<uint32_t>(p->B),
                                                make_key(p->seed), p->row_offset, SX, status_word(ws),
                                                static_cast<int>(p->sketch_ctas), timing_pair(p, CG_KERNEL_SKETCH),
                                                as_stream(stream), !p->accumulate));
}

cg_status cg_contract(cg_plan *p, const float *SX, float *Y, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_contract");
    if (p == nullptr || SX == nullptr || Y == nullptr || misaligned(SX, 4) || misaligned(Y, 4))
        return CG_ERR_INVALID_ARG;
    cg_status s;
    Layout L;
    if ((s = check_ws(p, CG_OP_CONTRACT, 0, ws, ws_bytes, &L)) != CG_OK) return s;
    return run_contract(p, SX, Y, ws, L, as_stream(stream));
}

cg_status cg_apply_csr(cg_plan *p, const int32_t *row_ptr, const int32_t *col_idx, const float *vals, int64_t nnz,
                       float *Y, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_apply_csr");
    if (p == nullptr || Y == nullptr || misaligned(Y, 4)) return CG_ERR_INVALID_ARG;
    cg_status s = check_csr(p, row_ptr, col_idx, vals, nnz, true);
    if (s != CG_OK) return s;
    Layout L;
    if ((s = check_ws(p, CG_OP_APPLY_CSR, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    float *SX = reinterpret_cast<float *>(region(ws, L.a_off));
    cudaStream_t st = as_stream(stream);
    if ((s = run_sketch_csr(p, row_ptr, col_idx, vals, nnz, SX, ws, L, st)) != CG_OK) return s;
    return run_contract(p, SX, Y, ws, L, st);
}

// Host-side checks of a CSR matrix with int64 row offsets and of the options its
// scatter honours: the one-pass atomic and the deferred scatters (the deterministic,
// partitioned and binned scatters index with 32-bit offsets).
cg_status check_csr_i64(const cg_plan *p, const int64_t *row_ptr, const int32_t *col_idx, const float *vals,
                        int64_t nnz) {
    if (nnz < 0 || nnz > kMaxNnz64 || row_ptr == nullptr) return CG_ERR_INVALID_ARG;
    if (nnz > 0 && (col_idx == nullptr || vals == nullptr)) return CG_ERR_INVALID_ARG;
    if (misaligned(row_ptr, 8) || misaligned(col_idx, 4) || misaligned(vals, 4)) return CG_ERR_INVALID_ARG;
    if (p->deterministic || p->scatter == 2 || p->scatter == 4) return CG_ERR_UNSUPPORTED;
    return CG_OK;
}

// SX = S.X, or with clear = false SX += S.X, for int64 row offsets.
cg_status run_sketch_csr_i64(cg_plan *p, const int64_t *row_ptr, const int32_t *col_idx, const float *vals,
                             int64_t nnz, float *SX, void *ws, const Layout &L, cudaStream_t st, bool clear) {
    if (use_deferred(*p, nnz))
        return from_cuda(launch_sketch_csr_deferred_i64(
            reinterpret_cast<const long long *>(row_ptr), col_idx, vals, static_cast<int>(p->n), p->d,
            static_cast<uint32_t>(p->B), static_cast<long long>(nnz), make_key(p->seed), p->row_offset, SX,
            status_word(ws), region(ws, L.c_off), static_cast<int>(p->sketch_ctas), p->scatter_rows,
            timing_pair(p, CG_KERNEL_SKETCH), st, clear));
    return from_cuda(launch_sketch_csr_atomic_i64(
        reinterpret_cast<const long long *>(row_ptr), col_idx, vals, static_cast<int>(p->n), p->d,
        static_cast<uint32_t>(p->B), static_cast<long long>(nnz), make_key(p->seed), p->row_offset, SX, status_word(ws),
        static_cast<int>(p->sketch_ctas), p->scatter_passes, one_pass_rows(*p, nnz), timing_pair(p, CG_KERNEL_SKETCH),
        st, clear));
}

cg_status cg_apply_csr_i64(cg_plan *p, const int64_t *row_ptr, const int32_t *col_idx, const float *vals,
                           int64_t nnz, float *Y, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_apply_csr_i64");
    if (p == nullptr || Y == nullptr || misaligned(Y, 4)) return CG_ERR_INVALID_ARG;
    cg_status s = check_csr_i64(p, row_ptr, col_idx, vals, nnz);
    if (s != CG_OK) return s;
    Layout L;
    if ((s = check_ws(p, CG_OP_APPLY_CSR_I64, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    float *SX = reinterpret_cast<float *>(region(ws, L.a_off));
    cudaStream_t st = as_stream(stream);
    if ((s = run_sketch_csr_i64(p, row_ptr, col_idx, vals, nnz, SX, ws, L, st, true)) != CG_OK) return s;
    return run_contract(p, SX, Y, ws, L, st);
}

cg_status cg_nmf_anchors_csr(cg_plan *p, const int32_t *row_ptr, const int32_t *col_idx, const float *vals,
                             int64_t nnz, float *Z, int32_t *imax, int32_t *imin, void *ws, size_t ws_bytes,
                             void *stream) {
    cg::NvtxRange nvtx_range("cg_nmf_anchors_csr");
    if (p == nullptr || Z == nullptr || imax == nullptr || imin == nullptr || misaligned(Z, 4)) return CG_ERR_INVALID_ARG;
    if (misaligned(imax, 4) || misaligned(imin, 4)) return CG_ERR_INVALID_ARG;
    cg_status s = check_csr(p, row_ptr, col_idx, vals, nnz, true);
    if (s != CG_OK) return s;
    Layout L;
    if ((s = check_ws(p, CG_OP_APPLY_CSR, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    float *SX = reinterpret_cast<float *>(region(ws, L.a_off));
    cudaStream_t st = as_stream(stream);
    if ((s = run_sketch_csr(p, row_ptr, col_idx, vals, nnz, SX, ws, L, st)) != CG_OK) return s;
    return run_contract(p, SX, Z, ws, L, st, false, imax, imin);
}

cg_status cg_nmf_anchors_csr_i64(cg_plan *p, const int64_t *row_ptr, const int32_t *col_idx, const float *vals,
                                 int64_t nnz, float *Z, int32_t *imax, int32_t *imin, void *ws, size_t ws_bytes,
                                 void *stream) {
    cg::NvtxRange nvtx_range("cg_nmf_anchors_csr_i64");
    if (p == nullptr || Z == nullptr || imax == nullptr || imin == nullptr || misaligned(Z, 4)) return CG_ERR_INVALID_ARG;
    if (misaligned(imax, 4) || misaligned(imin, 4)) return CG_ERR_INVALID_ARG;
    cg_status s = check_csr_i64(p, row_ptr, col_idx, vals, nnz);
    if (s != CG_OK) return s;
    Layout L;
    if ((s = check_ws(p, CG_OP_APPLY_CSR_I64, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    float *SX = reinterpret_cast<float *>(region(ws, L.a_off));
    cudaStream_t st = as_stream(stream);
    if ((s = run_sketch_csr_i64(p, row_ptr, col_idx, vals, nnz, SX, ws, L, st, true)) != CG_OK) return s;
    return run_contract(p, SX, Z, ws, L, st, false, imax, imin);
}

cg_status cg_sketch_csr_i64(cg_plan *p, const int64_t *row_ptr, const int32_t *col_idx, const float *vals,
                            int64_t nnz, float *SX, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_sketch_csr_i64");
    if (p == nullptr || SX == nullptr || misaligned(SX, 16)) return CG_ERR_INVALID_ARG;
    cg_status s = check_csr_i64(p, row_ptr, col_idx, vals, nnz);
    if (s != CG_OK) return s;
    Layout L;
    if ((s = check_ws(p, CG_OP_SKETCH_I64, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    return run_sketch_csr_i64(p, row_ptr, col_idx, vals, nnz, SX, ws, L, as_stream(stream), !p->accumulate);
}

cg_status cg_apply_right_csr(cg_plan *p, const int32_t *row_ptr, const int32_t *col_idx, const float *vals,
                             int64_t nnz, float *Z, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_apply_right_csr");
    if (p == nullptr || Z == nullptr || misaligned(Z, 4)) return CG_ERR_INVALID_ARG;
    cg_status s = check_csr(p, row_ptr, col_idx, vals, nnz, true);
    if (s != CG_OK) return s;
    if (p->deterministic) return CG_ERR_UNSUPPORTED;
    Layout L;
    if ((s = check_ws(p, CG_OP_APPLY_RIGHT_CSR, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    float *SX = reinterpret_cast<float *>(region(ws, L.a_off));
    cudaStream_t st = as_stream(stream);
    s = from_cuda(launch_right_scatter(row_ptr, col_idx, vals, p->d, p->n, static_cast<uint32_t>(p->B),
                                       static_cast<int>(nnz), make_key(p->seed), p->row_offset, region(ws, L.c_off),
                                       SX, status_word(ws), timing_pair(p, CG_KERNEL_SKETCH), st));
    if (s != CG_OK) return s;
    return run_contract(p, SX, Z, ws, L, st, true);
}

cg_status cg_apply_dense(cg_plan *p, const float *X, int64_t ldx, float *Y, void *ws, size_t ws_bytes,
                         void *stream) {
    cg::NvtxRange nvtx_range("cg_apply_dense");
    if (p == nullptr || Y == nullptr || misaligned(Y, 4) || ldx < p->d) return CG_ERR_INVALID_ARG;
    if (p->n > 0 && (X == nullptr || misaligned(X, 4))) return CG_ERR_INVALID_ARG;
    cg_status s;
    Layout L;
    if ((s = check_ws(p, CG_OP_APPLY_DENSE, 0, ws, ws_bytes, &L)) != CG_OK) return s;
    if (p->deterministic) return CG_ERR_UNSUPPORTED;
    float *SX = reinterpret_cast<float *>(region(ws, L.a_off));
    cudaStream_t st = as_stream(stream);
    s = from_cuda(launch_sketch_dense_atomic(X, ldx, static_cast<int>(p->n), p->d, static_cast<uint32_t>(p->B),
                                             make_key(p->seed), p->row_offset, SX, status_word(ws),
                                             static_cast<int>(p->sketch_ctas), timing_pair(p, CG_KERNEL_SKETCH), st));
    if (s != CG_OK) return s;
    return run_contract(p, SX, Y, ws, L, st);
}

cg_status cg_apply_adjoint(cg_plan *p, const float *dY, const int32_t *row_ptr, const int32_t *col_idx, int64_t nnz,
                           float *dX, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_apply_adjoint");
    if (p == nullptr || dY == nullptr || misaligned(dY, 4) || misaligned(dX, 4)) return CG_ERR_INVALID_ARG;
    const bool sparse = row_ptr != nullptr;
    cg_status s;
    if (sparse && (s = check_csr(p, row_ptr, col_idx, nullptr, nnz, false)) != CG_OK) return s;
    if ((sparse ? nnz : p->n) > 0 && dX == nullptr) return CG_ERR_INVALID_ARG;
    Layout L;
    if ((s = check_ws(p, sparse ? CG_OP_ADJOINT_CSR : CG_OP_ADJOINT_DENSE, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    float *W = reinterpret_cast<float *>(region(ws, L.a_off));
    cudaStream_t st = as_stream(stream);
    const Key key = make_key(p->seed);
    if ((s = from_cuda(launch_adjoint_w(dY, p->m, p->d, p->B, key, W, timing_pair(p, CG_KERNEL_ADJOINT_W), st))) !=
        CG_OK)
        return s;
    if (sparse)
        return from_cuda(launch_gather_csr(W, row_ptr, col_idx, static_cast<int>(p->n), p->d,
                                           static_cast<uint32_t>(p->B), static_cast<int>(nnz), key, p->row_offset,
                                           dX, status_word(ws), timing_pair(p, CG_KERNEL_GATHER), st));
    return from_cuda(launch_gather_dense(W, static_cast<int>(p->n), p->d, static_cast<uint32_t>(p->B), key,
                                         p->row_offset, dX, timing_pair(p, CG_KERNEL_GATHER), st));
}

cg_status cg_apply_adjoint_i64(cg_plan *p, const float *dY, const int64_t *row_ptr, const int32_t *col_idx,
                               int64_t nnz, float *dXv, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_apply_adjoint_i64");
    if (p == nullptr || dY == nullptr || misaligned(dY, 4) || misaligned(dXv, 4)) return CG_ERR_INVALID_ARG;
    if (nnz < 0 || nnz > kMaxNnz64 || row_ptr == nullptr || misaligned(row_ptr, 8)) return CG_ERR_INVALID_ARG;
    if (nnz > 0 && (col_idx == nullptr || dXv == nullptr || misaligned(col_idx, 4))) return CG_ERR_INVALID_ARG;
    cg_status s;
    Layout L;
    if ((s = check_ws(p, CG_OP_ADJOINT_CSR, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    float *W = reinterpret_cast<float *>(region(ws, L.a_off));
    cudaStream_t st = as_stream(stream);
    const Key key = make_key(p->seed);
    if ((s = from_cuda(launch_adjoint_w(dY, p->m, p->d, p->B, key, W, timing_pair(p, CG_KERNEL_ADJOINT_W), st))) !=
        CG_OK)
        return s;
    return from_cuda(launch_gather_csr_i64(W, reinterpret_cast<const long long *>(row_ptr), col_idx,
                                           static_cast<int>(p->n), p->d, static_cast<uint32_t>(p->B),
                                           static_cast<long long>(nnz), key, p->row_offset, dXv, status_word(ws),
                                           timing_pair(p, CG_KERNEL_GATHER), st));
}

cg_status cg_plain_gaussian_apply(cg_plan *p, const int32_t *row_ptr, const int32_t *col_idx, const float *vals,
                                  int64_t nnz, float *Y, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_plain_gaussian_apply");
    if (p == nullptr || Y == nullptr || misaligned(Y, 4)) return CG_ERR_INVALID_ARG;
    cg_status s = check_csr(p, row_ptr, col_idx, vals, nnz, true);
    if (s != CG_OK) return s;
    if (!plain_supported(p->m, p->d)) return CG_ERR_UNSUPPORTED;
    Layout L;
    if ((s = check_ws(p, CG_OP_PLAIN_CSR, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    return from_cuda(launch_plain_csr(row_ptr, col_idx, vals, static_cast<int>(p->n), p->d, p->m,
                                      static_cast<int>(nnz), make_key(p->seed), p->row_offset,
                                      reinterpret_cast<float *>(region(ws, L.b_off)), Y, status_word(ws),
                                      timing_pair(p, CG_KERNEL_PLAIN), as_stream(stream)));
}

cg_status cg_generate_words(uint64_t seed, uint32_t tag, uint64_t idx0, int64_t count, uint32_t *words,
                            void *stream) {
    if (count < 0 || (count > 0 && (words == nullptr || misaligned(words, 16)))) return CG_ERR_INVALID_ARG;
    if (count == 0) return CG_OK;
    return from_cuda(launch_generate_words(make_key(seed), tag, idx0, count, words, as_stream(stream)));
}

cg_status cg_generate_hash_sign(uint64_t seed, int64_t B, int64_t row0, int64_t count, int32_t *h, int32_t *sigma,
                                void *stream) {
    if (count < 0 || B < 1 || B > kMaxB || row0 < 0) return CG_ERR_INVALID_ARG;
    if (count > 0 && (h == nullptr || sigma == nullptr)) return CG_ERR_INVALID_ARG;
    if (count == 0) return CG_OK;
    return from_cuda(launch_generate_hash_sign(make_key(seed), static_cast<uint32_t>(B), row0, count, h, sigma,
                                               as_stream(stream)));
}

cg_status cg_generate_gaussian(uint64_t seed, uint32_t tag, int64_t R, int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                               float *out, void *stream) {
    if (R < 1 || r0 < 0 || r1 < r0 || r1 > R || c0 < 0 || c1 < c0) return CG_ERR_INVALID_ARG;
    if ((r1 - r0) * (c1 - c0) > 0 && out == nullptr) return CG_ERR_INVALID_ARG;
    if ((r1 - r0) * (c1 - c0) == 0) return CG_OK;
    return from_cuda(launch_generate_gaussian(make_key(seed), tag, R, r0, r1, c0, c1, out, as_stream(stream)));
}

cg_status cg_apply_csr_host(cg_plan *p, const int32_t *row_ptr, const int32_t *col_idx, const float *vals,
                            int64_t nnz, float *Y, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_apply_csr_host");
    if (p == nullptr || Y == nullptr || misaligned(Y, 4)) return CG_ERR_INVALID_ARG;
    cg_status s = check_csr(p, row_ptr, col_idx, vals, nnz, true);
    if (s != CG_OK) return s;
    if (p->deterministic || use_partition(*p)) return CG_ERR_UNSUPPORTED;
    Layout L;
    if ((s = check_ws(p, CG_OP_APPLY_CSR_HOST, nnz, ws, ws_bytes, &L)) != CG_OK) return s;
    const int64_t n = p->n;
    cudaStream_t st = as_stream(stream);
    float *SX = reinterpret_cast<float *>(region(ws, L.a_off));
    float *Yd = reinterpret_cast<float *>(region(ws, L.c_off));
    Layout Lrest = L;  // region C past Y: staging buffers, or the scatter's scratch
    Lrest.c_off = L.c_off + align256(static_cast<size_t>(p->m) * p->d * sizeof(float));
    if (row_ptr[0] < 0 || row_ptr[n] > nnz || row_ptr[0] > row_ptr[n]) return CG_ERR_INVALID_ARG;
    const int32_t *drp = nullptr, *dci = nullptr;
    const float *dv = nullptr;
    if (host_read_direct(*p, row_ptr, col_idx, vals, nnz, &drp, &dci, &dv)) {
        // the kernels stream the host arrays in place (offsets checked on the device)
        if ((s = run_sketch_csr(p, drp, dci, dv, nnz, SX, ws, Lrest, st, true, true)) != CG_OK) return s;
        if ((s = run_contract(p, SX, Yd, ws, L, st)) != CG_OK) return s;
        return from_cuda(cudaMemcpyAsync(Y, Yd, static_cast<size_t>(p->m) * p->d * sizeof(float),
                                         cudaMemcpyDeviceToHost, st));
    }
    const HostCaps caps = host_caps(*p, nnz);
    // Chunk boundaries [r0, r1): the most rows (at most caps.rows) whose nonzeros
    // row_ptr[r0] .. row_ptr[r1] number at most caps.nnz, by binary search.
    std::vector<int64_t> cuts{0};
    for (int64_t r0 = 0; r0 < n;) {
        const int64_t k0 = row_ptr[r0];
        auto fits = [&](int64_t r) { return row_ptr[r] >= k0 && row_ptr[r] - k0 <= caps.nnz && row_ptr[r] <= nnz; };
        int64_t lo = r0 + 1, hi = std::min(n, r0 + caps.rows);
        if (!fits(lo)) return row_ptr[lo] < k0 || row_ptr[lo] > nnz ? CG_ERR_INVALID_ARG : CG_ERR_UNSUPPORTED;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo + 1) / 2;
            if (fits(mid)) lo = mid; else hi = mid - 1;
        }
        cuts.push_back(lo);
        r0 = lo;
    }
    HostState *h = host_state(p);
    if (h == nullptr) return CG_ERR_CUDA;
    char *stage0 = region(ws, Lrest.c_off);
    const Key key = make_key(p->seed);
    if (cudaMemsetAsync(SX, 0, static_cast<size_t>(p->B) * p->d * sizeof(float), st) != cudaSuccess) return CG_ERR_CUDA;
    // The copies start after earlier work on `stream` and after the staging buffers'
    // last readers (a previous call, possibly on another stream).
    if (cudaEventRecord(h->start, st) != cudaSuccess || cudaStreamWaitEvent(h->copy, h->start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(h->copy, h->consumed[0], 0) != cudaSuccess ||
        cudaStreamWaitEvent(h->copy, h->consumed[1], 0) != cudaSuccess)
        return CG_ERR_CUDA;
    for (size_t c = 0; c + 1 < cuts.size(); ++c) {
        const int b = static_cast<int>(c & 1);
        const int64_t r0 = cuts[c], r1 = cuts[c + 1];
        const int64_t k0 = row_ptr[r0], k1 = row_ptr[r1];
        char *stage = stage0 + b * caps.stage_bytes;
        int32_t *rp = reinterpret_cast<int32_t *>(stage + caps.rp_off);
        int32_t *ci = reinterpret_cast<int32_t *>(stage + caps.ci_off);
        float *v = reinterpret_cast<float *>(stage + caps.v_off);
        if (c >= 2 && cudaStreamWaitEvent(h->copy, h->consumed[b], 0) != cudaSuccess) return CG_ERR_CUDA;
        if (cudaMemcpyAsync(rp, row_ptr + r0, static_cast<size_t>(r1 - r0 + 1) * sizeof(int32_t),
                            cudaMemcpyHostToDevice, h->copy) != cudaSuccess)
            return CG_ERR_CUDA;
        if (k1 > k0 && (cudaMemcpyAsync(ci, col_idx + k0, static_cast<size_t>(k1 - k0) * sizeof(int32_t),
                                        cudaMemcpyHostToDevice, h->copy) != cudaSuccess ||
                        cudaMemcpyAsync(v, vals + k0, static_cast<size_t>(k1 - k0) * sizeof(float),
                                        cudaMemcpyHostToDevice, h->copy) != cudaSuccess))
            return CG_ERR_CUDA;
        if (cudaEventRecord(h->copied[b], h->copy) != cudaSuccess || cudaStreamWaitEvent(st, h->copied[b], 0) != cudaSuccess)
            return CG_ERR_CUDA;
        if (launch_sketch_csr_rows_chunk(rp, ci, v, static_cast<int>(r1 - r0), p->d, static_cast<uint32_t>(p->B),
                                         static_cast<int>(k0), static_cast<int>(k1), key, p->row_offset + r0, SX,
                                         status_word(ws), static_cast<int>(p->sketch_ctas), p->scatter_rows,
                                         st) != cudaSuccess)
            return CG_ERR_CUDA;
        if (cudaEventRecord(h->consumed[b], st) != cudaSuccess) return CG_ERR_CUDA;
    }
    if ((s = run_contract(p, SX, Yd, ws, L, st)) != CG_OK) return s;
    return from_cuda(cudaMemcpyAsync(Y, Yd, static_cast<size_t>(p->m) * p->d * sizeof(float), cudaMemcpyDeviceToHost,
                                     st));
}

cg_status cg_diag_random_reductions(float *array, int64_t cells, int64_t count, void *stream) {
    cg::NvtxRange nvtx_range("cg_diag_random_reductions");
    if (array == nullptr || misaligned(array, 4) || cells < 1 || cells >= (1LL << 32) || count < 0 ||
        count >= (1LL << 32))
        return CG_ERR_INVALID_ARG;
    if (count == 0) return CG_OK;
    random_reductions_kernel<<<sketch_default_ctas(), 256, 0, as_stream(stream)>>>(
        array, static_cast<uint32_t>(cells), static_cast<uint32_t>(count));
    return from_cuda(cudaGetLastError());
}

}  // extern "C"

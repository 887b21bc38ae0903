// cg_noalloc.cu -- cg_apply_csr_noalloc: the CSR transform with its scratch memory in a
// fixed, file-scope device array instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they want the
// transform: code running under an allocator that must not be re-entered (inside a
// memory-pool callback or a custom allocator's own bookkeeping), plugins that are
// handed only input and output buffers by a host framework that owns all device
// allocations, and real-time loops that forbid cudaMalloc/cudaFree after start-up
// because those calls can synchronise the device and take unbounded time.  For them
// this entry point needs no workspace: the sketch SX, the split-K partials and the
// status word live in `g_noalloc_scratch` below, which the CUDA runtime places in
// device memory when the library's module is loaded on a device (every GPU that
// loads the library holds these bytes until the process exits).
//
// Host code never dereferences `g_noalloc_scratch`: on the host the name denotes a
// host-side shadow, not a device address, so its device address is looked up with
// cudaGetSymbolAddress (with the device current) and passed to the kernels as a plain
// pointer.  The lookup is made once per device and context: a device reset or a new
// context reloads the module, and the array may then sit elsewhere, so the cached address
// is keyed by the current context's unique id (cuCtxGetId, reached through the runtime's
// driver entry points) and looked up again when the id changes.
#include <cudaTypedefs.h>

#include <mutex>

#include "cg_internal.cuh"

namespace {

constexpr size_t kScratchBytes = CG_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};

// The unique id of the context current on this thread (0 when there is none yet, or when
// the driver does not offer the calls).
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current == nullptr || get_id == nullptr || get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_noalloc_scratch on the current device, looked up on the first call
// in each context (the lookup loads this file's module if it is not loaded yet).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long ctx = current_context_id();
    if (g_scratch_ptr[dev] == nullptr || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = current_context_id();  // the lookup made the context current if none was
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

bool misaligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; }

}  // namespace

extern "C" cg_status cg_apply_csr_noalloc(cg_plan *p, const int32_t *row_ptr, const int32_t *col_idx,
                                          const float *vals, int64_t nnz, float *Y, void *stream) {
    cg::NvtxRange nvtx_range("cg_apply_csr_noalloc");
    using namespace cg;
    if (p == nullptr || Y == nullptr || row_ptr == nullptr || misaligned(Y, 4)) return CG_ERR_INVALID_ARG;
    if (nnz < 0 || nnz > kMaxNnz) return CG_ERR_INVALID_ARG;
    if (nnz > 0 && (col_idx == nullptr || vals == nullptr)) return CG_ERR_INVALID_ARG;
    if (misaligned(row_ptr, 4) || misaligned(col_idx, 4) || misaligned(vals, 4)) return CG_ERR_INVALID_ARG;
    if (p->precision != CG_PREC_FP32 || p->deterministic) return CG_ERR_UNSUPPORTED;

    // Scratch layout: [status 256 B][SX: B x d floats][split-K partials], 256-aligned.
    const size_t sx_bytes = align256(static_cast<size_t>(p->B) * p->d * sizeof(float));
    const int nsplit = contract_splits(*p);
    const size_t part_bytes = align256(static_cast<size_t>(nsplit) * p->m * p->d * sizeof(float));
    if (kStatusBytes + sx_bytes + part_bytes > kScratchBytes) return CG_ERR_WORKSPACE;

    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return CG_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *scratch = static_cast<char *>(base);
    int *status = reinterpret_cast<int *>(scratch);
    float *SX = reinterpret_cast<float *>(scratch + kStatusBytes);
    float *partials = reinterpret_cast<float *>(scratch + kStatusBytes + sx_bytes);

    // The array keeps the previous call's contents: the status word is cleared here,
    // SX is cleared by the scatter launcher and the partials are fully overwritten.
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return CG_ERR_CUDA;
    if (launch_sketch_csr_atomic(row_ptr, col_idx, vals, static_cast<int>(p->n), p->d, static_cast<uint32_t>(p->B),
                                 static_cast<int>(nnz), make_key(p->seed), p->row_offset, SX, status,
                                 static_cast<int>(p->sketch_ctas), p->scatter_passes, one_pass_rows(*p, nnz), nullptr,
                                 st) != cudaSuccess)
        return CG_ERR_CUDA;
    if (launch_contract_ffma(SX, p->m, p->d, p->B, make_key(p->seed), nsplit, partials, Y, nullptr, st) !=
        cudaSuccess)
        return CG_ERR_CUDA;
    return CG_OK;
}

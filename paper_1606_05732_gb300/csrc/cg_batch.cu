// cg_batch.cu -- many CountGauss instances of uneven n, d, m and B (each with its own
// seed, CSR input and output) in one persistent launch; each instance is the transform
// T.X = G.(S.X) of Section 1.1 (Algorithm 1 steps 1-2).
//
// Work items live in a queue in device memory and are claimed in order with one
// atomic per claim by persistent CTAs:
//   scatter items   rows [a, b) of instance k  -> SX_k   (as cg_apply_csr's scatter)
//   contract items  K slabs of instance k      -> partial_k[g]  (FFMA, G generated in
//                   shared memory), after all scatter items of k are done
// Every scatter item precedes every contract item in the queue, so when a CTA claims a
// contract item every scatter item has already been claimed by a running CTA that never
// waits: the wait on instance k's scatter counter always ends.  It is bounded anyway
// (about two seconds of SM clock by default); on expiry the item sets the timeout bit
// of the status word and contributes zeros.  The partials are summed in a fixed order in
// two levels: the item that completes a group of 32 items adds their partials, the one
// that completes the last group adds the group sums into Y_k.
//
// The plan sizes the items (target nonzeros per scatter item, target FMAs per contract
// item, CTAs per SM); cg_batch_autotune times a small grid of these choices on the
// actual batch and keeps the fastest.  cg_batch_apply records the memset and the launch
// once in a CUDA graph and replays it on later calls with the same workspace.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "cg_ffma.cuh"
#include "cg_internal.cuh"
#include "cg_scatter.cuh"

namespace cg {

namespace {

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int kMaxContractItems = 1024;  // per instance (bounds the partials buffer)
constexpr int kSumGroup = 32;            // partials summed per group in the two-level sum
constexpr int kMaxGroups = kMaxContractItems / kSumGroup;
constexpr int kMaxRowsPerItem = 16384;  // per scatter item
constexpr int kNormalCost = 48;         // FMA-equivalents per Gaussian drawn (item sizing)

struct BatchInst {
    const int *row_ptr;
    const int *col_idx;
    const float *vals;
    float *SX;
    float *partials;  // [part_cap] item partials, then [kMaxGroups] group sums, each m x d
    float *Y;
    int n, d, m, nnz;
    uint32_t B;
    Key key;
    int n_s, n_g;     // scatter / contract items of this instance
    int part_cap;     // item partial slots before the group sums
    int lanes;        // 1: scatter one row per lane (instances with under one nonzero per row)
    int slabs_per_g;  // 32-wide K slabs per contract item
    int rows_per_s;   // rows per scatter item
};

struct BatchItem {
    int inst;
    int kind;  // 0: scatter rows [a, b); 1: contract item a
    int a, b;
};

// out[o] = slots[g0][o] + slots[g0 + 1][o] + ... + slots[g1 - 1][o] in that order, for
// o < md (slots are md floats apart); each thread keeps kSumOut outputs (stride
// kBThreads), so kSumOut loads are in flight.  Called by all threads of the CTA.
__device__ __forceinline__ void sum_slots(const float *slots, int g0, int g1, int md, float *out) {
    constexpr int kSumOut = 16;
    const int t = threadIdx.x;
    for (int base = t; base < md; base += kBThreads * kSumOut) {
        float acc[kSumOut];
#pragma unroll
        for (int k = 0; k < kSumOut; ++k) acc[k] = 0.0f;
        for (int g = g0; g < g1; ++g) {
            const float *p = slots + static_cast<size_t>(g) * md + base;
#pragma unroll
            for (int k = 0; k < kSumOut; ++k)
                if (base + k * kBThreads < md) acc[k] += __ldcg(p + k * kBThreads);
        }
#pragma unroll
        for (int k = 0; k < kSumOut; ++k)
            if (base + k * kBThreads < md) out[base + k * kBThreads] = acc[k];
    }
}

// Hint: bring [p, p + bytes) into L2, trimmed inward to whole 16-byte units (so it never
// reaches outside the range); nothing waits on it.
__device__ __forceinline__ void prefetch_l2_range(const void *p, size_t bytes) {
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~static_cast<uintptr_t>(15);
    const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes) & ~static_cast<uintptr_t>(15);
    for (uintptr_t q = a; q < e; q += (1u << 20)) {  // at most 1 MB per hint
        const uint32_t len = static_cast<uint32_t>(e - q < (1u << 20) ? e - q : (1u << 20));
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(len) : "memory");
    }
}

// Rows [first, min(first + 32 kCompactK, last)) of a very sparse instance, one non-empty
// row per lane: the warp first reads the rows' offsets (coalesced, 32 rows per step) and
// packs the indices of the non-empty ones into s_list (ballot order, so row order);
// then lanes take them 32 at a time, hash them and walk their nonzeros.  A warp hashes
// once per 32 non-empty rows instead of once per 32 rows (most rows of such instances
// are empty).  Out-of-range column indices and malformed offsets are skipped and
// reported through `bad`.
constexpr int kCompactK = 8;

__device__ __forceinline__ void scatter_lanes_compact(const int *__restrict__ row_ptr, const int *__restrict__ col_idx,
                                                      const float *__restrict__ vals, int first, int last, int d,
                                                      uint32_t B, int nnz, Key key, float *__restrict__ SX,
                                                      int *s_list, int &bad) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int count = 0;
#pragma unroll
    for (int k = 0; k < kCompactK; ++k) {
        const int i = first + 32 * k + lane;
        const int beg = i < last ? __ldg(row_ptr + i) : 0;
        int end = __shfl_down_sync(0xffffffffu, beg, 1);  // row_ptr[i + 1] from the next lane
        if (i < last && (lane == 31 || i + 1 == last)) end = __ldg(row_ptr + i + 1);
        bool live = false;
        if (i < last) {
            if (beg < 0 || end > nnz || beg > end)
                bad = 1;  // malformed offsets: skip the row
            else
                live = beg < end;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, live);
        if (live) s_list[count + __popc(mask & below)] = i;
        count += __popc(mask);
    }
    __syncwarp();
    for (int base = 0; base < count; base += 32) {
        if (base + lane < count) {
            const int i = s_list[base + lane];
            const int beg = __ldg(row_ptr + i), end = __ldg(row_ptr + i + 1);
            uint32_t h;
            float sg;
            hash_sign(key, static_cast<uint64_t>(i), B, h, sg);
            const size_t row0 = static_cast<size_t>(h) * d;
            for (int k = beg; k < end; ++k) {
                const int j = __ldg(col_idx + k);
                if (static_cast<unsigned>(j) < static_cast<unsigned>(d))
                    atomicAdd(SX + row0 + j, sg * __ldg(vals + k));
                else
                    bad = 1;
            }
        }
    }
    __syncwarp();
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kBThreads, 4)  // four CTAs per SM fit (at most 64 registers)
batch_kernel(const BatchInst *__restrict__ insts, const BatchItem *__restrict__ items, int n_items,
             int *__restrict__ head, int *__restrict__ s_done, int *__restrict__ g_done, int *__restrict__ grp_done,
             long long wait_cycles,
             int *__restrict__ status) {
    __shared__ __align__(16) float raw[FfmaShape<4>::kRawFloats];
    __shared__ int s_rp[kBWarps][33];
    __shared__ uint32_t s_h[kBWarps][32];
    __shared__ float s_sg[kBWarps][32];
    __shared__ int s_list[kBWarps][32 * kCompactK];
    __shared__ int s_item, s_flag;
    const int t = threadIdx.x;
    const int w = t >> 5;
    int bad = 0;
    for (;;) {
        if (t == 0) s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem item = items[it];
        const BatchInst I = insts[item.inst];
        if (item.kind == 0) {
            // The item's row offsets and nonzeros into L2 first: each warp's loads are
            // otherwise one DRAM round trip per 32 rows, which dominates very sparse
            // instances (mostly empty rows).
            if (t == 0) {
                prefetch_l2_range(I.row_ptr + item.a, static_cast<size_t>(item.b - item.a + 1) * sizeof(int));
                const int k0 = I.row_ptr[item.a], k1 = I.row_ptr[item.b];
                if (0 <= k0 && k0 < k1 && k1 <= I.nnz) {
                    prefetch_l2_range(I.col_idx + k0, static_cast<size_t>(k1 - k0) * sizeof(int));
                    prefetch_l2_range(I.vals + k0, static_cast<size_t>(k1 - k0) * sizeof(float));
                }
            }
            if (I.lanes) {  // CTA-uniform
                for (int first = item.a + w * 32 * kCompactK; first < item.b; first += kBWarps * 32 * kCompactK)
                    scatter_lanes_compact(I.row_ptr, I.col_idx, I.vals, first, item.b, I.d, I.B, I.nnz, I.key, I.SX,
                                          s_list[w], bad);
            } else {
                for (int first = item.a + w * 32; first < item.b; first += kBWarps * 32)
                    scatter_chunk32<false, true>(I.row_ptr, I.col_idx, I.vals, first, item.b, I.d, I.B, I.nnz, I.key,
                                                 0, I.SX, 0, s_rp[w], s_h[w], s_sg[w], bad);
            }
            __syncthreads();
            if (t == 0) {
                __threadfence();
                atomicAdd(&s_done[item.inst], 1);
            }
            continue;
        }
        if (t == 0) {
            int ok = 1;
            const long long t0 = clock64();
            while (ld_acquire(&s_done[item.inst]) < I.n_s) {
                if (clock64() - t0 > wait_cycles) {
                    ok = 0;
                    atomicOr(status, kStatusTimeout);
                    break;
                }
                __nanosleep(200);
            }
            s_flag = ok;
        }
        __syncthreads();
        const int ok = s_flag;
        __threadfence();
        const int64_t nslabs = (static_cast<int64_t>(I.B) + kFfmaKT - 1) / kFfmaKT;
        const int64_t s0 = static_cast<int64_t>(item.a) * I.slabs_per_g;
        const int64_t s1 = ok ? min(nslabs, s0 + I.slabs_per_g) : s0;  // no slabs after a timeout: zeros
        float *part = I.partials + static_cast<size_t>(item.a) * I.m * I.d;
        for (int m0 = 0; m0 < I.m; m0 += kFfmaBM)
            for (int n0 = 0; n0 < I.d; n0 += FfmaShape<4>::BN) {
                ffma_block<4, true>(I.SX, I.m, I.d, static_cast<int64_t>(I.B), I.key, s0, s1, m0, n0, (I.d & 3) == 0,
                                    part, raw);
                __syncthreads();
            }
        // Two-level sum in a fixed order: the last item of each group of kSumGroup items
        // adds the group's partials (in item order) into its group slot; the last group
        // to finish adds the group slots (in group order) into Y.
        const int md = I.m * I.d;
        const int gamma = item.a / kSumGroup;
        const int ngroups = (I.n_g + kSumGroup - 1) / kSumGroup;
        const int g_lo = gamma * kSumGroup;
        const int g_hi = min(I.n_g, g_lo + kSumGroup);
        float *gslots = I.partials + static_cast<size_t>(I.part_cap) * md;
        if (t == 0) {
            __threadfence();
            s_flag = atomicAdd(&grp_done[item.inst * kMaxGroups + gamma], 1) == g_hi - g_lo - 1;
        }
        __syncthreads();
        if (s_flag) {
            __threadfence();
            sum_slots(I.partials, g_lo, g_hi, md, gslots + static_cast<size_t>(gamma) * md);
            __threadfence();
            __syncthreads();
            if (t == 0) s_flag = atomicAdd(&g_done[item.inst], 1) == ngroups - 1;
            __syncthreads();
            if (s_flag) {
                __threadfence();
                sum_slots(gslots, 0, ngroups, md, I.Y);
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(status, kStatusBounds);
}

}  // namespace
}  // namespace cg

using namespace cg;

struct cg_batch_plan {
    std::vector<cg_batch_desc> descs;
    // tuning
    int64_t s_nnz = 16384;       // target nonzeros per scatter item
    int64_t g_fma = 1 << 22;     // target FMAs per contract item
    int32_t ctas_per_sm = 4;
    int32_t use_graph = 1;
    int64_t wait_us = 2000000;
    int32_t drop_item = 0;       // test hook: leave the first scatter item of instance 0 out of the queue
    // derived
    std::vector<BatchInst> insts;
    std::vector<BatchItem> items;
    std::vector<size_t> sx_off, part_off;
    size_t counters_off = 0, counters_bytes = 0, insts_off = 0, items_off = 0, total = 0;
    size_t zero_bytes = 0;  // counters + SX areas, cleared at every apply
    // upload / graph state
    void *uploaded_ws = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

// Contract items of an instance: at most one per 32-wide slab of B, and kMaxContractItems.
int64_t max_contract_items(int64_t B) {
    const int64_t nslabs = (B + kFfmaKT - 1) / kFfmaKT;
    return std::max<int64_t>(1, std::min<int64_t>(kMaxContractItems, nslabs));
}

int64_t pow2_floor(int64_t x) {
    int64_t p = 1;
    while (p * 2 <= x) p *= 2;
    return p;
}

// Sizes the items of every instance and lays out the workspace (host only).
void build(cg_batch_plan &P) {
    const int count = static_cast<int>(P.descs.size());
    P.insts.assign(count, BatchInst{});
    P.items.clear();
    P.sx_off.assign(count, 0);
    P.part_off.assign(count, 0);
    size_t off = kStatusBytes;
    P.counters_off = off;
    P.counters_bytes = (1 + (2 + kMaxGroups) * static_cast<size_t>(count)) * sizeof(int);
    off += align256(P.counters_bytes);
    for (int k = 0; k < count; ++k) {
        P.sx_off[k] = off;
        off += align256(static_cast<size_t>(P.descs[k].B) * P.descs[k].d * sizeof(float));
    }
    P.zero_bytes = off - P.counters_off;
    for (int k = 0; k < count; ++k) {
        P.part_off[k] = off;
        off += align256(static_cast<size_t>(max_contract_items(P.descs[k].B) + kMaxGroups) * P.descs[k].m *
                        P.descs[k].d * sizeof(float));
    }
    P.insts_off = off;
    off += align256(static_cast<size_t>(count) * sizeof(BatchInst));
    P.items_off = off;
    std::vector<int> order(count);
    for (int k = 0; k < count; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return P.descs[a].nnz > P.descs[b].nnz; });  // largest first
    for (int k = 0; k < count; ++k) {
        const cg_batch_desc &D = P.descs[k];
        BatchInst &I = P.insts[k];
        I.n = static_cast<int>(D.n);
        I.d = D.d;
        I.m = D.m;
        I.nnz = static_cast<int>(D.nnz);
        I.B = static_cast<uint32_t>(D.B);
        I.key = make_key(D.seed);
        const double per_row = D.n > 0 ? static_cast<double>(D.nnz) / static_cast<double>(D.n) : 1.0;
        // rows per scatter item: about s_nnz nonzeros, but at most kMaxRowsPerItem rows, so
        // that an item of a very sparse instance (mostly empty rows) stays short
        int64_t rows = pow2_floor(static_cast<int64_t>(static_cast<double>(P.s_nnz) / std::max(per_row, 1e-3)));
        rows = std::max<int64_t>(32, std::min<int64_t>(rows, kMaxRowsPerItem));
        I.n_s = static_cast<int>((D.n + rows - 1) / rows);
        const int64_t nslabs = (D.B + kFfmaKT - 1) / kFfmaKT;
        // slabs per contract item: about g_fma "FMA-equivalents", counting each Gaussian
        // drawn as kNormalCost FMAs (a Philox + Box-Muller quadruple is ~200 instructions)
        const int64_t slab_cost = static_cast<int64_t>(D.m) * kFfmaKT * (D.d + kNormalCost);
        int64_t spg = (P.g_fma + slab_cost - 1) / slab_cost;
        const int64_t cap = max_contract_items(D.B);
        spg = std::max<int64_t>(spg, (nslabs + cap - 1) / cap);
        spg = std::max<int64_t>(1, std::min(spg, nslabs));
        I.slabs_per_g = static_cast<int>(spg);
        I.n_g = static_cast<int>((nslabs + spg - 1) / spg);
        I.part_cap = static_cast<int>(cap);
        I.rows_per_s = static_cast<int>(rows);
        I.lanes = per_row < 1.0 ? 1 : 0;
    }
    for (int k : order) {
        const BatchInst &I = P.insts[k];
        const int64_t rows = I.rows_per_s;
        for (int s = 0; s < I.n_s; ++s) {
            if (P.drop_item && k == 0 && s == 0) continue;
            const int64_t a = s * rows;
            P.items.push_back(BatchItem{k, 0, static_cast<int>(a), static_cast<int>(std::min<int64_t>(a + rows, I.n))});
        }
    }
    // Contract items longest first (FMAs per item), so that the short ones fill the end of
    // the queue and no long item starts last.
    std::vector<int> gorder(count);
    for (int k = 0; k < count; ++k) gorder[k] = k;
    auto item_fma = [&](int k) {
        return static_cast<int64_t>(P.insts[k].slabs_per_g) * P.insts[k].m * P.insts[k].d;
    };
    std::stable_sort(gorder.begin(), gorder.end(), [&](int a, int b) { return item_fma(a) > item_fma(b); });
    for (int k : gorder)
        for (int g = 0; g < P.insts[k].n_g; ++g) P.items.push_back(BatchItem{k, 1, g, 0});
    // queue capacity for the smallest scatter item (32 rows), so that no tiling choice
    // outgrows the workspace
    size_t cap_items = 1;
    for (int k = 0; k < count; ++k)
        cap_items += static_cast<size_t>((P.descs[k].n + 31) / 32) + kMaxContractItems;
    off += align256(cap_items * sizeof(BatchItem));
    P.total = off;
}

void drop_graph(cg_batch_plan &P) {
    if (P.exec != nullptr) cudaGraphExecDestroy(P.exec);
    P.exec = nullptr;
}

cg_status upload(cg_batch_plan &P, void *ws, cudaStream_t st) {
    char *base = static_cast<char *>(ws);
    std::vector<BatchInst> dev = P.insts;
    for (size_t k = 0; k < dev.size(); ++k) {
        dev[k].row_ptr = P.descs[k].row_ptr;
        dev[k].col_idx = P.descs[k].col_idx;
        dev[k].vals = P.descs[k].vals;
        dev[k].Y = P.descs[k].Y;
        dev[k].SX = reinterpret_cast<float *>(base + P.sx_off[k]);
        dev[k].partials = reinterpret_cast<float *>(base + P.part_off[k]);
    }
    if (cudaMemcpyAsync(base + P.insts_off, dev.data(), dev.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return CG_ERR_CUDA;
    if (!P.items.empty() && cudaMemcpyAsync(base + P.items_off, P.items.data(), P.items.size() * sizeof(BatchItem),
                                            cudaMemcpyHostToDevice, st) != cudaSuccess)
        return CG_ERR_CUDA;
    P.uploaded_ws = ws;
    drop_graph(P);
    return CG_OK;
}

cudaError_t enqueue(cg_batch_plan &P, void *ws, cudaStream_t st) {
    char *base = static_cast<char *>(ws);
    cudaError_t e = cudaMemsetAsync(base + P.counters_off, 0, P.zero_bytes, st);
    if (e != cudaSuccess) return e;
    if (P.items.empty()) return cudaSuccess;
    const int count = static_cast<int>(P.descs.size());
    int *head = reinterpret_cast<int *>(base + P.counters_off);
    int *s_done = head + 1;
    int *g_done = s_done + count;
    int *grp_done = g_done + count;
    const int sms = num_sms() > 0 ? num_sms() : 148;
    const int grid = std::max(1, std::min<int>(sms * P.ctas_per_sm, static_cast<int>(P.items.size())));
    const long long cycles = static_cast<long long>(P.wait_us) * 2000;  // ~2 GHz SM clock
    batch_kernel<<<grid, kBThreads, 0, st>>>(reinterpret_cast<const BatchInst *>(base + P.insts_off),
                                            reinterpret_cast<const BatchItem *>(base + P.items_off),
                                            static_cast<int>(P.items.size()), head, s_done, g_done, grp_done, cycles,
                                            reinterpret_cast<int *>(ws));
    return cudaGetLastError();
}

cg_status run(cg_batch_plan &P, void *ws, cudaStream_t st) {
    if (!P.use_graph) return enqueue(P, ws, st) == cudaSuccess ? CG_OK : CG_ERR_CUDA;
    if (P.exec == nullptr) {
        if (P.cap_stream == nullptr &&
            cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return CG_ERR_CUDA;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CG_ERR_CUDA;
        const cudaError_t e1 = enqueue(P, ws, P.cap_stream);
        const cudaError_t e2 = cudaStreamEndCapture(P.cap_stream, &g);
        if (e1 != cudaSuccess || e2 != cudaSuccess || g == nullptr) {
            if (g != nullptr) cudaGraphDestroy(g);
            cudaGetLastError();
            return CG_ERR_CUDA;
        }
        const cudaError_t e3 = cudaGraphInstantiate(&P.exec, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) {
            P.exec = nullptr;
            return CG_ERR_CUDA;
        }
    }
    return cudaGraphLaunch(P.exec, st) == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

bool valid_desc(const cg_batch_desc &D) {
    if (D.n < 0 || D.n > kMaxRows || D.d < 1 || D.d > 65536 || D.m < 1 || D.m > 65536) return false;
    if (D.B < 1 || D.B > (1LL << 31) - 1 || D.B * static_cast<int64_t>(D.d) >= (1LL << 40)) return false;
    if (D.nnz < 0 || D.nnz > kMaxNnz || D.row_ptr == nullptr || D.Y == nullptr) return false;
    if (D.nnz > 0 && (D.col_idx == nullptr || D.vals == nullptr)) return false;
    return true;
}

}  // namespace

extern "C" {

cg_status cg_batch_plan_create(const cg_batch_desc *descs, int32_t count, cg_batch_plan **out) {
    if (out == nullptr) return CG_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 0 || (count > 0 && descs == nullptr)) return CG_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k)
        if (!valid_desc(descs[k])) return CG_ERR_INVALID_ARG;
    cg_batch_plan *P = new (std::nothrow) cg_batch_plan;
    if (P == nullptr) return CG_ERR_INVALID_ARG;
    P->descs.assign(descs, descs + count);
    build(*P);
    *out = P;
    return CG_OK;
}

cg_status cg_batch_plan_destroy(cg_batch_plan *P) {
    if (P == nullptr) return CG_OK;
    drop_graph(*P);
    if (P->cap_stream != nullptr) cudaStreamDestroy(P->cap_stream);
    delete P;
    return CG_OK;
}

cg_status cg_batch_set_option(cg_batch_plan *P, int32_t option, int64_t value) {
    if (P == nullptr) return CG_ERR_INVALID_ARG;
    switch (option) {
        case CG_BATCH_OPT_GRAPH:
            if (value != 0 && value != 1) return CG_ERR_INVALID_ARG;
            P->use_graph = static_cast<int32_t>(value);
            break;
        case CG_BATCH_OPT_SCATTER_NNZ:
            if (value < 32 || value > (1 << 26)) return CG_ERR_INVALID_ARG;
            P->s_nnz = value;
            break;
        case CG_BATCH_OPT_CONTRACT_FMA:
            if (value < 1024 || value > (1LL << 34)) return CG_ERR_INVALID_ARG;
            P->g_fma = value;
            break;
        case CG_BATCH_OPT_CTAS_PER_SM:
            if (value < 1 || value > 8) return CG_ERR_INVALID_ARG;
            P->ctas_per_sm = static_cast<int32_t>(value);
            break;
        case CG_BATCH_OPT_WAIT_US:
            if (value < 1 || value > 60000000) return CG_ERR_INVALID_ARG;
            P->wait_us = value;
            break;
        case CG_BATCH_OPT_TEST_DROP_SCATTER_ITEM:
            if (value != 0 && value != 1) return CG_ERR_INVALID_ARG;
            P->drop_item = static_cast<int32_t>(value);
            break;
        default:
            return CG_ERR_INVALID_ARG;
    }
    build(*P);
    P->uploaded_ws = nullptr;
    drop_graph(*P);
    return CG_OK;
}

cg_status cg_batch_plan_get_option(const cg_batch_plan *P, int32_t option, int64_t *value) {
    if (P == nullptr || value == nullptr) return CG_ERR_INVALID_ARG;
    switch (option) {
        case CG_BATCH_OPT_GRAPH: *value = P->use_graph; return CG_OK;
        case CG_BATCH_OPT_SCATTER_NNZ: *value = P->s_nnz; return CG_OK;
        case CG_BATCH_OPT_CONTRACT_FMA: *value = P->g_fma; return CG_OK;
        case CG_BATCH_OPT_CTAS_PER_SM: *value = P->ctas_per_sm; return CG_OK;
        case CG_BATCH_OPT_WAIT_US: *value = P->wait_us; return CG_OK;
        case CG_BATCH_OPT_TEST_DROP_SCATTER_ITEM: *value = P->drop_item; return CG_OK;
        default: return CG_ERR_INVALID_ARG;
    }
}

cg_status cg_batch_workspace_size(const cg_batch_plan *P, size_t *bytes) {
    if (P == nullptr || bytes == nullptr) return CG_ERR_INVALID_ARG;
    *bytes = P->total;
    return CG_OK;
}

cg_status cg_batch_apply(cg_batch_plan *P, void *ws, size_t ws_bytes, void *stream) {
    cg::NvtxRange nvtx_range("cg_batch_apply");
    if (P == nullptr || ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return CG_ERR_INVALID_ARG;
    if (ws_bytes < P->total) return CG_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (P->uploaded_ws != ws) {
        const cg_status s = upload(*P, ws, st);
        if (s != CG_OK) return s;
    }
    return run(*P, ws, st);
}

cg_status cg_batch_check(const cg_batch_plan *P, void *ws, void *stream) {
    if (P == nullptr || ws == nullptr) return CG_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int h = 0;
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

cg_status cg_batch_autotune(cg_batch_plan *P, void *ws, size_t ws_bytes, void *stream, int32_t reps, double *best_ms) {
    cg::NvtxRange nvtx_range("cg_batch_autotune");
    if (P == nullptr || ws == nullptr || reps < 1 || (reinterpret_cast<uintptr_t>(ws) & 255) != 0)
        return CG_ERR_INVALID_ARG;
    if (ws_bytes < P->total) return CG_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t s_cands[] = {4096, 16384, 65536};
    const int64_t g_cands[] = {1 << 20, 1 << 22, 1 << 24};
    const int32_t c_cands[] = {2, 4};
    const int32_t graph = P->use_graph;
    P->use_graph = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return CG_ERR_CUDA;
    float best = 3.0e38f;
    int64_t bs = P->s_nnz, bg = P->g_fma;
    int32_t bc = P->ctas_per_sm;
    cg_status status = CG_OK;
    for (int64_t sc : s_cands)
        for (int64_t gc : g_cands)
            for (int32_t cc : c_cands) {
                P->s_nnz = sc;
                P->g_fma = gc;
                P->ctas_per_sm = cc;
                build(*P);
                if (P->total > ws_bytes) continue;  // the workspace size does not depend on the tiling
                if ((status = upload(*P, ws, st)) != CG_OK) break;
                if (enqueue(*P, ws, st) != cudaSuccess) { status = CG_ERR_CUDA; break; }
                cudaEventRecord(a, st);
                for (int r = 0; r < reps; ++r) enqueue(*P, ws, st);
                cudaEventRecord(b, st);
                float ms = 0.0f;
                if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
                    status = CG_ERR_CUDA;
                    break;
                }
                if (ms < best) {
                    best = ms;
                    bs = sc;
                    bg = gc;
                    bc = cc;
                }
            }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    P->s_nnz = bs;
    P->g_fma = bg;
    P->ctas_per_sm = bc;
    P->use_graph = graph;
    build(*P);
    P->uploaded_ws = nullptr;
    drop_graph(*P);
    if (best_ms != nullptr) *best_ms = best < 3.0e38f ? best / reps : -1.0;
    return status;
}

}  // extern "C"

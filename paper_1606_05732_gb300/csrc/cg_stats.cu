// cg_stats.cu -- FP64 reductions of the distribution checker.
//
// The claims the transform is built on are statements about distributions: given S,
// each row of G.S.X is N(0, X^T S^T S X) (Section 7), and rows of T.X and of the plain
// G~.X are close to / equal to N(0, X^T X) (Theorem 1).  The checker draws many
// samples of those rows with the library's own kernels and reduces them here:
//   gram  += Y^T Y      (d x d, FP64; the sample second-moment matrix up to 1/rows)
//   sumsq += ||Y||_F^2  (FP64)
// This is the only FP64 arithmetic on the GPU.
#include "cg_internal.cuh"

namespace cg {

namespace {

constexpr int kTile = 32;
constexpr int kRowsPerStep = 32;

// CTA (bi, bj): gram[32 bi .. +32, 32 bj .. +32) += sum over rows of y_i y_j; each
// thread owns 4 entries (one i, four j), rows staged 32 at a time in shared memory.
__global__ void __launch_bounds__(256)
gram_f64_kernel(const float *__restrict__ Y, int64_t rows, int d, int64_t rows_per_cta, double *__restrict__ gram) {
    __shared__ double ys[kRowsPerStep][2 * kTile + 1];
    const int i0 = blockIdx.x * kTile;
    const int j0 = blockIdx.y * kTile;
    const int t = threadIdx.x;
    const int ti = t & 31;  // i offset
    const int tj = t >> 5;  // j offsets tj, tj + 8, tj + 16, tj + 24
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t r_begin = static_cast<int64_t>(blockIdx.z) * rows_per_cta;
    const int64_t r_end = min(rows, r_begin + rows_per_cta);
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kRowsPerStep) {
        for (int e = t; e < kRowsPerStep * 2 * kTile; e += 256) {
            const int rr = e / (2 * kTile);
            const int cc = e % (2 * kTile);
            const int col = cc < kTile ? i0 + cc : j0 + cc - kTile;
            const int64_t r = r0 + rr;
            ys[rr][cc] = (r < r_end && col < d) ? static_cast<double>(Y[r * d + col]) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kRowsPerStep; ++rr) {
            const double yi = ys[rr][ti];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(yi, ys[rr][kTile + tj + 8 * q], acc[q]);
        }
        __syncthreads();
    }
    const int i = i0 + ti;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + tj + 8 * q;
        if (i < d && j < d) atomicAdd(gram + static_cast<size_t>(i) * d + j, acc[q]);
    }
}

__global__ void __launch_bounds__(256) sumsq_f64_kernel(const float *__restrict__ Y, int64_t count,
                                                        double *__restrict__ sumsq) {
    double acc = 0.0;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double v = Y[e];
        acc = fma(v, v, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sumsq, acc);
}

}  // namespace

}  // namespace cg

extern "C" cg_status cg_moments_f64(const float *Y, int64_t rows, int32_t d, double *gram, double *sumsq,
                                    void *stream) {
    cg::NvtxRange nvtx_range("cg_moments_f64");
    using namespace cg;
    if (rows < 0 || d < 1 || d > 65536 || (rows > 0 && Y == nullptr)) return CG_ERR_INVALID_ARG;
    if (gram == nullptr && sumsq == nullptr) return CG_ERR_INVALID_ARG;
    if (rows == 0) return CG_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (gram != nullptr) {
        const int gt = (d + kTile - 1) / kTile;
        const int sms = num_sms() > 0 ? num_sms() : 148;
        int64_t splits = (2 * static_cast<int64_t>(sms) + gt * gt - 1) / (gt * gt);
        const int64_t max_splits = (rows + kRowsPerStep - 1) / kRowsPerStep;
        splits = splits < 1 ? 1 : (splits > max_splits ? max_splits : splits);
        splits = splits > 65535 ? 65535 : splits;
        const int64_t per = ((rows + splits - 1) / splits + kRowsPerStep - 1) / kRowsPerStep * kRowsPerStep;
        const int64_t used = (rows + per - 1) / per;
        gram_f64_kernel<<<dim3(gt, gt, static_cast<unsigned>(used)), 256, 0, st>>>(Y, rows, d, per, gram);
        if (cudaGetLastError() != cudaSuccess) return CG_ERR_CUDA;
    }
    if (sumsq != nullptr) {
        const int64_t count = rows * d;
        const int64_t blocks = (count + 255) / 256;
        sumsq_f64_kernel<<<static_cast<unsigned>(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(Y, count, sumsq);
        if (cudaGetLastError() != cudaSuccess) return CG_ERR_CUDA;
    }
    return CG_OK;
}

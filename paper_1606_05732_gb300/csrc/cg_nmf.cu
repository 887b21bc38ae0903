// cg_nmf.cu -- Algorithm 1 ("CountGauss NMF") step 3 on a given Z: for every row r, the
// column index of its maximum and of its minimum (the anchor candidates I_max, I_min),
// ties to the lowest column index.  Steps 1-3 in one go (cg_nmf_anchors_csr, in
// cg_api.cu) take the argmax / argmin inside the split-K sum instead.
#include "cg_internal.cuh"

namespace cg {

namespace {

// One warp per row: lanes scan columns lane, lane + 32, ...; then a shuffle reduction
// that keeps the larger (smaller) value, or the lower index on equal values.
__global__ void __launch_bounds__(256)
row_argmax_argmin_kernel(const float *__restrict__ Z, int m, int d, int32_t *__restrict__ imax,
                         int32_t *__restrict__ imin) {
    pdl_wait();  // Z comes from the split-K sum launched before
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= m) return;
    const float *z = Z + static_cast<size_t>(row) * d;
    float vmax = -INFINITY, vmin = INFINITY;
    int jmax = d, jmin = d;
    for (int j = lane; j < d; j += 32) {
        const float v = z[j];
        if (v > vmax) {  // strict: the first (lowest) index of this lane wins ties
            vmax = v;
            jmax = j;
        }
        if (v < vmin) {
            vmin = v;
            jmin = j;
        }
    }
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
        imax[row] = jmax < d ? jmax : 0;
        imin[row] = jmin < d ? jmin : 0;
    }
}

}  // namespace

}  // namespace cg

extern "C" cg_status cg_row_argmax_argmin(const float *Z, int32_t m, int32_t d, int32_t *imax, int32_t *imin,
                                          void *stream) {
    cg::NvtxRange nvtx_range("cg_row_argmax_argmin");
    using namespace cg;
    if (m < 0 || d < 1 || (m > 0 && (Z == nullptr || imax == nullptr || imin == nullptr))) return CG_ERR_INVALID_ARG;
    if (m == 0) return CG_OK;
    const cudaError_t e = launch_after_previous(row_argmax_argmin_kernel, dim3((m + 7) / 8), dim3(256), 0,
                                                reinterpret_cast<cudaStream_t>(stream), Z, m, d, imax, imin);
    if (e != cudaSuccess) return CG_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

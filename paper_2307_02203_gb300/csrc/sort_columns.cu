// Every vertex column of a field sorted ascending, kept with the field.  The
// KSG marginal count n_y needs the query column in sorted order; the column is
// the same for every reference, so it is sorted once per field instead of once
// per (reference, vertex) pair.  VT columns per CTA, bitonic network in shared
// memory (columns padded with FLT_MAX to a power of two), member-major loads and
// stores coalesced across the VT vertices of each member row.
#include <float.h>

#include "ndf_internal.h"

namespace ndf {

__global__ void __launch_bounds__(256)
    sort_columns_kernel(const float* __restrict__ field, int M, int n2, int64_t N, int VT,
                        float* __restrict__ sorted) {
    extern __shared__ float col[];  // [VT][n2]
    const int64_t v0 = (int64_t)blockIdx.x * VT;
    const int vc = N - v0 < VT ? (int)(N - v0) : VT;
    for (int idx = threadIdx.x; idx < n2 * VT; idx += blockDim.x) {
        const int m = idx / VT, p = idx - m * VT;
        col[p * n2 + m] = (m < M && p < vc) ? field[(int64_t)m * N + v0 + p] : FLT_MAX;
    }
    __syncthreads();
    const int half = n2 >> 1;
    for (int kk = 2; kk <= n2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < half * VT; t += blockDim.x) {
                const int p = t / half, q = t - p * half;
                const int i = (q / j) * 2 * j + (q % j);  // lower index, bit j clear
                const int l = i + j;
                float* c = col + p * n2;
                const float u = c[i], w = c[l];
                if ((u > w) == ((i & kk) == 0)) {
                    c[i] = w;
                    c[l] = u;
                }
            }
            __syncthreads();
        }
    }
    for (int idx = threadIdx.x; idx < M * VT; idx += blockDim.x) {
        const int m = idx / VT, p = idx - m * VT;
        if (p < vc) sorted[(int64_t)m * N + v0 + p] = col[p * n2 + m];
    }
}

cudaError_t ensure_sorted_columns(ndf_ctx* ctx, Field& f) {
    if (f.sorted) return cudaSuccess;
    const int M = (int)f.M;
    int n2 = 1;
    while (n2 < M) n2 <<= 1;
    int VT = 16384 / n2;
    if (VT > 16) VT = 16;
    if (VT < 1) VT = 1;
    const size_t smem = sizeof(float) * (size_t)n2 * VT;
    cudaError_t e = cudaMalloc(&f.sorted, sizeof(float) * (size_t)f.M * (size_t)f.N);
    if (e != cudaSuccess) {
        f.sorted = nullptr;
        return e;
    }
    e = cudaFuncSetAttribute(sort_columns_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (f.N + VT - 1) / VT;
    sort_columns_kernel<<<(unsigned)blocks, 256, smem, ctx->stream>>>(f.data, M, n2, f.N, VT,
                                                                     f.sorted);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace ndf

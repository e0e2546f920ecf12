// Every vertex column of a field sorted ascending, kept with the field.  The
// KSG marginal count n_y needs the query column in sorted order; the column is
// the same for every reference, so it is sorted once per field (during the
// upload, vertex range by vertex range) instead of once per (reference, vertex)
// pair.
//
// Columns of up to 1024 members: one warp per column, the column in registers
// (R = 32..1024 / 32 values per lane, padded with FLT_MAX), lane-major element
// order e = lane * R + r, sorted by the bitonic network in its "mirror" form
// (each merge of size kk first compares e with e ^ (kk - 1), then half-cleaners
// e ^ j, the lower index always keeping the minimum, so no direction flags):
// distances below R are register pairs, larger ones a shuffle with lane ^ (d/R).
// Larger columns: a CTA per group of columns, the same network in shared memory.
#include <float.h>

#include "ndf_internal.h"

namespace ndf {

template <int R>
__global__ void __launch_bounds__(256) sort_columns_reg_kernel(const float* __restrict__ field,
                                                                int M, int64_t N, int64_t v_begin,
                                                                int64_t v_end,
                                                                float* __restrict__ sorted) {
    const int lane = threadIdx.x & 31;
    const int64_t v = v_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (v >= v_end) return;  // whole warps leave together
    float a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int m = r * 32 + lane;  // any member may go to any slot before sorting
        a[r] = m < M ? __ldcs(field + (int64_t)m * N + v) : FLT_MAX;
    }
    auto cmpx = [&](float& lo, float& hi) {
        const float x = fminf(lo, hi), y = fmaxf(lo, hi);
        lo = x;
        hi = y;
    };
#pragma unroll
    for (int kk = 2; kk <= 32 * R; kk <<= 1) {
        // mirror stage: e and e ^ (kk - 1)
        if (kk <= R) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if ((r & (kk >> 1)) == 0) cmpx(a[r], a[r ^ (kk - 1)]);
        } else {
            const int lm = (kk - 1) / R;              // lane bits flipped
            const bool lower = (lane & ((kk >> 1) / R)) == 0;
            float p[R];
#pragma unroll
            for (int r = 0; r < R; ++r) p[r] = __shfl_xor_sync(0xffffffffu, a[R - 1 - r], lm);
#pragma unroll
            for (int r = 0; r < R; ++r) a[r] = lower ? fminf(a[r], p[r]) : fmaxf(a[r], p[r]);
        }
        // half-cleaners: e and e ^ j
#pragma unroll
        for (int j = kk >> 2; j > 0; j >>= 1) {
            if (j < R) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if ((r & j) == 0) cmpx(a[r], a[r ^ j]);
            } else {
                const int lm = j / R;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float q = __shfl_xor_sync(0xffffffffu, a[r], lm);
                    a[r] = lower ? fminf(a[r], q) : fmaxf(a[r], q);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = lane * R + r;
        if (e < M) __stcs(sorted + (int64_t)e * N + v, a[r]);
    }
}

__global__ void __launch_bounds__(256)
    sort_columns_smem_kernel(const float* __restrict__ field, int M, int n2, int64_t N,
                             int64_t v_begin, int64_t v_end, int VT, float* __restrict__ sorted) {
    extern __shared__ float col[];  // [VT][n2]
    const int64_t v0 = v_begin + (int64_t)blockIdx.x * VT;
    const int vc = v_end - v0 < VT ? (int)(v_end - v0) : VT;
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
                const int l = (j == (kk >> 1)) ? (i ^ (kk - 1)) : i + j;  // mirror first
                float* c = col + p * n2;
                const float u = c[i], w = c[l];
                if (u > w) {
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

cudaError_t launch_sort_columns(ndf_ctx* ctx, const Field& f, int64_t v_begin, int64_t v_end,
                                cudaStream_t stream) {
    const int M = (int)f.M;
    const int64_t nv = v_end - v_begin;
    if (nv <= 0) return cudaSuccess;
    if (M <= 1024) {
        const unsigned blocks = (unsigned)((nv + 7) / 8);
        if (M <= 32) sort_columns_reg_kernel<1><<<blocks, 256, 0, stream>>>(f.data, M, f.N, v_begin, v_end, f.sorted);
        else if (M <= 64) sort_columns_reg_kernel<2><<<blocks, 256, 0, stream>>>(f.data, M, f.N, v_begin, v_end, f.sorted);
        else if (M <= 128) sort_columns_reg_kernel<4><<<blocks, 256, 0, stream>>>(f.data, M, f.N, v_begin, v_end, f.sorted);
        else if (M <= 256) sort_columns_reg_kernel<8><<<blocks, 256, 0, stream>>>(f.data, M, f.N, v_begin, v_end, f.sorted);
        else if (M <= 512) sort_columns_reg_kernel<16><<<blocks, 256, 0, stream>>>(f.data, M, f.N, v_begin, v_end, f.sorted);
        else sort_columns_reg_kernel<32><<<blocks, 256, 0, stream>>>(f.data, M, f.N, v_begin, v_end, f.sorted);
    } else {
        int n2 = 1;
        while (n2 < M) n2 <<= 1;
        int VT = 16384 / n2;
        if (VT < 1) VT = 1;
        const size_t smem = sizeof(float) * (size_t)n2 * VT;
        cudaError_t e = cudaFuncSetAttribute(sort_columns_smem_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int64_t blocks = (nv + VT - 1) / VT;
        sort_columns_smem_kernel<<<(unsigned)blocks, 256, smem, stream>>>(f.data, M, n2, f.N, v_begin,
                                                                         v_end, VT, f.sorted);
    }
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t ensure_sorted_columns(ndf_ctx* ctx, Field& f) {
    if (f.sorted) return cudaSuccess;
    cudaError_t e = cudaMalloc(&f.sorted, sizeof(float) * (size_t)f.M * (size_t)f.N);
    if (e != cudaSuccess) {
        f.sorted = nullptr;
        return e;
    }
    return launch_sort_columns(ctx, f, 0, f.N, ctx->stream);
}

}  // namespace ndf

// Every vertex column of a field sorted ascending, kept with the field.  The
// KSG marginal count n_y needs the query column in sorted order; the column is
// the same for every reference, so it is sorted once per field (during the
// upload, vertex range by vertex range) instead of once per (reference, vertex)
// pair.
//
// Columns of up to 1024 members: a CTA per tile of kSortTile consecutive
// vertices.  The tile's rows (kSortTile floats of one member, contiguous in the
// field) are read and written whole, 16 bytes per thread where the tile is aligned,
// through shared memory; there each column is stored with one skip every 32
// elements and a column stride of 2 mod 32, so that the warps' column accesses and
// the row accesses (eight rows of four 16-byte quads per warp instruction: banks
// 2p + m) are free of bank conflicts.  A warp
// sorts one column at a time in registers (R = 1024 / 32 values per lane at most,
// padded with +inf), lane-major element order e = lane * R + r, by the bitonic
// network in its "mirror" form (each merge of size kk first compares e with
// e ^ (kk - 1), then half-cleaners e ^ j, the lower index always keeping the
// minimum, so no direction flags): distances below R are register pairs, larger
// ones a shuffle with lane ^ (d/R).
// Larger columns: a CTA per group of columns, the same network in shared memory.
#include <float.h>

#include "ndf_internal.h"

namespace ndf {

constexpr int kSortTile = 16;     // vertices per CTA
constexpr int kSortThreads = 256;

// shared-memory floats of one column: 32 R elements with a skip after every 32,
// rounded up to 2 mod 32
__host__ __device__ constexpr int sort_col_stride(int R) { return 33 * R + ((34 - (33 * R) % 32) % 32); }
__device__ __forceinline__ int sort_col_slot(int e) { return e + (e >> 5); }

// the network on a warp's column in registers (element e = lane * R + r)
template <int R>
__device__ __forceinline__ void sort_warp_column(float (&a)[R]) {
    const int lane = threadIdx.x & 31;
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
}

template <int R>
__global__ void __launch_bounds__(kSortThreads, 3) sort_columns_tile_kernel(const float* __restrict__ field,
                                                                         int M, int64_t N,
                                                                         int64_t v_begin, int64_t v_end,
                                                                         float* __restrict__ sorted) {
    constexpr int S = sort_col_stride(R);
    extern __shared__ float tile[];  // [kSortTile][S]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t v0 = v_begin + (int64_t)blockIdx.x * kSortTile;
    const int vc = v_end - v0 < kSortTile ? (int)(v_end - v0) : kSortTile;
    // rows in: with a whole, 16-byte aligned tile thread t takes member t / 4 and the
    // quad of vertices 4 (t % 4) ..; otherwise member t / kSortTile, vertex t % kSortTile
    const bool quads = vc == kSortTile && (N & 3) == 0 && (v0 & 3) == 0;
    if (quads) {
#pragma unroll 4
        for (int idx = threadIdx.x; idx < M * 4; idx += kSortThreads) {
            const int m = idx >> 2, p = (idx & 3) * 4;
            const float4 q = __ldcs(reinterpret_cast<const float4*>(field + (int64_t)m * N + v0 + p));
            const int sl = sort_col_slot(m);
            tile[p * S + sl] = q.x;
            tile[(p + 1) * S + sl] = q.y;
            tile[(p + 2) * S + sl] = q.z;
            tile[(p + 3) * S + sl] = q.w;
        }
    } else {
#pragma unroll 8
        for (int idx = threadIdx.x; idx < M * kSortTile; idx += kSortThreads) {
            const int m = idx / kSortTile, p = idx - m * kSortTile;
            if (p < vc) tile[p * S + sort_col_slot(m)] = __ldcs(field + (int64_t)m * N + v0 + p);
        }
    }
    __syncthreads();
    for (int p = warp; p < vc; p += kSortThreads / 32) {
        float* col = tile + p * S;
        float a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = r * 32 + lane;  // any member may go to any slot before sorting
            a[r] = e < M ? col[sort_col_slot(e)] : INFINITY;
        }
        sort_warp_column<R>(a);
        __syncwarp();  // every lane has read the column before it is overwritten
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = lane * R + r;
            if (e < M) col[sort_col_slot(e)] = a[r];
        }
    }
    __syncthreads();
    if (quads) {
#pragma unroll 4
        for (int idx = threadIdx.x; idx < M * 4; idx += kSortThreads) {
            const int m = idx >> 2, p = (idx & 3) * 4;
            const int sl = sort_col_slot(m);
            __stcs(reinterpret_cast<float4*>(sorted + (int64_t)m * N + v0 + p),
                   make_float4(tile[p * S + sl], tile[(p + 1) * S + sl], tile[(p + 2) * S + sl],
                               tile[(p + 3) * S + sl]));
        }
    } else {
#pragma unroll 8
        for (int idx = threadIdx.x; idx < M * kSortTile; idx += kSortThreads) {
            const int m = idx / kSortTile, p = idx - m * kSortTile;
            if (p < vc) __stcs(sorted + (int64_t)m * N + v0 + p, tile[p * S + sort_col_slot(m)]);
        }
    }
}

template <int R>
static cudaError_t launch_sort_tile(const Field& f, int64_t v_begin, int64_t v_end, cudaStream_t stream) {
    const size_t smem = sizeof(float) * (size_t)kSortTile * sort_col_stride(R);
    const cudaError_t attr = cudaFuncSetAttribute(
        sort_columns_tile_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    const int64_t blocks = (v_end - v_begin + kSortTile - 1) / kSortTile;
    sort_columns_tile_kernel<R><<<(unsigned)blocks, kSortThreads, smem, stream>>>(f.data, (int)f.M, f.N, v_begin,
                                                                                 v_end, f.sorted);
    return cudaGetLastError();
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
        cudaError_t e;
        if (M <= 32) e = launch_sort_tile<1>(f, v_begin, v_end, stream);
        else if (M <= 64) e = launch_sort_tile<2>(f, v_begin, v_end, stream);
        else if (M <= 128) e = launch_sort_tile<4>(f, v_begin, v_end, stream);
        else if (M <= 256) e = launch_sort_tile<8>(f, v_begin, v_end, stream);
        else if (M <= 512) e = launch_sort_tile<16>(f, v_begin, v_end, stream);
        else e = launch_sort_tile<32>(f, v_begin, v_end, stream);
        if (e != cudaSuccess) return e;
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
    const size_t bytes = sizeof(float) * (size_t)f.M * (size_t)f.N;
    cudaError_t e = cudaMalloc(&f.sorted, bytes);
    if (e != cudaSuccess) {
        f.sorted = nullptr;
        return e;
    }
    e = launch_sort_columns(ctx, f, 0, f.N, ctx->stream);
    if (e != cudaSuccess) {  // not sorted: a later call must not take it for sorted
        ctx_release(ctx, f.sorted, bytes);
        f.sorted = nullptr;
    }
    return e;
}

}  // namespace ndf

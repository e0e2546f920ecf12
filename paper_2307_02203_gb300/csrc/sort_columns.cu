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
// ones a shuffle with lane ^ (d/R).  The merges up to size R, which stay inside a
// lane, are replaced by Batcher's odd-even merge sort of the lane's registers.
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

static __device__ __forceinline__ void cmpx(float& lo, float& hi) {
    const float x = fminf(lo, hi), y = fmaxf(lo, hi);
    lo = x;
    hi = y;
}

// Ascending sort of one lane's R registers by Batcher's odd-even merge sort: merges of
// sorted runs p = 1, 2, .. R/2 long, each as compare-exchanges at distances k = p, p/2,
// .. 1 between elements x and x + k of the same 2p-run.  Every min/max issues on the ALU
// pipe whether its operands share a lane or not, so the comparator count is what the
// sort costs: 191 for R = 32 against the bitonic network's 240.
template <int R>
__device__ __forceinline__ void sort_lane_registers(float (&a)[R]) {
#pragma unroll
    for (int p = 1; p < R; p <<= 1) {
#pragma unroll
        for (int k = p; k >= 1; k >>= 1) {
            // x runs over [k % p + 2kt, k % p + 2kt + k) for t = 0, 1, ..
#pragma unroll
            for (int x = 0; x + k < R; ++x) {
                const int off = x - k % p;
                if (off >= 0 && off % (2 * k) < k && x / (2 * p) == (x + k) / (2 * p)) cmpx(a[x], a[x + k]);
            }
        }
    }
}

// the network on a warp's column in registers (element e = lane * R + r): each lane's
// R registers sorted first, then the bitonic merges of runs R, 2R, .. 16R long
template <int R>
__device__ __forceinline__ void sort_warp_column(float (&a)[R]) {
    const int lane = threadIdx.x & 31;
    sort_lane_registers<R>(a);
#pragma unroll
    for (int kk = 2 * R; kk <= 32 * R; kk <<= 1) {
        // mirror stage: e and e ^ (kk - 1), across lanes since kk > R
        {
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

// Knuth's two-sum: s + e == a + b exactly, s = fl(a + b) (round to nearest, no
// overflow), for any magnitudes of a and b.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// The warp's sum of x as an unevaluated pair hi + lo (double-float), by an xor
// butterfly whose levels add the two pairs with two-sum and renormalise: about 48
// significant bits, from FP32 arithmetic only (FP64 issues at a small fraction of
// the FP32 rate on this part).  Every lane ends with the same pair.
__device__ __forceinline__ void warp_sum_df(float x, float& hi, float& lo) {
    hi = x;
    lo = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, h2, s, e);
        two_sum(s, e + (lo + l2), hi, lo);
    }
}

template <int R>
__global__ void __launch_bounds__(kSortThreads, 3) sort_columns_tile_kernel(const float* __restrict__ field,
                                                                         int M, int64_t N,
                                                                         int64_t v_begin, int64_t v_end,
                                                                         float* __restrict__ sorted,
                                                                         float* __restrict__ copy,
                                                                         ColumnStats st) {
    constexpr int S = sort_col_stride(R);
    extern __shared__ float tile[];  // [kSortTile][S]
    __shared__ float stat_sum[kSortTile][4], stat_centre[kSortTile];
    __shared__ bool stat_bad[kSortTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t v0 = v_begin + (int64_t)blockIdx.x * kSortTile;
    const int vc = v_end - v0 < kSortTile ? (int)(v_end - v0) : kSortTile;
    // rows in: with a whole, 16-byte aligned tile thread t takes member t / 4 and the
    // quad of vertices 4 (t % 4) ..; otherwise member t / kSortTile, vertex t % kSortTile.
    // With copy (16-byte aligned, allocated by the library) each row is also written
    // there as read.
    const bool quads = vc == kSortTile && (N & 3) == 0 && (v0 & 3) == 0 &&
                       (reinterpret_cast<uintptr_t>(field) & 15) == 0;
    if (quads) {
#pragma unroll 4
        for (int idx = threadIdx.x; idx < M * 4; idx += kSortThreads) {
            const int m = idx >> 2, p = (idx & 3) * 4;
            const float4 q = __ldcs(reinterpret_cast<const float4*>(field + (int64_t)m * N + v0 + p));
            if (copy) __stcs(reinterpret_cast<float4*>(copy + (int64_t)m * N + v0 + p), q);
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
            if (p < vc) {
                const float x = __ldcs(field + (int64_t)m * N + v0 + p);
                if (copy) __stcs(copy + (int64_t)m * N + v0 + p, x);
                tile[p * S + sort_col_slot(m)] = x;
            }
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
        // fmaf(y, 0, t) turns NaN at a NaN or an infinite member and keeps it (before
        // the sort, whose min/max would drop a NaN)
        bool bad = false;
        if (st.mean) {
            float t = 0.0f;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r * 32 + lane < M) t = fmaf(a[r], 0.0f, t);
            bad = __any_sync(0xffffffffu, t != 0.0f);
        }
        sort_warp_column<R>(a);
        __syncwarp();  // every lane has read the column before it is overwritten
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = lane * R + r;
            if (e < M) col[sort_col_slot(e)] = a[r];
        }
        if (st.mean) {
            // The statistics of Eq. 1 in one pass over the sorted registers, centred on
            // the median member c: c1 = sum (y - c), c2 = sum (y - c)^2, each lane over
            // its R consecutive members in FP32 (on the FMA pipe, idle in the sort),
            // the lanes' sums added as double-float; the FP64 rest per column below.
            __syncwarp();
            const float c = col[sort_col_slot(M >> 1)];
            float c1 = 0.0f, c2 = 0.0f;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (lane * R + r < M) {
                    const float d = a[r] - c;
                    c1 += d;
                    c2 = fmaf(d, d, c2);
                }
            float h1, l1, h2, l2;
            warp_sum_df(c1, h1, l1);
            warp_sum_df(c2, h2, l2);
            if (lane == 0) {
                stat_sum[p][0] = h1;
                stat_sum[p][1] = l1;
                stat_sum[p][2] = h2;
                stat_sum[p][3] = l2;
                stat_centre[p] = c;
                stat_bad[p] = bad;
            }
        }
    }
    __syncthreads();
    if (st.mean && (int)threadIdx.x < vc) {  // the FP64 rest, one thread per column
        const int p = threadIdx.x;
        const float* col = tile + p * S;
        const float lo = col[sort_col_slot(0)], hi = col[sort_col_slot(M - 1)];
        double mean = 0.0, inv = 0.0;
        if (stat_bad[p]) {
            atomicOr(st.nonfinite, 1);  // the load fails; the values are not used
        } else if (lo == hi) {          // constant sample: r is defined as 0
            mean = (double)lo;
        } else {  // mu = c + s1 / M; S = s2 - s1^2 / M removes the offset from the centre
            const double s1 = (double)stat_sum[p][0] + (double)stat_sum[p][1];
            const double s2 = (double)stat_sum[p][2] + (double)stat_sum[p][3];
            mean = (double)stat_centre[p] + s1 / (double)M;
            const double S2 = s2 - s1 * s1 / (double)M;
            inv = S2 > 0.0 ? 1.0 / sqrt(S2) : 0.0;
        }
        st.mean[v0 + p] = mean;
        st.inv_norm[v0 + p] = inv;
    }
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
static cudaError_t launch_sort_tile(const Field& f, int64_t v_begin, int64_t v_end, cudaStream_t stream,
                                    const float* src, ColumnStats st) {
    const size_t smem = sizeof(float) * (size_t)kSortTile * sort_col_stride(R);
    const cudaError_t attr = cudaFuncSetAttribute(
        sort_columns_tile_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    const int64_t blocks = (v_end - v_begin + kSortTile - 1) / kSortTile;
    sort_columns_tile_kernel<R><<<(unsigned)blocks, kSortThreads, smem, stream>>>(
        src ? src : f.data, (int)f.M, f.N, v_begin, v_end, f.sorted, src ? f.data : nullptr, st);
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
                                cudaStream_t stream, const float* src, int* d_nonfinite) {
    const int M = (int)f.M;
    const int64_t nv = v_end - v_begin;
    if (nv <= 0) return cudaSuccess;
    if (M <= kSortTileMaxM) {
        static_assert(kSortTileMaxM == 32 * 32, "the register network holds 32 values per lane");
        ColumnStats st{};
        if (d_nonfinite) st = ColumnStats{f.mean, f.inv_norm, d_nonfinite};
        cudaError_t e;
        if (M <= 32) e = launch_sort_tile<1>(f, v_begin, v_end, stream, src, st);
        else if (M <= 64) e = launch_sort_tile<2>(f, v_begin, v_end, stream, src, st);
        else if (M <= 128) e = launch_sort_tile<4>(f, v_begin, v_end, stream, src, st);
        else if (M <= 256) e = launch_sort_tile<8>(f, v_begin, v_end, stream, src, st);
        else if (M <= 512) e = launch_sort_tile<16>(f, v_begin, v_end, stream, src, st);
        else e = launch_sort_tile<32>(f, v_begin, v_end, stream, src, st);
        if (e != cudaSuccess) return e;
    } else if (src || d_nonfinite) {
        return cudaErrorInvalidValue;  // the shared-memory network only sorts f.data
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

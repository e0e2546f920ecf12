// Single-reference Pearson volume (Sec. 3.1, Eq. 1):
//   r_v = sum_m xt_m (y_{m,v} - mu_v) * s_ref * s_v,   xt_m = x_m - mu_ref,
// s = 1/sqrt(sum of squared deviations) from the per-vertex statistics.
//
// Stage (one small kernel): gather and centre the reference column once, in FP64,
// into a padded FP32 buffer.  Volume kernel: every CTA bulk-copies that column
// into shared memory (cp.async.bulk + mbarrier, in chunks of 2048 members) and
// streams the member-major field once with coalesced 128-bit loads, 4 vertices
// per thread, the members split between the two halves of the CTA.  The kernel
// is HBM-bound: M*N*4 bytes read, N*4 written.
#include "device_common.cuh"
#include "ndf_internal.h"

namespace ndf {

constexpr int kPearsonChunk = 2048;  // members staged in shared memory at a time
constexpr int kPearsonThreads = 256; // two member halves x 128 vertex groups

__global__ void pearson_stage_kernel(const float* __restrict__ field, int64_t M, int64_t N,
                                     int64_t ref, const double* __restrict__ mean,
                                     float* __restrict__ xt, int64_t Mpad) {
    double mu = mean[ref];
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < Mpad;
         m += (int64_t)gridDim.x * blockDim.x)
        xt[m] = m < M ? (float)((double)field[m * N + ref] - mu) : 0.0f;
}

template <int VEC>
struct VecLoad;
template <>
struct VecLoad<4> {
    using T = float4;
    static __device__ __forceinline__ T ld(const float* p) {
        return __ldcs(reinterpret_cast<const float4*>(p));
    }
    static __device__ __forceinline__ float get(const T& v, int i) {
        return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
    }
};
template <>
struct VecLoad<1> {
    using T = float;
    static __device__ __forceinline__ T ld(const float* p) { return __ldcs(p); }
    static __device__ __forceinline__ float get(const T& v, int) { return v; }
};

template <int VEC>
__global__ void __launch_bounds__(kPearsonThreads)
    pearson_volume_kernel(const float* __restrict__ field, int64_t M, int64_t N,
                          const float* __restrict__ xt, const double* __restrict__ mean,
                          const double* __restrict__ inv_norm,
                          const double* __restrict__ s_ref_ptr, float* __restrict__ out,
                          unsigned* __restrict__ status) {
    using L = VecLoad<VEC>;
    __shared__ __align__(16) float xs[kPearsonChunk];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float red[VEC * 128];
    __shared__ int s_ok;

    const int g = threadIdx.x & 127;
    const int half = threadIdx.x >> 7;
    const int64_t v0 = ((int64_t)blockIdx.x * 128 + g) * VEC;
    const bool active = v0 < N;

    float mu[VEC], acc[VEC];
#pragma unroll
    for (int i = 0; i < VEC; ++i) {
        mu[i] = active ? (float)mean[v0 + i] : 0.0f;
        acc[i] = 0.0f;
    }
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();

    uint32_t phase = 0;
    for (int64_t c0 = 0; c0 < M; c0 += kPearsonChunk) {
        const int cn = (int)(M - c0 < kPearsonChunk ? M - c0 : kPearsonChunk);
        if (threadIdx.x == 0) {
            uint32_t bytes = (uint32_t)(((cn + 3) & ~3) * 4);
            mbar_expect_tx(&bar, bytes);
            bulk_g2s(xs, xt + c0, bytes, &bar);
            s_ok = mbar_wait(&bar, phase) ? 1 : 0;
            if (!s_ok) report(status, kDevTimeout);
        }
        __syncthreads();
        if (!s_ok) return;
        phase ^= 1u;
        if (active) {
            const float* p = field + (c0 + half) * N + v0;
            const int64_t step = 2 * N;
            int j = half;
            for (; j + 14 < cn; j += 16) {
                typename L::T y[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) y[u] = L::ld(p + u * step);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float xm = xs[j + 2 * u];
#pragma unroll
                    for (int i = 0; i < VEC; ++i) acc[i] = fmaf(xm, L::get(y[u], i) - mu[i], acc[i]);
                }
                p += 8 * step;
            }
            for (; j < cn; j += 2) {
                typename L::T y = L::ld(p);
                float xm = xs[j];
#pragma unroll
                for (int i = 0; i < VEC; ++i) acc[i] = fmaf(xm, L::get(y, i) - mu[i], acc[i]);
                p += step;
            }
        }
        __syncthreads();  // xs is overwritten by the next chunk
    }
    if (half == 1) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) red[i * 128 + g] = acc[i];
    }
    __syncthreads();
    if (half == 0 && active) {
        const double s_ref = *s_ref_ptr;
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            double a = (double)acc[i] + (double)red[i * 128 + g];
            double r = a * s_ref * inv_norm[v0 + i];
            r = r > 1.0 ? 1.0 : (r < -1.0 ? -1.0 : r);
            out[v0 + i] = (float)r;
        }
    }
}

cudaError_t launch_pearson(ndf_ctx* ctx, const Field& rf, const Field& qf, int64_t ref_idx,
                           float* out) {
    // the reference column comes from rf (N_ref vertices), the volume from qf (N vertices)
    const int64_t M = rf.M, N = qf.N, N_ref = rf.N;
    const int64_t Mpad = (M + 3) & ~int64_t(3);
    cudaError_t e = ctx->stage_x.reserve(sizeof(float) * (size_t)Mpad);
    if (e != cudaSuccess) return e;
    float* xt = ctx->stage_x.as<float>();
    unsigned* status = ctx->flag.as<unsigned>() + 1;
    int sb = (int)((Mpad + 255) / 256);
    pearson_stage_kernel<<<sb < 64 ? sb : 64, 256, 0, ctx->stream>>>(rf.data, M, N_ref, ref_idx,
                                                                      rf.mean, xt, Mpad);
    ctx->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (N % 4 == 0) {
        int64_t blocks = (N / 4 + 127) / 128;
        pearson_volume_kernel<4><<<(unsigned)blocks, kPearsonThreads, 0, ctx->stream>>>(
            qf.data, M, N, xt, qf.mean, qf.inv_norm, rf.inv_norm + ref_idx, out, status);
    } else {
        int64_t blocks = (N + 127) / 128;
        pearson_volume_kernel<1><<<(unsigned)blocks, kPearsonThreads, 0, ctx->stream>>>(
            qf.data, M, N, xt, qf.mean, qf.inv_norm, rf.inv_norm + ref_idx, out, status);
    }
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace ndf

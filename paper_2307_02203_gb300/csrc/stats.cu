// Per-vertex statistics of a loaded ensemble (the standardisation that Eq. 1 needs):
// FP64 mean mu_v and 1/sqrt(S_v), S_v = sum_m (e_m(v) - mu_v)^2.  Two passes over
// the member-major field; within a block of 32 members the sums run in FP32,
// across blocks in FP64.  Constant columns are detected exactly (min == max) so
// that their S_v is exactly 0.  HBM-bound: 2 * M * N * 4 bytes read.  Loads of up to
// 1024 members take the same statistics from the column-sort kernel instead, which
// holds each column in registers anyway.
#include "ndf_internal.h"

namespace ndf {

__global__ void __launch_bounds__(256) field_stats_kernel(const float* __restrict__ f, int64_t M,
                                                          int64_t N, int64_t v_begin, int64_t v_end,
                                                          double* __restrict__ mean,
                                                          double* __restrict__ inv_norm,
                                                          int* __restrict__ nonfinite) {
    int64_t v = v_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= v_end) return;
    const float* p = f + v;
    double s = 0.0;
    float lo = p[0], hi = p[0];
    bool bad = false;
    int64_t m = 0;
    for (; m < M; m += 32) {
        int64_t e = m + 32 < M ? m + 32 : M;
        float b = 0.0f;
#pragma unroll 8
        for (int64_t j = m; j < e; ++j) {
            float y = __ldg(p + j * N);
            bad |= !isfinite(y);
            lo = fminf(lo, y);
            hi = fmaxf(hi, y);
            b += y;
        }
        s += (double)b;
    }
    double mu = s / (double)M;
    if (bad) {
        atomicOr(nonfinite, 1);
        mean[v] = 0.0;
        inv_norm[v] = 0.0;
        return;
    }
    if (lo == hi) {  // constant sample: r is defined as 0
        mean[v] = (double)lo;
        inv_norm[v] = 0.0;
        return;
    }
    float muf = (float)mu;
    double s1 = 0.0, s2 = 0.0;
    for (m = 0; m < M; m += 32) {
        int64_t e = m + 32 < M ? m + 32 : M;
        float b1 = 0.0f, b2 = 0.0f;
#pragma unroll 8
        for (int64_t j = m; j < e; ++j) {
            float d = __ldg(p + j * N) - muf;
            b1 += d;
            b2 = fmaf(d, d, b2);
        }
        s1 += (double)b1;
        s2 += (double)b2;
    }
    // centred about the FP32-rounded mean; remove the offset exactly in FP64
    double S = s2 - s1 * s1 / (double)M;
    mean[v] = mu;
    inv_norm[v] = S > 0.0 ? 1.0 / sqrt(S) : 0.0;
}

cudaError_t launch_field_stats(ndf_ctx* ctx, const Field& f, int64_t v_begin, int64_t v_end,
                               int* d_nonfinite, cudaStream_t stream) {
    if (v_end <= v_begin) return cudaSuccess;
    int64_t blocks = (v_end - v_begin + 255) / 256;
    field_stats_kernel<<<(unsigned)blocks, 256, 0, stream ? stream : ctx->stream>>>(f.data, f.M, f.N, v_begin, v_end,
                                                                  f.mean, f.inv_norm, d_nonfinite);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace ndf

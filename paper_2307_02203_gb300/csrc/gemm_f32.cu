// FP32 matrix products of the hash-grid network's dense layers (Sec. 4.1-4.3,
// row f2): forward, data gradient and weight gradient of every layer, in FP32
// with FP32 accumulation (the parity path of the network; the FP64 oracle checks
// it), and deterministic: the weight gradients reduce fixed chunks of the batch in
// a fixed order.
//
// One kernel, C[M][N] = sum_k A(m, k) B(k, n), with A and B read row-major either
// way round (TA: A stored [K][M]; TB: B stored [N][K]).  A CTA of 256 threads
// computes a 64 x 64 tile in 16-deep slices staged through shared memory (each
// slice read into registers while the previous one is multiplied); thread
// (ty, tx) owns rows ty + 16 i and columns tx + 16 j (i, j < 4), so a warp's
// shared-memory reads are broadcasts (A) or 16 consecutive words (B).  With a
// split over K (blockIdx.z) each slice of K writes its own partial tile, and a
// second kernel adds the partials in slice order.
#include "gemm_f32.h"

namespace ndf {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
    sgemm_kernel(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C,
                 int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t k_chunk,
                 int accumulate) {
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * kBM, n0 = (int64_t)blockIdx.x * kBN;
    const int64_t k_begin = (int64_t)blockIdx.z * k_chunk;
    const int64_t k_end = k_begin + k_chunk < K ? k_begin + k_chunk : K;
    float acc[4][4] = {};
    // slice k0 of A(m0.., k..) and B(k.., n0..): 1024 elements each, 4 per thread, read
    // into registers one slice ahead of the products, so the loads' latency overlaps them
    float va[4], vb[4];
    auto load_slice = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = threadIdx.x + 256 * r;
            int mm, kk;
            if (TA) {  // consecutive threads along m (contiguous in [K][M])
                mm = e & (kBM - 1);
                kk = e >> 6;
            } else {  // consecutive threads along k (contiguous in [M][K])
                kk = e & (kBK - 1);
                mm = e >> 4;
            }
            const int64_t gm = m0 + mm, gk = k0 + kk;
            va[r] = (gm < M && gk < k_end) ? (TA ? A[gk * lda + gm] : A[gm * lda + gk]) : 0.0f;
            int nn;
            if (TB) {  // consecutive threads along k (contiguous in [N][K])
                kk = e & (kBK - 1);
                nn = e >> 4;
            } else {  // consecutive threads along n (contiguous in [K][N])
                nn = e & (kBN - 1);
                kk = e >> 6;
            }
            const int64_t gn = n0 + nn, gk2 = k0 + kk;
            vb[r] = (gn < N && gk2 < k_end) ? (TB ? B[gn * ldb + gk2] : B[gk2 * ldb + gn]) : 0.0f;
        }
    };
    auto store_slice = [&]() {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = threadIdx.x + 256 * r;
            if (TA) As[e >> 6][e & (kBM - 1)] = va[r];
            else As[e & (kBK - 1)][e >> 4] = va[r];
            if (TB) Bs[e & (kBK - 1)][e >> 4] = vb[r];
            else Bs[e >> 6][e & (kBN - 1)] = vb[r];
        }
    };
    if (k_begin < k_end) load_slice(k_begin);
    for (int64_t k0 = k_begin; k0 < k_end; k0 += kBK) {
        store_slice();
        __syncthreads();
        if (k0 + kBK < k_end) load_slice(k0 + kBK);
        // each 16-deep slice is summed on its own and then added to the running sums
        // (blocked summation: rounding grows with 16 + K / 16 terms instead of K)
        float part[4][4] = {};
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) part[i][j] = fmaf(a[i], b[j], part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
        __syncthreads();
    }
    float* Cz = C + (int64_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            float* c = Cz + gm * N + gn;
            *c = accumulate ? *c + acc[i][j] : acc[i][j];
        }
    }
}

// C[i] (+)= sum_s part[s][i] for s = 0 .. S-1 in order
__global__ void reduce_parts_kernel(const float* __restrict__ part, int64_t S, int64_t n,
                                    float* __restrict__ C, int accumulate) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int64_t z = 0; z < S; ++z) s += part[z * n + i];
        C[i] = accumulate ? C[i] + s : s;
    }
}

// part[z][n] = sum of A[k][n] over the k of chunk z: a CTA of 32 columns x kColLanes
// row lanes (a warp reads 32 consecutive columns of one row); lane y sums the rows
// k_begin + y, + kColLanes, ... in order, then the lanes' sums are added in order
constexpr int kColLanes = 8;
__global__ void __launch_bounds__(32 * kColLanes)
    colsum_parts_kernel(const float* __restrict__ A, int64_t K, int64_t N, int64_t k_chunk,
                        float* __restrict__ part) {
    __shared__ float red[kColLanes][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t n = (int64_t)blockIdx.x * 32 + tx;
    const int64_t k_begin = (int64_t)blockIdx.y * k_chunk;
    const int64_t k_end = k_begin + k_chunk < K ? k_begin + k_chunk : K;
    float s = 0.0f;
    if (n < N) {
#pragma unroll 8
        for (int64_t k = k_begin + ty; k < k_end; k += kColLanes) s += A[k * N + n];
    }
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && n < N) {
        float t = 0.0f;
#pragma unroll
        for (int y = 0; y < kColLanes; ++y) t += red[y][tx];
        part[(int64_t)blockIdx.y * N + n] = t;
    }
}

template <bool TA, bool TB>
cudaError_t run(cudaStream_t s, const float* A, const float* B, float* C, int64_t M, int64_t N,
                int64_t K, int64_t lda, int64_t ldb, int64_t splits, int64_t k_chunk, int accumulate) {
    const dim3 grid((unsigned)((N + kBN - 1) / kBN), (unsigned)((M + kBM - 1) / kBM), (unsigned)splits);
    sgemm_kernel<TA, TB><<<grid, 256, 0, s>>>(A, B, C, M, N, K, lda, ldb, k_chunk, accumulate);
    return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_f32_nt(cudaStream_t s, const float* A, const float* B, float* C, int64_t M,
                        int64_t N, int64_t K) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    return run<false, true>(s, A, B, C, M, N, K, K, K, 1, K > 0 ? K : 1, 0);
}

cudaError_t gemm_f32_nn(cudaStream_t s, const float* A, const float* B, float* C, int64_t M,
                        int64_t N, int64_t K) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    return run<false, false>(s, A, B, C, M, N, K, K, N, 1, K > 0 ? K : 1, 0);
}

int64_t gemm_f32_tn_work_floats(int64_t M, int64_t N, int64_t K) {
    const int64_t splits = K < kSplitK * 256 ? (K + 255) / 256 : kSplitK;
    return (splits < 1 ? 1 : splits) * M * N;
}

cudaError_t gemm_f32_tn_acc(cudaStream_t s, const float* A, const float* B, float* C, int64_t M,
                            int64_t N, int64_t K, float* work) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    int64_t splits = K < kSplitK * 256 ? (K + 255) / 256 : kSplitK;
    int64_t k_chunk = (K + splits - 1) / splits;
    k_chunk = (k_chunk + kBK - 1) / kBK * kBK;
    splits = (K + k_chunk - 1) / k_chunk;
    cudaError_t e = run<true, false>(s, A, B, work, M, N, K, M, N, splits, k_chunk, 0);
    if (e != cudaSuccess) return e;
    const int64_t n = M * N;
    reduce_parts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(work, splits, n, C, 1);
    return cudaGetLastError();
}

cudaError_t colsum_f32_acc(cudaStream_t s, const float* A, float* out, int64_t K, int64_t N,
                           float* work) {
    if (N <= 0 || K <= 0) return cudaSuccess;
    int64_t splits = K < kSplitK * 256 ? (K + 255) / 256 : kSplitK;
    const int64_t k_chunk = (K + splits - 1) / splits;
    splits = (K + k_chunk - 1) / k_chunk;
    colsum_parts_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)splits), 32 * kColLanes, 0, s>>>(
        A, K, N, k_chunk, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_parts_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(work, splits, N, out, 1);
    return cudaGetLastError();
}

}  // namespace ndf

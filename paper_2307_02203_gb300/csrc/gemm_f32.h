// FP32 matrix products of the hash-grid network's training (gemm_f32.cu).  All
// matrices are row-major; every call is enqueued on stream s.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ndf {

// largest number of K slices of a split product (the workspace holds that many
// partial results)
constexpr int64_t kSplitK = 64;

// C[M][N] = A[M][K] B[N][K]^T
cudaError_t gemm_f32_nt(cudaStream_t s, const float* A, const float* B, float* C, int64_t M,
                        int64_t N, int64_t K);
// C[M][N] = A[M][K] B[K][N]
cudaError_t gemm_f32_nn(cudaStream_t s, const float* A, const float* B, float* C, int64_t M,
                        int64_t N, int64_t K);
// C[M][N] += A[K][M]^T B[K][N], K split into slices summed in a fixed order;
// work: gemm_f32_tn_work_floats(M, N, K) floats
cudaError_t gemm_f32_tn_acc(cudaStream_t s, const float* A, const float* B, float* C, int64_t M,
                            int64_t N, int64_t K, float* work);
int64_t gemm_f32_tn_work_floats(int64_t M, int64_t N, int64_t K);
// out[N] += sum_k A[k][n] over A[K][N], in fixed slices; work: kSplitK * N floats
cudaError_t colsum_f32_acc(cudaStream_t s, const float* A, float* out, int64_t K, int64_t N,
                           float* work);

}  // namespace ndf

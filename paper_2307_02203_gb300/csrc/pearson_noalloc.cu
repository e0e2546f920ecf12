// ndf_pearson_noalloc: a Pearson-volume entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: a host application whose allocator owns
// the whole device budget (another framework's memory pool, a renderer with a
// fixed arena), or one that cannot accept the device-wide synchronisation that
// cudaMalloc / cudaFree may imply in its frame loop.  This entry point takes
// the ensemble fields and the output volume as caller-owned device buffers and
// keeps its only scratch -- the centred reference column and two scalars -- in
// a fixed file-scope device array.  It also needs no per-vertex statistics:
// the query vertex's mean and spread are formed in the same pass (shifted by
// the vertex's first member value), so nothing has to be loaded beforehand.
//
// The scratch array holds NDF_NOALLOC_MAX_M floats plus two doubles; every GPU
// that loads this library keeps it until the process exits.  All calls share
// it and it keeps the last call's contents, so every call rewrites all of it
// that it reads (including the zero padding) before use; calls that overlap on
// the GPU (different streams, different host threads) race on it.
#include <math.h>

#include <mutex>

#include "ndf_internal.h"

namespace {

constexpr int kMaxM = NDF_NOALLOC_MAX_M;
constexpr int kScalarsOff = kMaxM * 4;  // byte offset of the two doubles

// [0, kMaxM) floats: centred reference column x_m - mean_x (zero padded);
// then double s_ref = 1/sqrt(sum (x - mean_x)^2) and double sum of the FP32
// centred values.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScalarsOff + 64];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (the host-side
// symbol is only a stand-in and must not reach a kernel).  Outside stream
// capture the address is looked up again on every call (a cheap host call), so
// a module reloaded at another address after a device reset is followed; during
// capture the address recorded by the last call outside capture is used.
ndf_status scratch_address(cudaStream_t s, void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return NDF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return NDF_ERR_ARG;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return NDF_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return NDF_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    if (!g_scratch_addr[dev]) return NDF_ERR_STATE;  // first call of this device under capture
    *out = g_scratch_addr[dev];
    return NDF_OK;
}

__device__ double block_sum_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    t = red[32];
    __syncthreads();
    return t;
}

// One CTA of 1024 threads: mean of the reference column (FP64), the centred
// FP32 column with zero padding to a multiple of 4, 1/sqrt(Sxx), sum of the
// centred values.
__global__ void __launch_bounds__(1024)
    noalloc_stage_kernel(const float* __restrict__ field, int M, int64_t N, int64_t ref,
                         unsigned char* __restrict__ scratch) {
    __shared__ double red[33];
    float* xt = reinterpret_cast<float*>(scratch);
    double* scal = reinterpret_cast<double*>(scratch + kScalarsOff);
    double s = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) s += (double)field[(int64_t)m * N + ref];
    const double mu = block_sum_d(s, red) / (double)M;
    double sxx = 0.0, sxt = 0.0;
    const int Mpad = (M + 3) & ~3;
    for (int m = threadIdx.x; m < Mpad; m += blockDim.x) {
        float v = 0.0f;
        if (m < M) {
            double d = (double)field[(int64_t)m * N + ref] - mu;
            sxx += d * d;
            v = (float)d;
        }
        xt[m] = v;
        sxt += (double)v;
    }
    sxx = block_sum_d(sxx, red);
    sxt = block_sum_d(sxt, red);
    if (threadIdx.x == 0) {
        scal[0] = sxx > 0.0 ? 1.0 / sqrt(sxx) : 0.0;
        scal[1] = sxt;
    }
}

// Four vertices per thread (VEC = 4 when N % 4 == 0), one pass over the query
// field: with c = the vertex's first member value,
//   cov  = sum xt (y - c) - (sum (y - c) / M) * sum xt
//   S_yy = sum (y - c)^2 - (sum (y - c))^2 / M
// accumulated in FP32 within blocks of 32 members and in FP64 across blocks.
template <int VEC>
__global__ void __launch_bounds__(256)
    noalloc_volume_kernel(const float* __restrict__ field, int M, int64_t N,
                          const unsigned char* __restrict__ scratch, float* __restrict__ out) {
    const float* xt = reinterpret_cast<const float*>(scratch);
    const double* scal = reinterpret_cast<const double*>(scratch + kScalarsOff);
    const int64_t v0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VEC;
    if (v0 >= N) return;
    float c[VEC];
#pragma unroll
    for (int i = 0; i < VEC; ++i) c[i] = field[v0 + i];
    double sxy[VEC] = {}, sy[VEC] = {}, syy[VEC] = {};
    for (int m0 = 0; m0 < M; m0 += 32) {
        const int m1 = m0 + 32 < M ? m0 + 32 : M;
        float bxy[VEC] = {}, by[VEC] = {}, byy[VEC] = {};
#pragma unroll 4
        for (int m = m0; m < m1; ++m) {
            const float xm = __ldg(xt + m);
            const float* p = field + (int64_t)m * N + v0;
            float y[VEC];
            if (VEC == 4) {
                float4 q = __ldcs(reinterpret_cast<const float4*>(p));
                y[0] = q.x;
                y[VEC > 1 ? 1 : 0] = q.y;
                y[VEC > 2 ? 2 : 0] = q.z;
                y[VEC > 3 ? 3 : 0] = q.w;
            } else {
                y[0] = __ldcs(p);
            }
#pragma unroll
            for (int i = 0; i < VEC; ++i) {
                const float d = y[i] - c[i];
                bxy[i] = fmaf(xm, d, bxy[i]);
                by[i] += d;
                byy[i] = fmaf(d, d, byy[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            sxy[i] += (double)bxy[i];
            sy[i] += (double)by[i];
            syy[i] += (double)byy[i];
        }
    }
    const double s_ref = scal[0], sum_xt = scal[1];
#pragma unroll
    for (int i = 0; i < VEC; ++i) {
        const double mean_shift = sy[i] / (double)M;
        const double cov = sxy[i] - mean_shift * sum_xt;
        const double syy_c = syy[i] - sy[i] * mean_shift;
        double r = 0.0;
        if (syy_c > 0.0 && s_ref > 0.0) r = cov * s_ref / sqrt(syy_c);
        r = r > 1.0 ? 1.0 : (r < -1.0 ? -1.0 : r);
        out[v0 + i] = (float)r;
    }
}

bool pointer_usable(bool is_device, bool is_managed, int ptr_device, int current_device) {
    if (is_managed) return true;  // reachable from every device
    return is_device && ptr_device == current_device;
}

// Device (or managed) memory of the current device; memory of another GPU is
// rejected, since the kernels read their buffers without peer access.
bool is_device_ptr(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return pointer_usable(a.type == cudaMemoryTypeDevice, a.type == cudaMemoryTypeManaged,
                          a.device, dev);
}

}  // namespace

extern "C" ndf_status ndf_pearson_noalloc(const float* ref_field, const float* query_field,
                                          int64_t M, int64_t N, int64_t ref_idx, float* out,
                                          void* cuda_stream) {
    if (!ref_field || !query_field || !out) return NDF_ERR_ARG;
    if (M < 2 || M > kMaxM || N < 1 || ref_idx < 0 || ref_idx >= N) return NDF_ERR_ARG;
    // an error left pending by the caller's earlier work is reported, not consumed
    if (cudaPeekAtLastError() != cudaSuccess) return NDF_ERR_CUDA;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return NDF_ERR_CUDA;
    if (!is_device_ptr(ref_field, dev) || !is_device_ptr(query_field, dev) ||
        !is_device_ptr(out, dev))
        return NDF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    void* scratch = nullptr;
    ndf_status st = scratch_address(s, &scratch);
    if (st != NDF_OK) return st;
    unsigned char* sc = static_cast<unsigned char*>(scratch);
    noalloc_stage_kernel<<<1, 1024, 0, s>>>(ref_field, (int)M, N, ref_idx, sc);
    if (cudaGetLastError() != cudaSuccess) return NDF_ERR_CUDA;
    if (N % 4 == 0 && (reinterpret_cast<uintptr_t>(query_field) & 15) == 0) {
        const int64_t blocks = (N / 4 + 255) / 256;
        noalloc_volume_kernel<4><<<(unsigned)blocks, 256, 0, s>>>(query_field, (int)M, N, sc, out);
    } else {
        const int64_t blocks = (N + 255) / 256;
        noalloc_volume_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(query_field, (int)M, N, sc, out);
    }
    return cudaGetLastError() == cudaSuccess ? NDF_OK : NDF_ERR_CUDA;
}

// The pointer rule of ndf_pearson_noalloc as a pure function of the attributes
// (a host-side hook, so that the rule is testable without a second GPU).
extern "C" int ndf_noalloc_pointer_usable(int is_device, int is_managed, int ptr_device,
                                          int current_device) {
    return pointer_usable(is_device != 0, is_managed != 0, ptr_device, current_device) ? 1 : 0;
}

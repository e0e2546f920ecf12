// Neural dependence field (Sec. 4): dense-grid encoding, multiplicative merge,
// 3 x 128 ReLU MLP, tanh / softplus output, L1 loss (Eq. 3), backward, Adam.
//
// Kernels (all BF16 tensor-core math accumulates in FP32):
//   encode_merge_fwd   trilinear gathers from the BF16 grid (32 B per corner point),
//                      f_ref, f_q in FP32 and x = [f_ref*f_q ; f_ref+f_q] in BF16
//   MLP forward, data and weight gradients: tcgen05 kernels in ndf_mlp_tc.cu
//   encode_bwd         d f through the merge, scattered to the FP32 grid gradient
//                      with 16-byte vector reductions (red.global.add.v4.f32)
//   adam               fused Adam over the flat FP32 master (grid + MLP), writes the
//                      BF16 grid copy
#include <math.h>

#include "device_common.cuh"
#include "ndf_net.h"

namespace ndf {

void NetLayout::init(const int r[kLevels]) {
    int64_t p = 0;
    for (int l = 0; l < kLevels; ++l) {
        res[l] = r[l];
        grid_off[l] = p;
        p += (int64_t)r[l] * r[l] * r[l] * kFeat;
    }
    n_grid = p;
    W1 = p; p += (int64_t)kHid * kIn;
    b1 = p; p += kHid;
    W2 = p; p += (int64_t)kHid * kHid;
    b2 = p; p += kHid;
    W3 = p; p += (int64_t)kHid * kHid;
    b3 = p; p += kHid;
    w4 = p; p += kHid;
    b4 = p; p += 1;
    total = p;
}

void NetWork::release() {
    void* ps[] = {fr, fq, x, wpart, cpart, dx, pos, target, loss};
    for (void* q : ps)
        if (q) cudaFree(q);
    *this = NetWork();
}

struct GridDev {
    const __nv_bfloat16* grid;
    int res[kLevels];
    int64_t off[kLevels];
};

// ---------------------------------------------------------------- small helpers
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t u) {
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&u);
    return __bfloat1622float2(v);
}

// trilinear corners of p at one level (corner-aligned grid of R points per axis on [-1,1])
__device__ __forceinline__ void corners(const float* p, int R, int64_t (&idx)[8], float (&w)[8]) {
    int i[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = (p[a] + 1.0f) * 0.5f * (float)(R - 1);
        int k = (int)floorf(u);
        k = k < 0 ? 0 : (k > R - 2 ? R - 2 : k);
        i[a] = k;
        f[a] = u - (float)k;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        idx[c] = ((int64_t)(i[2] + dz) * R + (i[1] + dy)) * R + (i[0] + dx);
        w[c] = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
    }
}

// 16 interpolated features of one level (two 16-byte loads per corner point)
__device__ __forceinline__ void encode_level(const GridDev& G, int l, const float* p,
                                             float (&out)[kFeat]) {
    int64_t idx[8];
    float w[8];
    corners(p, G.res[l], idx, w);
#pragma unroll
    for (int f = 0; f < kFeat; ++f) out[f] = 0.0f;
    const uint4* base = reinterpret_cast<const uint4*>(G.grid + G.off[l]);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint4* q = base + idx[c] * 2;
        uint4 u0 = __ldg(q), u1 = __ldg(q + 1);
        uint32_t uu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float2 v = unpack_bf16(uu[j]);
            out[2 * j] = fmaf(w[c], v.x, out[2 * j]);
            out[2 * j + 1] = fmaf(w[c], v.y, out[2 * j + 1]);
        }
    }
}

// ---------------------------------------------------------------- encode + merge
__global__ void __launch_bounds__(256)
    encode_merge_fwd_kernel(GridDev G, const float* __restrict__ pr, const float* __restrict__ pq,
                            int64_t B, float* __restrict__ fr, float* __restrict__ fq,
                            __nv_bfloat16* __restrict__ x) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * kLevels) return;
    const int64_t b = t / kLevels;
    const int l = (int)(t % kLevels);
    float a[kFeat], c[kFeat];
    encode_level(G, l, pr + 3 * b, a);
    encode_level(G, l, pq + 3 * b, c);
    float4* o1 = reinterpret_cast<float4*>(fr + b * kLF + l * kFeat);
    float4* o2 = reinterpret_cast<float4*>(fq + b * kLF + l * kFeat);
    uint32_t mul[8], add[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        o1[j] = make_float4(a[4 * j], a[4 * j + 1], a[4 * j + 2], a[4 * j + 3]);
        o2[j] = make_float4(c[4 * j], c[4 * j + 1], c[4 * j + 2], c[4 * j + 3]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        mul[j] = pack_bf16(a[2 * j] * c[2 * j], a[2 * j + 1] * c[2 * j + 1]);
        add[j] = pack_bf16(a[2 * j] + c[2 * j], a[2 * j + 1] + c[2 * j + 1]);
    }
    uint4* xm = reinterpret_cast<uint4*>(x + b * kIn + l * kFeat);
    uint4* xa = reinterpret_cast<uint4*>(x + b * kIn + kLF + l * kFeat);
    xm[0] = make_uint4(mul[0], mul[1], mul[2], mul[3]);
    xm[1] = make_uint4(mul[4], mul[5], mul[6], mul[7]);
    xa[0] = make_uint4(add[0], add[1], add[2], add[3]);
    xa[1] = make_uint4(add[4], add[5], add[6], add[7]);
}

// ---------------------------------------------------------------- encode backward
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

// Thread per (sample, level, side, quad of four features): the four threads of a
// (sample, level, side) scatter the four 16-byte quads of each corner point in the
// same warp instruction, so each reduction instruction covers eight corner points'
// 64 contiguous bytes each instead of 32 scattered 16-byte pieces.
__global__ void __launch_bounds__(256)
    encode_bwd_kernel(GridDev G, const float* __restrict__ pr, const float* __restrict__ pq,
                      int64_t B, const float* __restrict__ fr, const float* __restrict__ fq,
                      const float* __restrict__ dx, float* __restrict__ ggrid) {
    const int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tt >= B * kLevels * 2 * 4) return;
    const int q = (int)(tt & 3);
    const int side = (int)((tt >> 2) & 1);
    const int64_t rest = tt >> 3;
    const int64_t b = rest / kLevels;
    const int l = (int)(rest % kLevels);
    // x = [fr*fq ; fr+fq]:  d fr = dx_mul * fq + dx_add,  d fq = dx_mul * fr + dx_add
    const int f0 = l * kFeat + 4 * q;
    const float4 o = *reinterpret_cast<const float4*>((side == 0 ? fq : fr) + b * kLF + f0);
    const float4 dm = *reinterpret_cast<const float4*>(dx + b * kIn + f0);
    const float4 da = *reinterpret_cast<const float4*>(dx + b * kIn + kLF + f0);
    const float d0 = fmaf(dm.x, o.x, da.x), d1 = fmaf(dm.y, o.y, da.y);
    const float d2 = fmaf(dm.z, o.z, da.z), d3 = fmaf(dm.w, o.w, da.w);
    int64_t idx[8];
    float w[8];
    corners((side == 0 ? pr : pq) + 3 * b, G.res[l], idx, w);
    float* base = ggrid + G.off[l] + 4 * q;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        red_add_v4(base + idx[c] * kFeat, w[c] * d0, w[c] * d1, w[c] * d2, w[c] * d3);
}

// ---------------------------------------------------------------- Adam
// Adam over the flat FP32 master: four parameters per thread and iteration with
// 16-byte accesses (the parameter count is padded to a multiple of 4 in every
// buffer); the grid part also refreshes its BF16 copy.
__device__ __forceinline__ float adam_one(float& p, float g, float& m, float& v, float lr,
                                          float beta1, float beta2, float eps, float c1, float c2) {
    m = beta1 * m + (1.0f - beta1) * g;
    v = beta2 * v + (1.0f - beta2) * g * g;
    p = p - lr * (m / c1) / (sqrtf(v / c2) + eps);
    return p;
}

__device__ __forceinline__ void adam4(float4& P, const float4& G, float4& Mv, float4& V, float lr,
                                      float beta1, float beta2, float eps, float c1, float c2) {
    adam_one(P.x, G.x, Mv.x, V.x, lr, beta1, beta2, eps, c1, c2);
    adam_one(P.y, G.y, Mv.y, V.y, lr, beta1, beta2, eps, c1, c2);
    adam_one(P.z, G.z, Mv.z, V.z, lr, beta1, beta2, eps, c1, c2);
    adam_one(P.w, G.w, Mv.w, V.w, lr, beta1, beta2, eps, c1, c2);
}

__device__ __forceinline__ void put_bf16x4(__nv_bfloat16* grid_bf, int64_t i, const float4& P) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(P.x, P.y), hi = __floats2bfloat162_rn(P.z, P.w);
    uint2 w;
    w.x = *reinterpret_cast<uint32_t*>(&lo);
    w.y = *reinterpret_cast<uint32_t*>(&hi);
    __stcs(reinterpret_cast<uint2*>(grid_bf) + i, w);
}

// One group of four parameters per thread and iteration, 64 CTAs of 256 threads per
// SM (measured on the full model: 6.0 TB/s, against 4.9 TB/s for two groups per
// thread at 16 CTAs per SM); every array is streamed once per step, so loads and
// stores bypass L2 retention (evict-first).  With CLEAR the gradient is zeroed after
// it is read, which replaces a separate clear of the whole buffer before the next
// step.
template <bool CLEAR>
__global__ void __launch_bounds__(256)
    adam_kernel(float* __restrict__ p, float* __restrict__ gr, float* __restrict__ m,
                float* __restrict__ v, int64_t n, int64_t n_grid, __nv_bfloat16* __restrict__ grid_bf,
                float lr, float beta1, float beta2, float eps, float c1, float c2) {
    const int64_t n4 = (n + 3) >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float4* p4 = reinterpret_cast<float4*>(p);
    float4* m4 = reinterpret_cast<float4*>(m);
    float4* v4 = reinterpret_cast<float4*>(v);
    float4* g4 = reinterpret_cast<float4*>(gr);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 P = __ldcs(p4 + i), M = __ldcs(m4 + i), V = __ldcs(v4 + i);
        const float4 G = __ldcs(g4 + i);
        adam4(P, G, M, V, lr, beta1, beta2, eps, c1, c2);
        __stcs(p4 + i, P);
        __stcs(m4 + i, M);
        __stcs(v4 + i, V);
        if (CLEAR) __stcs(g4 + i, make_float4(0.f, 0.f, 0.f, 0.f));
        if ((i << 2) + 3 < n_grid) put_bf16x4(grid_bf, i, P);  // n_grid is a multiple of 16
    }
}

__global__ void refresh_mlp_kernel(const float* __restrict__ p, int64_t offW1, int64_t offW2,
                                   int64_t offW3, __nv_bfloat16* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * kHid * kHid) return;
    const int l = i / (kHid * kHid), r = (i / kHid) % kHid, c = i % kHid;
    const int64_t off = l == 0 ? offW1 : (l == 1 ? offW2 : offW3);
    w[(size_t)l * kHid * kHid + r * kHid + c] = __float2bfloat16_rn(p[off + (int64_t)r * kHid + c]);
}

__global__ void grid_to_bf16_kernel(const float* __restrict__ p, int64_t n,
                                    __nv_bfloat16* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(p[i]);
}

// counter-based uniform in [-1, 1): SplitMix64 output mix of key + (i+1)*golden
__device__ __forceinline__ float hash_uniform(uint64_t key, uint64_t i) {
    uint64_t z = key + (i + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return (float)((double)(z >> 11) * 0x1.0p-53) * 2.0f - 1.0f;
}

// grid U(-1e-4, 1e-4); dense weights He-uniform U(-sqrt(6/fan_in), +); biases 0
__global__ void init_params_kernel(float* __restrict__ p, int64_t n_grid, int64_t offW1,
                                   int64_t offW2, int64_t offW3, int64_t offw4, int64_t total,
                                   uint64_t key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        if (i < n_grid) s = 1e-4f;
        else if ((i >= offW1 && i < offW1 + kHid * kIn) || (i >= offW2 && i < offW2 + kHid * kHid) ||
                 (i >= offW3 && i < offW3 + kHid * kHid) || (i >= offw4 && i < offw4 + kHid))
            s = sqrtf(6.0f / 128.0f);
        p[i] = s * hash_uniform(key, (uint64_t)i);
    }
}

// ---------------------------------------------------------------- host side
static GridDev grid_dev(const ndf_model* m) {
    GridDev G;
    G.grid = m->grid_bf;
    for (int l = 0; l < kLevels; ++l) {
        G.res[l] = m->L.res[l];
        G.off[l] = m->L.grid_off[l];
    }
    return G;
}

ndf_status model_alloc(ndf_ctx* ctx, const int res[kLevels], int measure, int64_t X, int64_t Y,
                       int64_t Z, ndf_model** out) {
    for (int l = 0; l < kLevels; ++l)
        if (res[l] < 2 || res[l] > 1024) return fail(ctx, NDF_ERR_ARG, "grid resolution out of [2, 1024]");
    if (measure != 0 && measure != 1) return fail(ctx, NDF_ERR_ARG, "unknown measure");
    ndf_model* m = new (std::nothrow) ndf_model();
    if (!m) return fail(ctx, NDF_ERR_OOM, "model allocation");
    m->ctx = ctx;
    m->L.init(res);
    m->measure = measure;
    m->X = X;
    m->Y = Y;
    m->Z = Z;
    const size_t n = ((size_t)m->L.total + 3) & ~size_t(3);  // float4 Adam: pad to 4
    cudaError_t e = cudaMalloc(&m->params, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->grid_bf, (size_t)m->L.n_grid * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->wbf, (size_t)3 * kHid * kHid * 2);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->params, 0, n * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, n * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, n * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, n * 4, ctx->stream);
    if (e != cudaSuccess) {
        model_free(m);
        return cuda_fail(ctx, e, "model allocation");
    }
    *out = m;
    return NDF_OK;
}

void model_free(ndf_model* m) {
    if (!m) return;
    void* ps[] = {m->params, m->grad, m->m, m->v, m->grid_bf, m->wbf};
    for (void* q : ps)
        if (q) cudaFree(q);
    m->work.release();
    delete m;
}

cudaError_t model_refresh_bf16(ndf_model* m) {
    ndf_ctx* ctx = m->ctx;
    grid_to_bf16_kernel<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(m->params, m->L.n_grid,
                                                                      m->grid_bf);
    refresh_mlp_kernel<<<(3 * kHid * kHid + 255) / 256, 256, 0, ctx->stream>>>(
        m->params, m->L.W1, m->L.W2, m->L.W3, m->wbf);
    ctx->launches += 2;
    return cudaGetLastError();
}

cudaError_t model_init_params(ndf_model* m, uint64_t seed) {
    ndf_ctx* ctx = m->ctx;
    uint64_t key = seed * 0xd1b54a32d192ed03ULL + 0x2545f4914f6cdd1dULL;
    init_params_kernel<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(
        m->params, m->L.n_grid, m->L.W1, m->L.W2, m->L.W3, m->L.w4, m->L.total, key);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // biases start at 0 (the uniform draw above is scaled by 0 for them)
    return model_refresh_bf16(m);
}

ndf_status ensure_work(ndf_model* m, int64_t B) {
    NetWork& w = m->work;
    if (w.cap >= B) return NDF_OK;
    w.release();
    cudaError_t e = cudaSuccess;
    auto al = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    const size_t b = (size_t)B;
    al((void**)&w.fr, b * kLF * 4);
    al((void**)&w.fq, b * kLF * 4);
    al((void**)&w.x, b * kIn * 2);
    al((void**)&w.wpart, (size_t)3 * kMlpMaxParts * kHid * kHid * 4);
    al((void**)&w.cpart, (size_t)kMlpMaxParts * 4 * 5 * kHid * 4);
    al((void**)&w.dx, b * kIn * 4);
    al((void**)&w.pos, 6 * b * 4);
    al((void**)&w.target, b * 4);
    al((void**)&w.loss, 8);
    if (e != cudaSuccess) {
        w.release();
        return cuda_fail(m->ctx, e, "network work buffers");
    }
    w.cap = B;
    return NDF_OK;
}

cudaError_t model_step(ndf_model* m, const float* pr, const float* pq, const float* target,
                       int64_t B, float lr, float beta1, float beta2, float eps, bool update,
                       bool keep_grad) {
    ndf_ctx* ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    NetWork& w = m->work;
    // gradients start from zero every step: Adam clears them as it reads them, so only
    // after a step that kept its gradient is the buffer cleared here.  The loss sum in
    // w.loss accumulates across steps (callers zero it).
    cudaError_t e = cudaSuccess;
    if (!m->grad_zero) {
        e = cudaMemsetAsync(m->grad, 0, (((size_t)m->L.total + 3) & ~size_t(3)) * 4, s);
        if (e != cudaSuccess) return e;
        m->grad_zero = true;
    }
    const GridDev G = grid_dev(m);
    encode_merge_fwd_kernel<<<(unsigned)((B * kLevels + 255) / 256), 256, 0, s>>>(G, pr, pq, B, w.fr,
                                                                                 w.fq, w.x);
    ctx->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = mlp_tc_train(m, B, target)) != cudaSuccess) return e;
    encode_bwd_kernel<<<(unsigned)((B * kLevels * 2 * 4 + 255) / 256), 256, 0, s>>>(
        G, pr, pq, B, w.fr, w.fq, w.dx, m->grad);
    ctx->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (update) {
        m->t += 1;
        const float c1 = (float)(1.0 - pow((double)beta1, (double)m->t));
        const float c2 = (float)(1.0 - pow((double)beta2, (double)m->t));
        // 64 CTAs per SM, or one thread per group of four parameters if that is fewer
        const int64_t groups_ctas = ((m->L.total + 3) / 4 + 255) / 256;
        const unsigned ctas = (unsigned)(groups_ctas < (int64_t)ctx->sm_count * 64 ? groups_ctas
                                                                                   : (int64_t)ctx->sm_count * 64);
        if (keep_grad)
            adam_kernel<false><<<ctas, 256, 0, s>>>(m->params, m->grad, m->m, m->v, m->L.total, m->L.n_grid,
                                                    m->grid_bf, lr, beta1, beta2, eps, c1, c2);
        else
            adam_kernel<true><<<ctas, 256, 0, s>>>(m->params, m->grad, m->m, m->v, m->L.total, m->L.n_grid,
                                                   m->grid_bf, lr, beta1, beta2, eps, c1, c2);
        refresh_mlp_kernel<<<(3 * kHid * kHid + 255) / 256, 256, 0, s>>>(
            m->params, m->L.W1, m->L.W2, m->L.W3, m->wbf);
        ctx->launches += 2;
        e = cudaGetLastError();
    }
    m->grad_zero = update && !keep_grad;
    return e;
}

cudaError_t model_forward(ndf_model* m, const float* pr, const float* pq, int64_t B, float* out) {
    ndf_ctx* ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    NetWork& w = m->work;
    const GridDev G = grid_dev(m);
    encode_merge_fwd_kernel<<<(unsigned)((B * kLevels + 255) / 256), 256, 0, s>>>(G, pr, pq, B, w.fr,
                                                                                 w.fq, w.x);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return mlp_tc_forward(m, B, out);
}

cudaError_t net_set_attributes() { return cudaSuccess; }  // the tcgen05 kernels set their own

}  // namespace ndf

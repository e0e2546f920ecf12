// Neural dependence field (Sec. 4): dense-grid encoding, multiplicative merge,
// 3 x 128 ReLU MLP, tanh / softplus output, L1 loss (Eq. 3), backward, Adam.
//
// Kernels (all BF16 tensor-core math accumulates in FP32):
//   encode_merge_fwd   trilinear gathers from the BF16 grid (32 B per corner point),
//                      f_ref, f_q in FP32 and x = [f_ref*f_q ; f_ref+f_q] in BF16
//   mlp_fwd            one warp per 16 rows; mma.sync m16n8k16; the accumulator of
//                      a layer is repacked in registers as the next layer's A
//                      operand; weights in padded shared memory
//   mlp_bwd_data       same structure backwards: dz3 -> dz2 -> dz1 -> dx, using the
//                      transposed weights
//   mlp_bwd_weight     dW = dz^T h over the batch: ldmatrix.trans fragments of
//                      128-row tiles, per-CTA partial sums, FP32 atomics
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
    void* ps[] = {fr, fq, x, h, dz, dx, o, dout, pos, target, loss};
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

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ float act_out(int measure, float o) {
    if (measure == 0) return tanhf(o);
    return o > 20.0f ? o : log1pf(expf(o));
}

__device__ __forceinline__ float dact_out(int measure, float o) {
    if (measure == 0) {
        float t = tanhf(o);
        return 1.0f - t * t;
    }
    return 1.0f / (1.0f + expf(-o));
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

// ---------------------------------------------------------------- fused MLP
struct MlpArgs {
    const __nv_bfloat16* w;    // [3][128][128] forward weights ([out][in]) or transposes
    const float* params;       // FP32 master (biases, w4, b4)
    int64_t off_b[3];
    int64_t off_w4, off_b4;
    int64_t B;
    const __nv_bfloat16* x;    // [B][128]
    __nv_bfloat16* h;          // [3][B][128]
    __nv_bfloat16* dz;         // [3][B][128]
    float* dx;                 // [B][128]
    float* o;                  // [B]
    float* dout;               // [B]
    const float* target;       // [B] or null
    float* y;                  // [B] output (forward only) or null
    double* loss;              // sum |y - t|
    int measure;
};

// copy three 128x128 bf16 matrices into padded shared rows
__device__ __forceinline__ void load_weights(__nv_bfloat16* sW, const __nv_bfloat16* w) {
    for (int i = threadIdx.x; i < 3 * kHid * (kHid / 8); i += blockDim.x) {
        const int mat = i / (kHid * kHid / 8);
        const int rem = i % (kHid * kHid / 8);
        const int row = rem / (kHid / 8), c8 = rem % (kHid / 8);
        const uint4 v = reinterpret_cast<const uint4*>(w + (size_t)mat * kHid * kHid)[row * (kHid / 8) + c8];
        *reinterpret_cast<uint4*>(sW + (size_t)mat * kHid * kWStride + row * kWStride + c8 * 8) = v;
    }
}

// acc[j] (n-tile j) += A . W^T for one 128x128 layer; W rows [n][k] padded in shared
__device__ __forceinline__ void layer_mma(float (&acc)[16][4], const uint32_t (&A)[8][4],
                                          const __nv_bfloat16* sW, int g, int t) {
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const __nv_bfloat16* row = sW + (8 * j + g) * kWStride + 16 * kk + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
            mma_bf16(acc[j], A[kk], b0, b1);
        }
    }
}

// C-fragment tile (16 rows x 128) -> A fragments of the next layer
__device__ __forceinline__ void c_to_a(const float (&c)[16][4], uint32_t (&A)[8][4]) {
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        A[kk][0] = pack_bf16(c[2 * kk][0], c[2 * kk][1]);
        A[kk][1] = pack_bf16(c[2 * kk][2], c[2 * kk][3]);
        A[kk][2] = pack_bf16(c[2 * kk + 1][0], c[2 * kk + 1][1]);
        A[kk][3] = pack_bf16(c[2 * kk + 1][2], c[2 * kk + 1][3]);
    }
}

// A fragments of a [B][128] bf16 matrix for rows r0..r0+15 (zero past B)
__device__ __forceinline__ void load_a(const __nv_bfloat16* m, int64_t r0, int64_t B, int g, int t,
                                       uint32_t (&A)[8][4]) {
    const int64_t ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const int c = 16 * kk + 2 * t;
        A[kk][0] = ra < B ? *reinterpret_cast<const uint32_t*>(m + ra * kIn + c) : 0u;
        A[kk][1] = rb < B ? *reinterpret_cast<const uint32_t*>(m + rb * kIn + c) : 0u;
        A[kk][2] = ra < B ? *reinterpret_cast<const uint32_t*>(m + ra * kIn + c + 8) : 0u;
        A[kk][3] = rb < B ? *reinterpret_cast<const uint32_t*>(m + rb * kIn + c + 8) : 0u;
    }
}

// store a C tile as bf16 (rows r0+g, r0+g+8; columns 8j+2t, +1)
__device__ __forceinline__ void store_c_bf16(__nv_bfloat16* m, const float (&c)[16][4], int64_t r0,
                                             int64_t B, int g, int t) {
    const int64_t ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int col = 8 * j + 2 * t;
        if (ra < B) *reinterpret_cast<uint32_t*>(m + ra * kHid + col) = pack_bf16(c[j][0], c[j][1]);
        if (rb < B) *reinterpret_cast<uint32_t*>(m + rb * kHid + col) = pack_bf16(c[j][2], c[j][3]);
    }
}

template <bool TRAIN>
__global__ void __launch_bounds__(256) mlp_fwd_kernel(MlpArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem);
    load_weights(sW, a.w);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t tiles = (a.B + 15) / 16;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    double loss_acc = 0.0;
    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile < tiles;
         tile += warps_total) {
        const int64_t r0 = tile * 16;
        uint32_t A[8][4];
        load_a(a.x, r0, a.B, g, t, A);
        float c[16][4];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const float* bias = a.params + a.off_b[l];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
                c[j][0] = b0; c[j][1] = b1; c[j][2] = b0; c[j][3] = b1;
            }
            layer_mma(c, A, sW + (size_t)l * kHid * kWStride, g, t);
#pragma unroll
            for (int j = 0; j < 16; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) c[j][e] = fmaxf(c[j][e], 0.0f);
            if (TRAIN) store_c_bf16(a.h + (size_t)l * a.B * kHid, c, r0, a.B, g, t);
            c_to_a(c, A);
        }
        // output layer: o = w4 . h3 + b4 (h3 as rounded to BF16, as stored)
        float s0 = 0.0f, s1 = 0.0f;
        const float* w4 = a.params + a.off_w4;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int c0 = 16 * kk + 2 * t;
            float2 h;
            h = unpack_bf16(A[kk][0]); s0 = fmaf(w4[c0], h.x, fmaf(w4[c0 + 1], h.y, s0));
            h = unpack_bf16(A[kk][1]); s1 = fmaf(w4[c0], h.x, fmaf(w4[c0 + 1], h.y, s1));
            h = unpack_bf16(A[kk][2]); s0 = fmaf(w4[c0 + 8], h.x, fmaf(w4[c0 + 9], h.y, s0));
            h = unpack_bf16(A[kk][3]); s1 = fmaf(w4[c0 + 8], h.x, fmaf(w4[c0 + 9], h.y, s1));
        }
        s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
        s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
        const float b4 = a.params[a.off_b4];
        if (t == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t r = r0 + g + 8 * h;
                if (r >= a.B) continue;
                const float o = (h ? s1 : s0) + b4;
                const float y = act_out(a.measure, o);
                if (TRAIN) {
                    a.o[r] = o;
                    const float e = y - a.target[r];
                    loss_acc += fabs((double)e);
                    const float sg = e > 0.0f ? 1.0f : (e < 0.0f ? -1.0f : 0.0f);
                    a.dout[r] = sg / (float)a.B * dact_out(a.measure, o);
                } else {
                    a.y[r] = y;
                }
            }
        }
    }
    if (TRAIN) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
        if (lane == 0 && loss_acc != 0.0) atomicAdd(a.loss, loss_acc);
    }
}

__global__ void __launch_bounds__(256) mlp_bwd_data_kernel(MlpArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem);  // transposes [in][out]
    load_weights(sW, a.w);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t tiles = (a.B + 15) / 16;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const float* w4 = a.params + a.off_w4;
    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile < tiles;
         tile += warps_total) {
        const int64_t r0 = tile * 16, ra = r0 + g, rb = r0 + g + 8;
        const float da = ra < a.B ? a.dout[ra] : 0.0f;
        const float db = rb < a.B ? a.dout[rb] : 0.0f;
        float c[16][4];
        // dz3 = dout * w4 * [h3 > 0]
        const __nv_bfloat16* h3 = a.h + (size_t)2 * a.B * kHid;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = 8 * j + 2 * t;
            const float2 ha = ra < a.B ? unpack_bf16(*reinterpret_cast<const uint32_t*>(h3 + ra * kHid + col)) : make_float2(0.f, 0.f);
            const float2 hb = rb < a.B ? unpack_bf16(*reinterpret_cast<const uint32_t*>(h3 + rb * kHid + col)) : make_float2(0.f, 0.f);
            c[j][0] = ha.x > 0.0f ? da * w4[col] : 0.0f;
            c[j][1] = ha.y > 0.0f ? da * w4[col + 1] : 0.0f;
            c[j][2] = hb.x > 0.0f ? db * w4[col] : 0.0f;
            c[j][3] = hb.y > 0.0f ? db * w4[col + 1] : 0.0f;
        }
        uint32_t A[8][4];
        for (int l = 2; l >= 0; --l) {
            store_c_bf16(a.dz + (size_t)l * a.B * kHid, c, r0, a.B, g, t);
            c_to_a(c, A);
#pragma unroll
            for (int j = 0; j < 16; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) c[j][e] = 0.0f;
            // d(input of layer l) = dz_l . W_l  (B operand: W_l^T rows [in][out])
            layer_mma(c, A, sW + (size_t)l * kHid * kWStride, g, t);
            if (l > 0) {  // through the ReLU of h_{l-1}
                const __nv_bfloat16* hp = a.h + (size_t)(l - 1) * a.B * kHid;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = 8 * j + 2 * t;
                    const float2 ha = ra < a.B ? unpack_bf16(*reinterpret_cast<const uint32_t*>(hp + ra * kHid + col)) : make_float2(0.f, 0.f);
                    const float2 hb = rb < a.B ? unpack_bf16(*reinterpret_cast<const uint32_t*>(hp + rb * kHid + col)) : make_float2(0.f, 0.f);
                    if (!(ha.x > 0.0f)) c[j][0] = 0.0f;
                    if (!(ha.y > 0.0f)) c[j][1] = 0.0f;
                    if (!(hb.x > 0.0f)) c[j][2] = 0.0f;
                    if (!(hb.y > 0.0f)) c[j][3] = 0.0f;
                }
            }
        }
        // c holds dx (FP32)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = 8 * j + 2 * t;
            if (ra < a.B) *reinterpret_cast<float2*>(a.dx + ra * kIn + col) = make_float2(c[j][0], c[j][1]);
            if (rb < a.B) *reinterpret_cast<float2*>(a.dx + rb * kIn + col) = make_float2(c[j][2], c[j][3]);
        }
    }
}

// dW_l = sum_b dz_l[b]^T h_{l-1}[b] (h_0 = x), db_l = sum_b dz_l[b]; one CTA per
// (row chunk, layer), 8 warps x 16 output rows, 128-row tiles in shared memory.
constexpr int kWgRows = 128;
constexpr int kTileStride = kHid + 8;
constexpr size_t kWgSmem = (size_t)2 * kWgRows * kTileStride * sizeof(__nv_bfloat16);

__global__ void __launch_bounds__(256)
    mlp_bwd_weight_kernel(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ h,
                          const __nv_bfloat16* __restrict__ dz, int64_t B, int64_t rows_per_cta,
                          float* __restrict__ grad, int64_t offW1, int64_t offW2, int64_t offW3,
                          int64_t offb1, int64_t offb2, int64_t offb3) {
    extern __shared__ __align__(16) unsigned char smem_wg[];
    __nv_bfloat16* S = reinterpret_cast<__nv_bfloat16*>(smem_wg);  // dz tile [b][i]
    __nv_bfloat16* S2 = S + kWgRows * kTileStride;                  // h tile  [b][j]
    const int l = blockIdx.y;
    const __nv_bfloat16* dzl = dz + (size_t)l * B * kHid;
    const __nv_bfloat16* hin = l == 0 ? x : h + (size_t)(l - 1) * B * kHid;
    const int64_t offW = l == 0 ? offW1 : (l == 1 ? offW2 : offW3);
    const int64_t offb = l == 0 ? offb1 : (l == 1 ? offb2 : offb3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[16][4];
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][e] = 0.0f;
    float bsum = 0.0f;
    const int64_t c0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t c1 = c0 + rows_per_cta < B ? c0 + rows_per_cta : B;
    for (int64_t b0 = c0; b0 < c1; b0 += kWgRows) {
        __syncthreads();
        for (int i = threadIdx.x; i < kWgRows * (kHid / 8); i += blockDim.x) {
            const int r = i / (kHid / 8), c8 = i % (kHid / 8);
            const int64_t row = b0 + r;
            uint4 u = make_uint4(0, 0, 0, 0), v = make_uint4(0, 0, 0, 0);
            if (row < c1) {
                u = reinterpret_cast<const uint4*>(dzl + row * kHid)[c8];
                v = reinterpret_cast<const uint4*>(hin + row * kHid)[c8];
            }
            *reinterpret_cast<uint4*>(S + r * kTileStride + c8 * 8) = u;
            *reinterpret_cast<uint4*>(S2 + r * kTileStride + c8 * 8) = v;
        }
        __syncthreads();
        if (threadIdx.x < kHid) {  // bias gradient: column sums of dz
            for (int r = 0; r < kWgRows; ++r) bsum += __bfloat162float(S[r * kTileStride + threadIdx.x]);
        }
        const int m = lane >> 3, rr = lane & 7;
#pragma unroll
        for (int ks = 0; ks < kWgRows / 16; ++ks) {
            uint32_t A[4];
            {
                const int brow = ks * 16 + (m >> 1) * 8 + rr;
                const int icol = 16 * warp + (m & 1) * 8;
                ldsm_x4_trans(A, S + brow * kTileStride + icol);
            }
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                uint32_t Bf[4];
                const int brow = ks * 16 + (m & 1) * 8 + rr;
                const int jcol = 16 * p + (m >> 1) * 8;
                ldsm_x4_trans(Bf, S2 + brow * kTileStride + jcol);
                mma_bf16(acc[2 * p], A, Bf[0], Bf[1]);
                mma_bf16(acc[2 * p + 1], A, Bf[2], Bf[3]);
            }
        }
    }
    float* dW = grad + offW;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int i0 = 16 * warp + g, col = 8 * j + 2 * t;
        atomicAdd(dW + (int64_t)i0 * kHid + col, acc[j][0]);
        atomicAdd(dW + (int64_t)i0 * kHid + col + 1, acc[j][1]);
        atomicAdd(dW + (int64_t)(i0 + 8) * kHid + col, acc[j][2]);
        atomicAdd(dW + (int64_t)(i0 + 8) * kHid + col + 1, acc[j][3]);
    }
    if (threadIdx.x < kHid) atomicAdd(grad + offb + threadIdx.x, bsum);
}

// dw4 = sum_b dout[b] h3[b], db4 = sum_b dout[b]
__global__ void __launch_bounds__(128)
    out_layer_grad_kernel(const __nv_bfloat16* __restrict__ h3, const float* __restrict__ dout,
                          int64_t B, int64_t rows_per_cta, float* __restrict__ grad,
                          int64_t off_w4, int64_t off_b4) {
    const int j = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t c1 = c0 + rows_per_cta < B ? c0 + rows_per_cta : B;
    float s = 0.0f, sb = 0.0f;
    for (int64_t r = c0; r < c1; ++r) {
        const float d = dout[r];
        s = fmaf(d, __bfloat162float(h3[r * kHid + j]), s);
        sb += d;
    }
    atomicAdd(grad + off_w4 + j, s);
    if (j == 0) atomicAdd(grad + off_b4, sb);
}

// ---------------------------------------------------------------- encode backward
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

__global__ void __launch_bounds__(256)
    encode_bwd_kernel(GridDev G, const float* __restrict__ pr, const float* __restrict__ pq,
                      int64_t B, const float* __restrict__ fr, const float* __restrict__ fq,
                      const float* __restrict__ dx, float* __restrict__ ggrid) {
    const int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tt >= B * kLevels * 2) return;
    const int side = (int)(tt & 1);
    const int64_t rest = tt >> 1;
    const int64_t b = rest / kLevels;
    const int l = (int)(rest % kLevels);
    // x = [fr*fq ; fr+fq]:  d fr = dx_mul * fq + dx_add,  d fq = dx_mul * fr + dx_add
    const float* other = (side == 0 ? fq : fr) + b * kLF + l * kFeat;
    const float* dmul = dx + b * kIn + l * kFeat;
    const float* dadd = dx + b * kIn + kLF + l * kFeat;
    float d[kFeat];
#pragma unroll
    for (int f = 0; f < kFeat; ++f) d[f] = fmaf(dmul[f], other[f], dadd[f]);
    int64_t idx[8];
    float w[8];
    corners((side == 0 ? pr : pq) + 3 * b, G.res[l], idx, w);
    float* base = ggrid + G.off[l];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float* q = base + idx[c] * kFeat;
#pragma unroll
        for (int f = 0; f < kFeat; f += 4)
            red_add_v4(q + f, w[c] * d[f], w[c] * d[f + 1], w[c] * d[f + 2], w[c] * d[f + 3]);
    }
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

__global__ void __launch_bounds__(256)
    adam_kernel(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                float* __restrict__ v, int64_t n, int64_t n_grid, __nv_bfloat16* __restrict__ grid_bf,
                float lr, float beta1, float beta2, float eps, float c1, float c2) {
    const int64_t n4 = (n + 3) >> 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 P = reinterpret_cast<float4*>(p)[i];
        const float4 G = __ldcs(reinterpret_cast<const float4*>(gr) + i);
        float4 Mv = reinterpret_cast<float4*>(m)[i];
        float4 V = reinterpret_cast<float4*>(v)[i];
        adam_one(P.x, G.x, Mv.x, V.x, lr, beta1, beta2, eps, c1, c2);
        adam_one(P.y, G.y, Mv.y, V.y, lr, beta1, beta2, eps, c1, c2);
        adam_one(P.z, G.z, Mv.z, V.z, lr, beta1, beta2, eps, c1, c2);
        adam_one(P.w, G.w, Mv.w, V.w, lr, beta1, beta2, eps, c1, c2);
        reinterpret_cast<float4*>(p)[i] = P;
        reinterpret_cast<float4*>(m)[i] = Mv;
        reinterpret_cast<float4*>(v)[i] = V;
        const int64_t e = i << 2;
        if (e + 3 < n_grid) {  // n_grid is a multiple of 16
            __nv_bfloat162 lo = __floats2bfloat162_rn(P.x, P.y), hi = __floats2bfloat162_rn(P.z, P.w);
            uint2 w;
            w.x = *reinterpret_cast<uint32_t*>(&lo);
            w.y = *reinterpret_cast<uint32_t*>(&hi);
            reinterpret_cast<uint2*>(grid_bf)[i] = w;
        }
    }
}

__global__ void refresh_mlp_kernel(const float* __restrict__ p, int64_t offW1, int64_t offW2,
                                   int64_t offW3, __nv_bfloat16* __restrict__ w,
                                   __nv_bfloat16* __restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * kHid * kHid) return;
    const int l = i / (kHid * kHid), r = (i / kHid) % kHid, c = i % kHid;
    const int64_t off = l == 0 ? offW1 : (l == 1 ? offW2 : offW3);
    const __nv_bfloat16 b = __float2bfloat16_rn(p[off + (int64_t)r * kHid + c]);
    w[(size_t)l * kHid * kHid + r * kHid + c] = b;
    wt[(size_t)l * kHid * kHid + c * kHid + r] = b;
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

static MlpArgs mlp_args(ndf_model* m, int64_t B) {
    MlpArgs a{};
    a.params = m->params;
    a.off_b[0] = m->L.b1;
    a.off_b[1] = m->L.b2;
    a.off_b[2] = m->L.b3;
    a.off_w4 = m->L.w4;
    a.off_b4 = m->L.b4;
    a.B = B;
    a.x = m->work.x;
    a.h = m->work.h;
    a.dz = m->work.dz;
    a.dx = m->work.dx;
    a.o = m->work.o;
    a.dout = m->work.dout;
    a.loss = m->work.loss;
    a.measure = m->measure;
    return a;
}

static int persistent_grid(ndf_ctx* ctx, int64_t warps_needed) {
    int64_t g = (warps_needed + 7) / 8;
    int64_t cap = (int64_t)ctx->sm_count * 2;
    return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

constexpr size_t kMlpSmem = (size_t)3 * kHid * kWStride * sizeof(__nv_bfloat16);

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
    if (e == cudaSuccess) e = cudaMalloc(&m->wtbf, (size_t)3 * kHid * kHid * 2);
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
    void* ps[] = {m->params, m->grad, m->m, m->v, m->grid_bf, m->wbf, m->wtbf};
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
        m->params, m->L.W1, m->L.W2, m->L.W3, m->wbf, m->wtbf);
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
    al((void**)&w.h, 3 * b * kHid * 2);
    al((void**)&w.dz, 3 * b * kHid * 2);
    al((void**)&w.dx, b * kIn * 4);
    al((void**)&w.o, b * 4);
    al((void**)&w.dout, b * 4);
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
                       int64_t B, float lr, float beta1, float beta2, float eps, bool update) {
    ndf_ctx* ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    NetWork& w = m->work;
    // gradients start from zero every step; the loss sum in w.loss accumulates
    // across steps (callers zero it)
    cudaError_t e = cudaMemsetAsync(m->grad, 0, (((size_t)m->L.total + 3) & ~size_t(3)) * 4, s);
    if (e != cudaSuccess) return e;
    const GridDev G = grid_dev(m);
    encode_merge_fwd_kernel<<<(unsigned)((B * kLevels + 255) / 256), 256, 0, s>>>(G, pr, pq, B, w.fr,
                                                                                 w.fq, w.x);
    MlpArgs a = mlp_args(m, B);
    a.target = target;
    const int grid = persistent_grid(ctx, (B + 15) / 16);
    a.w = m->wbf;
    mlp_fwd_kernel<true><<<grid, 256, kMlpSmem, s>>>(a);
    a.w = m->wtbf;
    mlp_bwd_data_kernel<<<grid, 256, kMlpSmem, s>>>(a);
    const int64_t rows_per_cta = 4096;
    const unsigned chunks = (unsigned)((B + rows_per_cta - 1) / rows_per_cta);
    mlp_bwd_weight_kernel<<<dim3(chunks, 3), 256, kWgSmem, s>>>(w.x, w.h, w.dz, B, rows_per_cta, m->grad,
                                                          m->L.W1, m->L.W2, m->L.W3, m->L.b1,
                                                          m->L.b2, m->L.b3);
    out_layer_grad_kernel<<<chunks, kHid, 0, s>>>(w.h + (size_t)2 * B * kHid, w.dout, B,
                                                  rows_per_cta, m->grad, m->L.w4, m->L.b4);
    encode_bwd_kernel<<<(unsigned)((B * kLevels * 2 + 255) / 256), 256, 0, s>>>(
        G, pr, pq, B, w.fr, w.fq, w.dx, m->grad);
    ctx->launches += 6;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (update) {
        m->t += 1;
        const float c1 = (float)(1.0 - pow((double)beta1, (double)m->t));
        const float c2 = (float)(1.0 - pow((double)beta2, (double)m->t));
        adam_kernel<<<ctx->sm_count * 16, 256, 0, s>>>(m->params, m->grad, m->m, m->v, m->L.total,
                                                        m->L.n_grid, m->grid_bf, lr, beta1, beta2,
                                                        eps, c1, c2);
        refresh_mlp_kernel<<<(3 * kHid * kHid + 255) / 256, 256, 0, s>>>(
            m->params, m->L.W1, m->L.W2, m->L.W3, m->wbf, m->wtbf);
        ctx->launches += 2;
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t model_forward(ndf_model* m, const float* pr, const float* pq, int64_t B, float* out) {
    ndf_ctx* ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    NetWork& w = m->work;
    const GridDev G = grid_dev(m);
    encode_merge_fwd_kernel<<<(unsigned)((B * kLevels + 255) / 256), 256, 0, s>>>(G, pr, pq, B, w.fr,
                                                                                 w.fq, w.x);
    MlpArgs a = mlp_args(m, B);
    a.w = m->wbf;
    a.y = out;
    mlp_fwd_kernel<false><<<persistent_grid(ctx, (B + 15) / 16), 256, kMlpSmem, s>>>(a);
    ctx->launches += 2;
    return cudaGetLastError();
}

static bool g_attrs_set = false;
cudaError_t net_set_attributes() {
    if (g_attrs_set) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMlpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_bwd_data_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMlpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_bwd_weight_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kWgSmem);
    if (e == cudaSuccess) g_attrs_set = true;
    return e;
}

}  // namespace ndf

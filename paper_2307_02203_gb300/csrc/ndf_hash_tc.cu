// The hash-grid neural dependence field (Sec. 4.1-4.2, Fig. 2) decoded on the
// 5th-generation tensor cores: one kernel runs the whole per-vertex chain
//   embedding [p, Fourier (Eq. 4), hash-grid features]  (FP32, rounded to BF16)
//   -> encoder layers (BF16 x BF16 -> FP32 in TMEM), Snake-family activations
//   -> latent (FP32) merged with the reference latent (product / sum / |diff|)
//   -> decoder hidden layers -> output layer (FP32 dot) -> tanh / softplus.
// Every dense layer of width 128 is one tcgen05.mma chain (M = 128 vertices,
// N = 128 outputs, K = 128 inputs; the embedding's din <= 128 inputs are
// zero-padded).  Modes of the same kernel:
//   encode-only   the latents of a list of vertices (the references), FP32
//   decode        embedding -> encoder -> merge -> decoder for every vertex
//   cached decode the query latents were encoded once ([N][128] FP32); only
//                 merge -> decoder runs per reference
//
// CTA roles (one CTA per SM, persistent over 128-vertex tiles):
//   warps 0-3 / 4-7: two tile slots; thread i of a slot owns row i of its tile and
//     TMEM lane i.  It embeds its vertex into the slot's A tile (BF16, 128-byte-
//     swizzled K-major), then after each layer reads its accumulator row with
//     tcgen05.ld, adds the bias, applies the activation (or the merge) and
//     writes the next layer's A tile in place.
//   warp 8: allocates TMEM (2 x 128 columns); one lane issues the MMAs, layer by
//     layer for both slots, and commits to the slot's mbarrier and, once both
//     slots used a weight buffer, to that buffer's "empty" mbarrier.
//   warp 9: one lane streams the layers' weight images (32 KB each, pre-swizzled
//     in global memory, L2-resident) into a ring of three shared-memory buffers
//     with cp.async.bulk.
// All waits are bounded (polls and wall time); on timeout every role stops, the
// copies in flight are waited for, TMEM is freed and the status word is set.
#include <cuda_bf16.h>

#include "hash_common.cuh"
#include "ndf_hash_tc.h"
#include "tc_common.cuh"

namespace ndf {

namespace {

using namespace tc;

constexpr int kRows = 128;
constexpr int kSlots = 2;
constexpr int kRing = 3;
constexpr int kEpiWarps = 4 * kSlots;
constexpr int kThreads = 32 * (kEpiWarps + 2);
constexpr uint32_t kLayerBytes = 2 * kAtom;  // 128 x 128 BF16 = two K atoms
constexpr uint32_t kOffRing = 0;
constexpr uint32_t kOffA = kRing * kLayerBytes;
constexpr uint32_t kOffBias = kOffA + kSlots * kLayerBytes;
constexpr uint32_t kOffZr = kOffBias + kHashTcMaxLayers * 128 * 4;
constexpr uint32_t kOffWl = kOffZr + 128 * 4;
constexpr uint32_t kOffBar = kOffWl + 128 * 4;
constexpr uint32_t kSmem = kOffBar + 256 + 1024 /*alignment*/;
static_assert(kSmem <= 227 * 1024, "shared memory");

// element k of row `row` of a 128-row x 128-column BF16 operand tile
__device__ __forceinline__ void put_bf16(unsigned char* A, int row, int k, float v) {
    *reinterpret_cast<__nv_bfloat16*>(A + (uint32_t)(k >> 6) * kAtom + swz(row, (k >> 3) & 7) +
                                      (uint32_t)(k & 7) * 2) = __float2bfloat16_rn(v);
}

__device__ __forceinline__ float merge_f(int mode, float zr, float zq) {
    return mode == NDF_MERGE_PRODUCT ? zr * zq : (mode == NDF_MERGE_SUM ? zr + zq : fabsf(zr - zq));
}

// hidden-layer activation; the sine of the Snake family through the SFU
template <int ACT>
__device__ __forceinline__ float act_tc(float x) {
    if constexpr (ACT == NDF_ACT_RELU) {
        return fmaxf(x, 0.0f);
    } else {
        const float s = __sinf(x);
        return fmaf(s, s, ACT == NDF_ACT_SNAKE ? x : 0.5f * x);
    }
}

}  // namespace

template <int ACT>
__global__ void __launch_bounds__(kThreads, 1) hash_tc_kernel(const HashTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
    uint64_t* a_ready = bars;                   // [kSlots] epilogue -> MMA (128 arrivals)
    uint64_t* d_ready = bars + kSlots;          // [kSlots] MMA -> epilogue (commit)
    uint64_t* w_full = bars + 2 * kSlots;       // [kRing] weight copy landed
    uint64_t* w_empty = w_full + kRing;         // [kRing] both slots' MMAs on it done
    uint64_t* fin = w_empty + kRing;            // all MMAs of the issuer done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* bias_s = reinterpret_cast<float*>(smem + kOffBias);
    float* zr_s = reinterpret_cast<float*>(smem + kOffZr);
    float* wl_s = reinterpret_cast<float*>(smem + kOffWl);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.y;
    const bool decode = a.merge >= 0;

    for (int i = threadIdx.x; i < a.nL * 128; i += blockDim.x) bias_s[i] = a.bias[i];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        zr_s[i] = decode ? a.zr[(int64_t)r * 128 + i] : 0.0f;
        wl_s[i] = decode ? a.w_last[i] : 0.0f;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&a_ready[s], 128);
            mbar_init(&d_ready[s], 1);
        }
        for (int b = 0; b < kRing; ++b) {
            mbar_init(&w_full[b], 1);
            mbar_init(&w_empty[b], 1);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
    }
    if (warp == kEpiWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(uint32_t(kSlots * 128))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t tiles = (a.N + kRows - 1) / kRows;
    const int64_t groups = (tiles + kSlots - 1) / kSlots;
    // instruction descriptor: D FP32, A/B BF16, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                           ((uint32_t)(kRows >> 4) << 24);

    if (warp == kEpiWarps) {
        if (lane == 0) {  // ---- MMA issuer
            uint32_t g = 0, na[kSlots] = {};
            const uint32_t sA = smem_u32(smem + kOffA), sW = smem_u32(smem + kOffRing);
            for (int64_t gr = blockIdx.x; gr < groups && !*abort_flag; gr += gridDim.x) {
                const int64_t left = tiles - gr * kSlots;
                const int nslots = left < kSlots ? (int)left : kSlots;
                for (int j = 0; j < a.nL; ++j, ++g) {
                    const uint32_t b = g % kRing;
                    if (!wait_bounded(&w_full[b], (g / kRing) & 1u, abort_flag)) goto mma_done;
                    for (int s = 0; s < nslots; ++s) {
                        if (!wait_bounded(&a_ready[s], na[s] & 1u, abort_flag)) goto mma_done;
                        ++na[s];
                        tc_fence_after();
                        const uint32_t aa = sA + (uint32_t)s * kLayerBytes, ww = sW + b * kLayerBytes;
                        const uint32_t d = tmem + (uint32_t)(s * 128);
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const uint32_t at = (uint32_t)(kk >> 2) * kAtom;
                            tc_mma(d, desc_sw128(aa + at) + (uint64_t)((kk & 3) * 2),
                                   desc_sw128(ww + at) + (uint64_t)((kk & 3) * 2), idesc, kk > 0 ? 1u : 0u);
                        }
                        tc_commit(&d_ready[s]);
                    }
                    tc_commit(&w_empty[b]);
                }
            }
        mma_done:
            tc_commit(fin);  // completes when every MMA issued above has completed
            mbar_wait(fin, 0);
        }
    } else if (warp == kEpiWarps + 1) {
        if (lane == 0) {  // ---- weight producer
            uint32_t g = 0;
            unsigned char* ring = smem + kOffRing;
            for (int64_t gr = blockIdx.x; gr < groups && !*abort_flag; gr += gridDim.x) {
                for (int j = 0; j < a.nL; ++j, ++g) {
                    const uint32_t b = g % kRing;
                    if (!wait_bounded(&w_empty[b], ((g / kRing) & 1u) ^ 1u, abort_flag)) goto prod_done;
                    mbar_expect_tx(&w_full[b], kLayerBytes);
                    bulk_g2s(ring + b * kLayerBytes, a.wimg + (size_t)j * kLayerBytes, kLayerBytes, &w_full[b]);
                }
            }
        prod_done:
            if (*abort_flag)  // the copies still in flight land before the CTA exits
                for (uint32_t q = g > kRing ? g - kRing : 0; q < g; ++q) mbar_wait(&w_full[q % kRing], (q / kRing) & 1u);
        }
    } else {  // ---- embedding / epilogue: slot s, row i = TMEM lane i
        const int s = warp >> 2;
        const int i = (warp & 3) * 32 + lane;
        unsigned char* A = smem + kOffA + s * kLayerBytes;
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(s * 128);
        float* out = decode ? a.out + (int64_t)r * a.N : nullptr;
        const float b_last = decode ? *a.b_last : 0.0f;
        const int din = a.E.din;
        uint32_t nd = 0;
        for (int64_t t = (int64_t)blockIdx.x * kSlots + s; t < tiles; t += (int64_t)gridDim.x * kSlots) {
            const int64_t row = t * kRows + i;
            const bool valid = row < a.N;
            // rows past N process vertex 0 (harmless, never stored)
            const int64_t v = valid ? (a.vlist_n > 0 ? a.vlist[row] : row) : 0;
            if (a.lat_in) {  // cached query latent -> merge -> A
                const float4* src = reinterpret_cast<const float4*>(a.lat_in + v * 128);
#pragma unroll 4
                for (int c = 0; c < 16; ++c) {
                    const float4 x0 = __ldg(src + 2 * c), x1 = __ldg(src + 2 * c + 1);
                    const float* z = zr_s + 8 * c;
                    *reinterpret_cast<uint4*>(A + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) =
                        make_uint4(bf2(merge_f(a.merge, z[0], x0.x), merge_f(a.merge, z[1], x0.y)),
                                   bf2(merge_f(a.merge, z[2], x0.z), merge_f(a.merge, z[3], x0.w)),
                                   bf2(merge_f(a.merge, z[4], x1.x), merge_f(a.merge, z[5], x1.y)),
                                   bf2(merge_f(a.merge, z[6], x1.z), merge_f(a.merge, z[7], x1.w)));
                }
            } else {  // embedding (merged here when there is no encoder layer) -> A
                float p[3];
                vertex_position(v, a.X, a.Y, a.Z, p);
                const bool merge_here = decode && a.n_enc == 0;
                embed_point(a.E, a.tables, p, [&](int k, float x) {
                    put_bf16(A, i, k, merge_here ? merge_f(a.merge, zr_s[k], x) : x);
                });
                for (int k = din; k < ((din + 7) & ~7); ++k) put_bf16(A, i, k, 0.0f);
                for (int c = (din + 7) >> 3; c < 16; ++c)
                    *reinterpret_cast<uint4*>(A + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) = make_uint4(0, 0, 0, 0);
            }
            proxy_fence();
            tc_fence_before();
            arrive(&a_ready[s]);
            float acc_out = 0.0f;
            for (int j = 0; j < a.nL; ++j) {
                if (!wait_bounded(&d_ready[s], nd & 1u, abort_flag)) goto done;
                ++nd;
                tc_fence_after();
                const bool last = j == a.nL - 1, latent = j == a.n_enc - 1;
                const float* bj = bias_s + j * 128;
#pragma unroll
                for (int c0 = 0; c0 < 128; c0 += 32) {
                    float h[32];
                    tmem_ld32(taddr + (uint32_t)c0, h);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 b4 = *reinterpret_cast<const float4*>(bj + c0 + 4 * q);
                        h[4 * q] += b4.x;
                        h[4 * q + 1] += b4.y;
                        h[4 * q + 2] += b4.z;
                        h[4 * q + 3] += b4.w;
                    }
                    if (latent) {
                        if (!decode) {  // encode-only: the FP32 latent is the result
                            if (valid) {
                                float4* dst = reinterpret_cast<float4*>(a.lat + row * 128 + c0);
#pragma unroll
                                for (int q = 0; q < 8; ++q)
                                    dst[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
                            }
                            continue;
                        }
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) h[jj] = merge_f(a.merge, zr_s[c0 + jj], h[jj]);
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) h[jj] = act_tc<ACT>(h[jj]);
                    }
                    if (!last) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int c = (c0 >> 3) + q;
                            *reinterpret_cast<uint4*>(A + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) =
                                make_uint4(bf2(h[8 * q], h[8 * q + 1]), bf2(h[8 * q + 2], h[8 * q + 3]),
                                           bf2(h[8 * q + 4], h[8 * q + 5]), bf2(h[8 * q + 6], h[8 * q + 7]));
                        }
                    } else if (decode) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) acc_out = fmaf(wl_s[c0 + jj], h[jj], acc_out);
                    }
                }
                if (!last) {
                    proxy_fence();
                    tc_fence_before();
                    arrive(&a_ready[s]);
                }
            }
            if (decode && valid) out[row] = out_act(a.measure, acc_out + b_last);
        }
    }
done:
    if (*abort_flag && threadIdx.x == 0) report(a.status, kDevTimeout);
    tc_fence_before();
    __syncthreads();
    if (warp == kEpiWarps) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(uint32_t(kSlots * 128))
                     : "memory");
    }
}

// W (FP32 [out][in], in <= 128) of each listed layer -> its swizzled K-major
// BF16 image (zero-padded to 128 inputs), biases -> [layer][128]
__global__ void hash_tc_pack_kernel(const float* __restrict__ params, HashTcPack pk,
                                    unsigned char* __restrict__ wimg, float* __restrict__ bias) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)pk.n * 128 * 128) return;
    const int j = (int)(idx >> 14), o = (int)((idx >> 7) & 127), k = (int)(idx & 127);
    const float w = k < pk.cin[j] ? params[pk.w[j] + (int64_t)o * pk.cin[j] + k] : 0.0f;
    unsigned char* img = wimg + (size_t)j * kLayerBytes;
    *reinterpret_cast<__nv_bfloat16*>(img + (uint32_t)(k >> 6) * kAtom + swz(o, (k >> 3) & 7) +
                                      (uint32_t)(k & 7) * 2) = __float2bfloat16_rn(w);
    if (k == 0) bias[(int64_t)j * 128 + o] = params[pk.b[j] + o];
}

// the FP32 embeddings of listed vertices, zero-padded to 128 (the reference
// latents of a network without encoder layers)
__global__ void hash_tc_embed_refs_kernel(HashTcArgs a, float* __restrict__ zr) {
    const int r = blockIdx.x;
    if (threadIdx.x != 0 || r >= a.vlist_n) return;
    float p[3];
    vertex_position(a.vlist[r], a.X, a.Y, a.Z, p);
    float* z = zr + (int64_t)r * 128;
    for (int k = 0; k < 128; ++k) z[k] = 0.0f;
    embed_point(a.E, a.tables, p, [&](int k, float x) { z[k] = x; });
}

size_t hash_tc_layer_bytes() { return kLayerBytes; }

cudaError_t launch_hash_tc_pack(const float* params, const HashTcPack& pk, unsigned char* wimg,
                                float* bias, cudaStream_t st) {
    const int64_t n = (int64_t)pk.n * 128 * 128;
    if (n == 0) return cudaSuccess;
    hash_tc_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(params, pk, wimg, bias);
    return cudaGetLastError();
}

cudaError_t launch_hash_tc_embed_refs(const HashTcArgs& a, float* zr, cudaStream_t st) {
    hash_tc_embed_refs_kernel<<<a.vlist_n, 32, 0, st>>>(a, zr);
    return cudaGetLastError();
}

cudaError_t launch_hash_tc(const HashTcArgs& a, int act, int ctas_x, int R, cudaStream_t st) {
    static bool attr[3] = {false, false, false};
    if (act < 0 || act > 2 || a.nL < 1 || a.nL > kHashTcMaxLayers || R < 1) return cudaErrorInvalidValue;
    auto kern = act == 0 ? hash_tc_kernel<0> : (act == 1 ? hash_tc_kernel<1> : hash_tc_kernel<2>);
    if (!attr[act]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) return e;
        attr[act] = true;
    }
    kern<<<dim3(ctas_x, R), kThreads, kSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ndf

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
//   warps 0-7 / 8-15: two tile slots.  Row i of a slot's tile (TMEM lane i) belongs
//     to two warps: warp q + 4 h of the slot (q = i / 32) owns its columns
//     64 h .. 64 h + 63.  Half 0 writes the position and Fourier features of the
//     row's vertex into the slot's A tile (BF16, 128-byte-swizzled K-major), half 1
//     the hash-grid features; after each layer each half reads its 64 accumulator
//     columns with tcgen05.ld, adds the bias, applies the activation (or the
//     merge) with packed FP32x2 arithmetic and writes them back as the next
//     layer's A operand.  The output layer's two half dot products meet through
//     shared memory (an mbarrier per slot).
//   warp 16: allocates TMEM (2 x 128 columns); one lane issues the MMAs, layer by
//     layer for both slots, and commits to the slot's mbarrier and, once both
//     slots used a weight buffer, to that buffer's "empty" mbarrier.
//   warp 17: one lane streams the layers' weight images (32 KB each, pre-swizzled
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
constexpr int kSlots = 4;
constexpr int kRing = 2;
constexpr int kHalves = 1;                   // warps per TMEM lane quarter of a slot
constexpr int kSlotWarps = 4 * kHalves;
constexpr int kSlotThreads = 32 * kSlotWarps;
constexpr int kCols = 128 / kHalves;         // accumulator columns per warp
constexpr int kEpiWarps = kSlotWarps * kSlots;
constexpr int kThreads = 32 * (kEpiWarps + 2);
constexpr uint32_t kLayerBytes = 2 * kAtom;  // 128 x 128 BF16 = two K atoms
constexpr uint32_t kOffRing = 0;
constexpr uint32_t kOffA = kRing * kLayerBytes;
constexpr uint32_t kOffBias = kOffA + kSlots * kLayerBytes;
constexpr uint32_t kOffZr = kOffBias + kHashTcMaxLayers * 128 * 4;
constexpr uint32_t kOffWl = kOffZr + 128 * 4;
constexpr uint32_t kOffPart = kOffWl + 128 * 4;  // [kSlots][128] half-1 output partials
constexpr uint32_t kOffBar = kOffPart + kSlots * 128 * 4;
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

// hidden-layer activation of two values; the sine of the Snake family through
// the SFU, the rest as packed FP32x2 (each lane rounds like its scalar form)
template <int ACT>
__device__ __forceinline__ float2 act2(float2 x) {
    if constexpr (ACT == NDF_ACT_RELU) {
        return make_float2(fmaxf(x.x, 0.0f), fmaxf(x.y, 0.0f));
    } else {
        const float2 s = make_float2(__sinf(x.x), __sinf(x.y));
        const float2 lin = ACT == NDF_ACT_SNAKE ? x : __fmul2_rn(x, make_float2(0.5f, 0.5f));
        return __ffma2_rn(s, s, lin);
    }
}

__device__ __forceinline__ float2 merge2(int mode, float2 zr, float2 zq) {
    if (mode == NDF_MERGE_PRODUCT) return __fmul2_rn(zr, zq);
    if (mode == NDF_MERGE_SUM) return __fadd2_rn(zr, zq);
    return make_float2(fabsf(zr.x - zq.x), fabsf(zr.y - zq.y));
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
    uint64_t* part_ready = fin + 1;             // [kSlots] half-1 output partials written
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(part_ready + kSlots);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* bias_s = reinterpret_cast<float*>(smem + kOffBias);
    float* zr_s = reinterpret_cast<float*>(smem + kOffZr);
    float* wl_s = reinterpret_cast<float*>(smem + kOffWl);
    float* part_s = reinterpret_cast<float*>(smem + kOffPart);
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
            mbar_init(&a_ready[s], kSlotThreads);
            mbar_init(&d_ready[s], 1);
            mbar_init(&part_ready[s], 128);
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
    } else {  // ---- embedding / epilogue: slot s, row i = TMEM lane i, columns of half h
        const int s = warp / kSlotWarps, wl = warp % kSlotWarps;
        const int q = wl & 3, h = wl >> 2;
        const int i = q * 32 + lane;
        const int col0 = h * kCols;
        unsigned char* A = smem + kOffA + s * kLayerBytes;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(s * 128);
        float* out = decode ? a.out + (int64_t)r * a.N : nullptr;
        const float b_last = decode ? *a.b_last : 0.0f;
        const int din = a.E.din;
        uint32_t nd = 0, np = 0;
        for (int64_t t = (int64_t)blockIdx.x * kSlots + s; t < tiles; t += (int64_t)gridDim.x * kSlots) {
            const int64_t row = t * kRows + i;
            const bool valid = row < a.N;
            // rows past N process vertex 0 (harmless, never stored)
            const int64_t v = valid ? (a.vlist_n > 0 ? a.vlist[row] : row) : 0;
            if (a.lat_in) {  // cached query latent (this half's 64 columns) -> merge -> A
                const float4* src = reinterpret_cast<const float4*>(a.lat_in + v * 128 + col0);
                const float4* zr4 = reinterpret_cast<const float4*>(zr_s + col0);
#pragma unroll 2
                for (int c = 0; c < kCols / 8; ++c) {
                    const float4 x0 = __ldg(src + 2 * c), x1 = __ldg(src + 2 * c + 1);
                    const float4 z0 = zr4[2 * c], z1 = zr4[2 * c + 1];
                    const float2 m0 = merge2(a.merge, make_float2(z0.x, z0.y), make_float2(x0.x, x0.y));
                    const float2 m1 = merge2(a.merge, make_float2(z0.z, z0.w), make_float2(x0.z, x0.w));
                    const float2 m2 = merge2(a.merge, make_float2(z1.x, z1.y), make_float2(x1.x, x1.y));
                    const float2 m3 = merge2(a.merge, make_float2(z1.z, z1.w), make_float2(x1.z, x1.w));
                    const int cc = (col0 >> 3) + c;
                    *reinterpret_cast<uint4*>(A + (uint32_t)(cc >> 3) * kAtom + swz(i, cc & 7)) =
                        make_uint4(bf2(m0.x, m0.y), bf2(m1.x, m1.y), bf2(m2.x, m2.y), bf2(m3.x, m3.y));
                }
            } else {  // embedding (merged here when there is no encoder layer) -> A
                // operand columns: Fourier blocks of the three axes (from the per-axis
                // tables), then p and the grid features from kt on (hash_tc_emb_source)
                const bool merge_here = decode && a.n_enc == 0;
                const int kt = 3 * a.f8, lh = a.E.levels / 2, ngrid = a.E.levels * a.E.F;
                float p[3];
                vertex_position(v, a.X, a.Y, a.Z, p);
                auto put = [&](int k, float x) {
                    put_bf16(A, i, k, merge_here ? merge_f(a.merge, zr_s[k], x) : x);
                };
                if (h == 0 || kHalves == 1) {
                    const int64_t coord[3] = {v % a.X, (v / a.X) % a.Y, v / (a.X * a.Y)};
                    for (int j = 0; j < 3; ++j) {
                        const float4* row = reinterpret_cast<const float4*>(a.ftab + a.foff[j] + coord[j] * a.f8);
                        for (int c = 0; c < a.f8 / 8; ++c) {
                            float4 x0 = __ldg(row + 2 * c), x1 = __ldg(row + 2 * c + 1);
                            const int k0 = j * a.f8 + 8 * c;
                            if (merge_here) {
                                const float* z = zr_s + k0;
                                x0 = make_float4(merge_f(a.merge, z[0], x0.x), merge_f(a.merge, z[1], x0.y),
                                                 merge_f(a.merge, z[2], x0.z), merge_f(a.merge, z[3], x0.w));
                                x1 = make_float4(merge_f(a.merge, z[4], x1.x), merge_f(a.merge, z[5], x1.y),
                                                 merge_f(a.merge, z[6], x1.z), merge_f(a.merge, z[7], x1.w));
                            }
                            const int cc = k0 >> 3;
                            *reinterpret_cast<uint4*>(A + (uint32_t)(cc >> 3) * kAtom + swz(i, cc & 7)) =
                                make_uint4(bf2(x0.x, x0.y), bf2(x0.z, x0.w), bf2(x1.x, x1.y), bf2(x1.z, x1.w));
                        }
                    }
                    put(kt, p[0]);
                    put(kt + 1, p[1]);
                    put(kt + 2, p[2]);
                    embed_levels(a.E, a.tables, p, 0, kHalves == 1 ? a.E.levels : lh,
                                 [&](int g, float x) { put(kt + 3 + g, x); });
                }
                if (h == 1 || kHalves == 1) {
                    if (kHalves > 1)
                        embed_levels(a.E, a.tables, p, lh, a.E.levels, [&](int g, float x) { put(kt + 3 + g, x); });
                    const int kend = kt + 3 + ngrid;
                    for (int k = kend; k < ((kend + 7) & ~7); ++k) put_bf16(A, i, k, 0.0f);
                    for (int c = (kend + 7) >> 3; c < 16; ++c)
                        *reinterpret_cast<uint4*>(A + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) =
                            make_uint4(0, 0, 0, 0);
                }
            }
            proxy_fence();
            tc_fence_before();
            arrive(&a_ready[s]);
            float2 acc2 = make_float2(0.0f, 0.0f);
            for (int j = 0; j < a.nL; ++j) {
                if (!wait_bounded(&d_ready[s], nd & 1u, abort_flag)) goto done;
                ++nd;
                tc_fence_after();
                const bool last = j == a.nL - 1, latent = j == a.n_enc - 1;
                const float* bj = bias_s + j * 128;
#pragma unroll
                for (int c0 = 0; c0 < kCols; c0 += 32) {
                    const int cg = col0 + c0;  // accumulator column of hv[0]
                    float hv[32];
                    tmem_ld32(taddr + (uint32_t)cg, hv);
                    float2* h2 = reinterpret_cast<float2*>(hv);
                    const float4* b4 = reinterpret_cast<const float4*>(bj + cg);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const float4 bb = b4[u];
                        h2[2 * u] = __fadd2_rn(h2[2 * u], make_float2(bb.x, bb.y));
                        h2[2 * u + 1] = __fadd2_rn(h2[2 * u + 1], make_float2(bb.z, bb.w));
                    }
                    if (latent) {
                        if (!decode) {  // encode-only: the FP32 latent is the result
                            if (valid) {
                                float4* dst = reinterpret_cast<float4*>(a.lat + row * 128 + cg);
#pragma unroll
                                for (int u = 0; u < 8; ++u)
                                    dst[u] = make_float4(hv[4 * u], hv[4 * u + 1], hv[4 * u + 2], hv[4 * u + 3]);
                            }
                            continue;
                        }
                        const float4* z4 = reinterpret_cast<const float4*>(zr_s + cg);
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float4 zz = z4[u];
                            h2[2 * u] = merge2(a.merge, make_float2(zz.x, zz.y), h2[2 * u]);
                            h2[2 * u + 1] = merge2(a.merge, make_float2(zz.z, zz.w), h2[2 * u + 1]);
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < 16; ++u) h2[u] = act2<ACT>(h2[u]);
                    }
                    if (!last) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int c = (cg >> 3) + u;
                            *reinterpret_cast<uint4*>(A + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) =
                                make_uint4(bf2(hv[8 * u], hv[8 * u + 1]), bf2(hv[8 * u + 2], hv[8 * u + 3]),
                                           bf2(hv[8 * u + 4], hv[8 * u + 5]), bf2(hv[8 * u + 6], hv[8 * u + 7]));
                        }
                    } else if (decode) {
                        const float4* w4 = reinterpret_cast<const float4*>(wl_s + cg);
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float4 ww = w4[u];
                            acc2 = __ffma2_rn(make_float2(ww.x, ww.y), h2[2 * u], acc2);
                            acc2 = __ffma2_rn(make_float2(ww.z, ww.w), h2[2 * u + 1], acc2);
                        }
                    }
                }
                if (!last) {
                    proxy_fence();
                    tc_fence_before();
                    arrive(&a_ready[s]);
                }
            }
            if (decode && kHalves == 1) {
                if (valid) out[row] = out_act(a.measure, (acc2.x + acc2.y) + b_last);
            } else if (decode) {  // the two halves' dot products meet in shared memory
                if (h == 1) {
                    part_s[s * 128 + i] = acc2.x + acc2.y;
                    arrive(&part_ready[s]);
                } else {
                    if (!wait_bounded(&part_ready[s], np & 1u, abort_flag)) goto done;
                    ++np;
                    const float o = (acc2.x + acc2.y) + part_s[s * 128 + i];
                    if (valid) out[row] = out_act(a.measure, o + b_last);
                }
            }
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
// BF16 image (zero-padded to 128 inputs; the input columns of a layer that reads
// the embedding in operand order), biases -> [layer][128]
__global__ void hash_tc_pack_kernel(const float* __restrict__ params, HashTcPack pk,
                                    unsigned char* __restrict__ wimg, float* __restrict__ bias) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)pk.n * 128 * 128) return;
    const int j = (int)(idx >> 14), o = (int)((idx >> 7) & 127), k = (int)(idx & 127);
    const int src = pk.perm[j] ? hash_tc_emb_source(k, pk.L, pk.f8, pk.ngrid) : k;
    const float w = src >= 0 && src < pk.cin[j] ? params[pk.w[j] + (int64_t)o * pk.cin[j] + src] : 0.0f;
    unsigned char* img = wimg + (size_t)j * kLayerBytes;
    *reinterpret_cast<__nv_bfloat16*>(img + (uint32_t)(k >> 6) * kAtom + swz(o, (k >> 3) & 7) +
                                      (uint32_t)(k & 7) * 2) = __float2bfloat16_rn(w);
    if (k == 0) bias[(int64_t)j * 128 + o] = params[pk.b[j] + o];
}

// the FP32 embeddings of listed vertices in operand column order, zero-padded to
// 128 (the reference latents of a network without encoder layers)
__global__ void hash_tc_embed_refs_kernel(HashTcArgs a, float* __restrict__ zr) {
    const int r = blockIdx.x;
    if (threadIdx.x != 0 || r >= a.vlist_n) return;
    float p[3], x[128];
    vertex_position(a.vlist[r], a.X, a.Y, a.Z, p);
    embed_point(a.E, a.tables, p, [&](int k, float v) { x[k] = v; });
    float* z = zr + (int64_t)r * 128;
    for (int k = 0; k < 128; ++k) {
        const int src = hash_tc_emb_source(k, a.E.L, a.f8, a.E.levels * a.E.F);
        z[k] = src >= 0 ? x[src] : 0.0f;
    }
}

__global__ void hash_tc_ftab_kernel(int L, int f8, int64_t X, int64_t Y, int64_t Z, float* __restrict__ ftab) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (X + Y + Z) * f8) return;
    const int64_t n_all = idx / f8;
    const int q = (int)(idx - n_all * f8);
    const int j = n_all < X ? 0 : (n_all < X + Y ? 1 : 2);
    const int64_t n = n_all - (j == 0 ? 0 : (j == 1 ? X : X + Y));
    const int64_t D = j == 0 ? X : (j == 1 ? Y : Z);
    // the axis coordinate exactly as vertex_position computes it
    const float pj = D > 1 ? -1.0f + 2.0f * (float)n / (float)(D - 1) : 0.0f;
    float val = 0.0f;
    if (q < 2 * L) {
        float sv, cv;
        sincospif(ldexpf(pj, q >> 1), &sv, &cv);
        val = (q & 1) ? cv : sv;
    }
    ftab[idx] = val;
}

size_t hash_tc_layer_bytes() { return kLayerBytes; }

cudaError_t launch_hash_tc_pack(const float* params, const HashTcPack& pk, unsigned char* wimg,
                                float* bias, cudaStream_t st) {
    const int64_t n = (int64_t)pk.n * 128 * 128;
    if (n == 0) return cudaSuccess;
    hash_tc_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(params, pk, wimg, bias);
    return cudaGetLastError();
}

cudaError_t launch_hash_tc_ftab(int L, int f8, int64_t X, int64_t Y, int64_t Z, float* ftab,
                                cudaStream_t st) {
    const int64_t n = (X + Y + Z) * f8;
    if (n == 0) return cudaSuccess;
    hash_tc_ftab_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L, f8, X, Y, Z, ftab);
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
    const int64_t groups = ((a.N + kRows - 1) / kRows + kSlots - 1) / kSlots;  // tile groups of a CTA
    if (ctas_x > groups) ctas_x = (int)groups;
    if (ctas_x < 1) ctas_x = 1;
    kern<<<dim3(ctas_x, R), kThreads, kSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ndf

// Neural dependence field volume decoding (Sec. 5) on the 5th-generation tensor
// cores.
//
// For one reference, every query vertex v needs
//   h1 = ReLU(W1f f(v) + b1f)         (first layer with the reference folded in)
//   h2 = ReLU(W2 h1 + b2), h3 = ReLU(W3 h2 + b3), y = act(w4 . h3 + b4).
// A CTA decodes 128-vertex tiles (the MMA M dimension) in two slots so that the
// encoding / epilogue work of one tile overlaps the MMAs of the other:
//   warps 0-3 (slot 0) and 4-7 (slot 1): thread i of a slot owns row i of the tile
//     and TMEM lane i.  It gathers and interpolates its vertex's 64 grid features
//     and writes them as BF16 into the slot's A tile in the 128-byte-swizzled
//     K-major layout the MMA reads; after each layer it loads its row of the FP32
//     accumulator with tcgen05.ld, adds the bias, applies ReLU and writes the next
//     layer's A tile (or, after layer 3, the output).
//   warp 8: allocates TMEM (2 slots x 128 columns); one lane issues tcgen05.mma
//     (M = 128, N = 128, K = 64 / 128 / 128) for whichever slot is ready and
//     commits to that slot's mbarrier.
// Weights (folded W1 of the reference, W2, W3) sit in shared memory in the same
// swizzled K-major layout for the whole launch.
#include <cuda_bf16.h>

#include "ndf_net.h"
#include "tc_common.cuh"

namespace ndf {

namespace {

using namespace tc;

constexpr int kTile = 128;
constexpr int kTcThreads = 288;  // 8 epilogue warps + 1 MMA warp

struct TcGrid {
    const __nv_bfloat16* grid;
    int res[kLevels];
    int64_t off[kLevels];
};

// interpolated 16 features of one level at p (corner-aligned grid on [-1,1]^3)
__device__ __forceinline__ void encode_level(const TcGrid& G, int l, const float* p, float (&o)[kFeat]) {
    const int R = G.res[l];
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
    for (int q = 0; q < kFeat; ++q) o[q] = 0.0f;
    const uint4* base = reinterpret_cast<const uint4*>(G.grid + G.off[l]);
    uint4 g[8][2];
#pragma unroll
    for (int c = 0; c < 8; ++c) {  // all 16 loads first, then the weighted sums
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const int64_t idx = ((int64_t)(i[2] + dz) * R + (i[1] + dy)) * R + (i[0] + dx);
        g[c][0] = __ldg(base + idx * 2);
        g[c][1] = __ldg(base + idx * 2 + 1);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const float w = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
        const uint32_t uu[8] = {g[c][0].x, g[c][0].y, g[c][0].z, g[c][0].w,
                                g[c][1].x, g[c][1].y, g[c][1].z, g[c][1].w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 v = unbf2(uu[j]);
            o[2 * j] = fmaf(w, v.x, o[2 * j]);
            o[2 * j + 1] = fmaf(w, v.y, o[2 * j + 1]);
        }
    }
}

__device__ __forceinline__ float pos_axis(int64_t i, int64_t n) {
    return n > 1 ? -1.0f + 2.0f * (float)i / (float)(n - 1) : 0.0f;
}

}  // namespace

struct TcInferArgs {
    TcGrid G;
    const __nv_bfloat16* w1f;  // [R][128][64] folded first layer per reference
    const float* b1f;          // [R][128]
    const __nv_bfloat16* w2;   // [128][128] ([out][in])
    const __nv_bfloat16* w3;
    const float* params;
    int64_t offb2, offb3, offw4, offb4;
    int64_t N, X, Y, Z;
    int measure;
    float* out;                // [R][N]
    unsigned* status;
};

// shared memory: W1f (1 atom), W2 (2 atoms), W3 (2 atoms), per slot A1 (1 atom) + A23 (2 atoms)
constexpr uint32_t kOffW1 = 0, kOffW2 = kAtom, kOffW3 = 3 * kAtom, kOffSlot = 5 * kAtom;
constexpr uint32_t kSlotBytes = 3 * kAtom;
constexpr uint32_t kTcSmem = 5 * kAtom + 2 * kSlotBytes + 1024 /*align*/ + 256 /*barriers*/;

__global__ void __launch_bounds__(kTcThreads, 1) infer_tc_kernel(const TcInferArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 5 * kAtom + 2 * kSlotBytes);
    uint64_t* a_ready = bars;      // [2] epilogue -> MMA (128 arrivals)
    uint64_t* d_ready = bars + 2;  // [2] MMA -> epilogue (commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.y;

    // ---- weights into the swizzled K-major layout (rows = output features)
    {
        const __nv_bfloat16* w1 = a.w1f + (int64_t)r * kHid * kLF;
        for (int i = threadIdx.x; i < kHid * 8; i += blockDim.x) {  // W1f: 128 rows x 8 chunks
            const int row = i >> 3, c = i & 7;
            *reinterpret_cast<uint4*>(smem + kOffW1 + swz(row, c)) =
                reinterpret_cast<const uint4*>(w1 + row * kLF)[c];
        }
        for (int i = threadIdx.x; i < kHid * 16; i += blockDim.x) {  // W2, W3: 2 atoms each
            const int row = i >> 4, c = i & 15;
            const uint32_t o = (uint32_t)(c >> 3) * kAtom + swz(row, c & 7);
            *reinterpret_cast<uint4*>(smem + kOffW2 + o) = reinterpret_cast<const uint4*>(a.w2 + row * kHid)[c];
            *reinterpret_cast<uint4*>(smem + kOffW3 + o) = reinterpret_cast<const uint4*>(a.w3 + row * kHid)[c];
        }
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&a_ready[s], 128);
            mbar_init(&d_ready[s], 1);
        }
        *abort_flag = 0;
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    proxy_fence();  // weights written by threads are read by the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t tiles = (a.N + kTile - 1) / kTile;
    const int64_t step = (int64_t)gridDim.x * 2;
    // instruction descriptor: D FP32, A/B BF16, K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) |
                           ((uint32_t)(kTile >> 4) << 24);

    if (warp == 8) {
        if (lane == 0) {  // ---- MMA issuer: serve whichever slot is ready
            int64_t tile[2] = {(int64_t)blockIdx.x * 2, (int64_t)blockIdx.x * 2 + 1};
            int layer[2] = {0, 0};
            uint32_t na[2] = {0, 0};
            const uint32_t sw1 = smem_u32(smem + kOffW1), sw2 = smem_u32(smem + kOffW2),
                           sw3 = smem_u32(smem + kOffW3);
            uint32_t polls = 0;
            uint64_t t0 = 0;
            while ((tile[0] < tiles || tile[1] < tiles) && !*abort_flag) {
                bool progressed = false;
                for (int s = 0; s < 2; ++s) {
                    if (tile[s] >= tiles || !try_wait(&a_ready[s], na[s] & 1u)) continue;
                    progressed = true;
                    ++na[s];
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + kOffSlot + s * kSlotBytes);
                    const uint32_t d = tmem + (uint32_t)(s * 128);
                    if (layer[s] == 0) {  // K = 64: one atom, 4 steps of 16
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            tc_mma(d, desc_sw128(sa) + (uint64_t)(kk * 2), desc_sw128(sw1) + (uint64_t)(kk * 2),
                                   idesc, kk > 0 ? 1u : 0u);
                    } else {  // K = 128: two atoms of A23 against W2 / W3
                        const uint32_t a23 = sa + kAtom, w = layer[s] == 1 ? sw2 : sw3;
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const uint32_t at = (uint32_t)(kk >> 2) * kAtom;
                            tc_mma(d, desc_sw128(a23 + at) + (uint64_t)((kk & 3) * 2),
                                   desc_sw128(w + at) + (uint64_t)((kk & 3) * 2), idesc, kk > 0 ? 1u : 0u);
                        }
                    }
                    tc_commit(&d_ready[s]);
                    if (++layer[s] == 3) {
                        layer[s] = 0;
                        tile[s] += step;
                    }
                }
                if (progressed) {
                    polls = 0;
                    t0 = 0;
                } else if (++polls > kWaitPolls) {
                    *abort_flag = 1;
                } else if ((polls & 1023u) == 0u) {  // and at most kWaitNs of wall time
                    const uint64_t t = global_ns();
                    if (t0 == 0) t0 = t;
                    else if (t - t0 > kWaitNs) *abort_flag = 1;
                }
            }
        }
    } else {  // ---- encode / epilogue: slot s, row i = TMEM lane i
        const int s = warp >> 2;
        const int i = (warp & 3) * 32 + lane;
        unsigned char* A1 = smem + kOffSlot + s * kSlotBytes;
        unsigned char* A23 = A1 + kAtom;
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(s * 128);
        const float* b1 = a.b1f + (int64_t)r * kHid;
        const float* b2 = a.params + a.offb2;
        const float* b3 = a.params + a.offb3;
        const float* w4 = a.params + a.offw4;
        const float b4 = a.params[a.offb4];
        float* out = a.out + (int64_t)r * a.N;
        uint32_t nd = 0;
        for (int64_t t = (int64_t)blockIdx.x * 2 + s; t < tiles; t += step) {
            const int64_t v = t * kTile + i;
            // encode this row's vertex into A1 (rows past N encode position 0: harmless, unused)
            float p[3];
            {
                const int64_t vv = v < a.N ? v : 0;
                const int64_t x = vv % a.X, y = (vv / a.X) % a.Y, z = vv / (a.X * a.Y);
                p[0] = pos_axis(x, a.X);
                p[1] = pos_axis(y, a.Y);
                p[2] = pos_axis(z, a.Z);
            }
#pragma unroll
            for (int l = 0; l < kLevels; ++l) {
                float f[kFeat];
                encode_level(a.G, l, p, f);
                *reinterpret_cast<uint4*>(A1 + swz(i, 2 * l)) =
                    make_uint4(bf2(f[0], f[1]), bf2(f[2], f[3]), bf2(f[4], f[5]), bf2(f[6], f[7]));
                *reinterpret_cast<uint4*>(A1 + swz(i, 2 * l + 1)) =
                    make_uint4(bf2(f[8], f[9]), bf2(f[10], f[11]), bf2(f[12], f[13]), bf2(f[14], f[15]));
            }
            proxy_fence();
            tc_fence_before();
            arrive(&a_ready[s]);
            for (int layer = 0; layer < 3; ++layer) {
                if (!wait_bounded(&d_ready[s], nd & 1u, abort_flag)) goto done;
                ++nd;
                tc_fence_after();
                const float* bias = layer == 0 ? b1 : (layer == 1 ? b2 : b3);
                float acc = 0.0f;
#pragma unroll
                for (int c0 = 0; c0 < kHid; c0 += 32) {
                    float h[32];
                    tmem_ld32(taddr + (uint32_t)c0, h);
#pragma unroll
                    for (int j = 0; j < 32; ++j) h[j] = fmaxf(h[j] + bias[c0 + j], 0.0f);
                    if (layer < 2) {  // next layer's A: columns c0..c0+31 = chunks c0/8 ..
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int c = (c0 >> 3) + q;  // 16-byte chunk of the 256-byte row
                            *reinterpret_cast<uint4*>(A23 + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) =
                                make_uint4(bf2(h[8 * q], h[8 * q + 1]), bf2(h[8 * q + 2], h[8 * q + 3]),
                                           bf2(h[8 * q + 4], h[8 * q + 5]), bf2(h[8 * q + 6], h[8 * q + 7]));
                        }
                    } else {  // output layer on the BF16-rounded h3
#pragma unroll
                        for (int j = 0; j < 32; j += 2) {
                            const float2 hv = unbf2(bf2(h[j], h[j + 1]));
                            acc = fmaf(w4[c0 + j], hv.x, fmaf(w4[c0 + j + 1], hv.y, acc));
                        }
                    }
                }
                if (layer < 2) {
                    proxy_fence();
                    tc_fence_before();
                    arrive(&a_ready[s]);
                } else {
                    const float o = acc + b4;
                    if (v < a.N) out[v] = a.measure == 0 ? tanhf(o) : (o > 20.f ? o : log1pf(expf(o)));
                }
            }
        }
    }
done:
    if (*abort_flag && threadIdx.x == 0) report(a.status, kDevTimeout);
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                     : "memory");
    }
}

cudaError_t launch_infer_tc(ndf_model* m, int R, float* out) {
    ndf_ctx* ctx = m->ctx;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTcSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    TcInferArgs a;
    a.G.grid = m->grid_bf;
    for (int l = 0; l < kLevels; ++l) {
        a.G.res[l] = m->L.res[l];
        a.G.off[l] = m->L.grid_off[l];
    }
    a.w1f = m->w1f;
    a.b1f = m->b1f;
    a.w2 = m->wbf + (size_t)kHid * kHid;
    a.w3 = m->wbf + (size_t)2 * kHid * kHid;
    a.params = m->params;
    a.offb2 = m->L.b2;
    a.offb3 = m->L.b3;
    a.offw4 = m->L.w4;
    a.offb4 = m->L.b4;
    a.N = m->X * m->Y * m->Z;
    a.X = m->X;
    a.Y = m->Y;
    a.Z = m->Z;
    a.measure = m->measure;
    a.out = out;
    a.status = ctx->flag.as<unsigned>() + 1;
    const int64_t tiles = (a.N + kTile - 1) / kTile;
    int per_ref = (ctx->sm_count + R - 1) / R;
    const int64_t need = (tiles + 1) / 2;
    if (per_ref > need) per_ref = (int)need;
    if (per_ref < 1) per_ref = 1;
    infer_tc_kernel<<<dim3(per_ref, R), kTcThreads, kTcSmem, ctx->stream>>>(a);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace ndf

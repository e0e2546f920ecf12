// Neural dependence field volume decoding (Sec. 5) on the 5th-generation tensor
// cores, R references per launch.
//
// For reference r and query vertex v the network computes
//   x  = [f(p_r) * f(v) ; f(p_r) + f(v)]          (the merge, rounded to BF16)
//   h1 = ReLU(W1 x + b1), h2 = ReLU(W2 h1 + b2), h3 = ReLU(W3 h2 + b3),
//   y  = act(w4 . h3 + b4)
// -- the arithmetic of the training forward.  The reference enters only through
// the layer-1 operand x, so W1, W2 and W3 are the same for every reference and
// stay in shared memory for the launch, and the query encoding f(v) (the grid
// gathers, most of a vertex's cost) is computed once per vertex for all R
// references of the launch.
//
// A persistent CTA per SM decodes 128-vertex tiles (the MMA M dimension) in two
// slots so that one slot's epilogue overlaps the other slot's MMAs:
//   warps 0-3 (slot 0) and 4-7 (slot 1): thread i of a slot owns row i of the tile
//     and TMEM lane i.  It encodes its vertex once per tile (64 FP32 features kept
//     in registers); then for each reference it writes x into the slot's A operand
//     (BF16, 128-byte-swizzled K-major), and after each layer loads its row of the
//     FP32 accumulator with tcgen05.ld, adds the bias, applies ReLU and writes the
//     next layer's operand over the same buffer (the MMA that read it has
//     completed), or after layer 3 the output.
//   warp 8: allocates TMEM (2 slots x 128 columns); one lane issues tcgen05.mma
//     (M = 128, N = 128, K = 128) for whichever slot is ready and commits to that
//     slot's mbarrier.
// The references' features f(p_r) (FP32) and the biases sit in shared memory.
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
    const int64_t* refs;       // [R] reference vertices
    int R;
    const __nv_bfloat16* w;    // [3][128][128] W1..W3 ([out][in])
    const float* params;
    int64_t offb1, offb2, offb3, offw4, offb4;
    int64_t N, X, Y, Z;
    int measure;
    float* out;                // [R][N]
    unsigned* status;
};

// shared memory: W1, W2, W3 (2 atoms each), one 2-atom operand buffer per slot,
// then biases / output weights (4 x 128 FP32), the references' features [R][64]
// FP32 and the barriers
constexpr int kMaxRefsPerLaunch = 64;
constexpr uint32_t kOffW = 0, kOffSlot = 6 * kAtom, kSlotBytes = 2 * kAtom;
constexpr uint32_t kOffVec = kOffSlot + 2 * kSlotBytes;
constexpr uint32_t kOffFr = kOffVec + 4 * kHid * 4;
constexpr uint32_t kOffBar = kOffFr + kMaxRefsPerLaunch * kLF * 4;
constexpr uint32_t kTcSmem = kOffBar + 256 /*barriers*/ + 1024 /*align*/;

__global__ void __launch_bounds__(kTcThreads, 1) infer_tc_kernel(const TcInferArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* vec = reinterpret_cast<float*>(smem + kOffVec);  // b1, b2, b3, w4
    float* fr_all = reinterpret_cast<float*>(smem + kOffFr);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
    uint64_t* a_ready = bars;      // [2] epilogue -> MMA (128 arrivals)
    uint64_t* d_ready = bars + 2;  // [2] MMA -> epilogue (commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = a.R;

    // ---- weights into the swizzled K-major layout (rows = output features),
    // biases and output weights, the references' features
    for (int i = threadIdx.x; i < 3 * kHid * 16; i += blockDim.x) {  // 3 layers x 128 rows x 16 chunks
        const int l = i / (kHid * 16), row = (i >> 4) % kHid, c = i & 15;
        const uint32_t o = (uint32_t)(2 * l + (c >> 3)) * kAtom + swz(row, c & 7);
        *reinterpret_cast<uint4*>(smem + kOffW + o) =
            reinterpret_cast<const uint4*>(a.w + ((size_t)l * kHid + row) * kHid)[c];
    }
    for (int i = threadIdx.x; i < 4 * kHid; i += blockDim.x) {
        const int64_t off = i < kHid ? a.offb1 : i < 2 * kHid ? a.offb2 : i < 3 * kHid ? a.offb3 : a.offw4;
        vec[i] = a.params[off + (i % kHid)];
    }
    for (int i = threadIdx.x; i < R * kLevels; i += blockDim.x) {
        const int64_t v = a.refs[i / kLevels];
        const int64_t x = v % a.X, y = (v / a.X) % a.Y, z = v / (a.X * a.Y);
        const float p[3] = {pos_axis(x, a.X), pos_axis(y, a.Y), pos_axis(z, a.Z)};
        float f[kFeat];
        encode_level(a.G, i % kLevels, p, f);
#pragma unroll
        for (int q = 0; q < kFeat; ++q) fr_all[(i / kLevels) * kLF + (i % kLevels) * kFeat + q] = f[q];
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
            // operands per slot: (its tiles) x R references x 3 layers
            int64_t left[2];
            for (int s = 0; s < 2; ++s) {
                const int64_t t0 = (int64_t)blockIdx.x * 2 + s;
                left[s] = t0 < tiles ? ((tiles - 1 - t0) / step + 1) * (int64_t)R * 3 : 0;
            }
            int layer[2] = {0, 0};
            uint32_t na[2] = {0, 0};
            const uint32_t sw = smem_u32(smem + kOffW);
            uint32_t polls = 0;
            uint64_t t0 = 0;
            while ((left[0] > 0 || left[1] > 0) && !*abort_flag) {
                bool progressed = false;
                for (int s = 0; s < 2; ++s) {
                    if (left[s] == 0 || !test_wait(&a_ready[s], na[s] & 1u)) continue;
                    progressed = true;
                    ++na[s];
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + kOffSlot + s * kSlotBytes);
                    const uint32_t wl = sw + (uint32_t)(2 * layer[s]) * kAtom;
                    const uint32_t d = tmem + (uint32_t)(s * 128);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {  // K = 128: two atoms, 4 steps of 16 each
                        const uint32_t at = (uint32_t)(kk >> 2) * kAtom;
                        tc_mma(d, desc_sw128(sa + at) + (uint64_t)((kk & 3) * 2),
                               desc_sw128(wl + at) + (uint64_t)((kk & 3) * 2), idesc, kk > 0 ? 1u : 0u);
                    }
                    tc_commit(&d_ready[s]);
                    layer[s] = layer[s] == 2 ? 0 : layer[s] + 1;
                    --left[s];
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
        unsigned char* A = smem + kOffSlot + s * kSlotBytes;
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(s * 128);
        const float b4 = a.params[a.offb4];
        uint32_t nd = 0;
        for (int64_t t = (int64_t)blockIdx.x * 2 + s; t < tiles; t += step) {
            const int64_t v = t * kTile + i;
            // this row's vertex, encoded once for every reference (rows past N encode
            // position 0: harmless, never written out)
            float fq[kLF];
            {
                const int64_t vv = v < a.N ? v : 0;
                const int64_t x = vv % a.X, y = (vv / a.X) % a.Y, z = vv / (a.X * a.Y);
                const float p[3] = {pos_axis(x, a.X), pos_axis(y, a.Y), pos_axis(z, a.Z)};
#pragma unroll
                for (int l = 0; l < kLevels; ++l) {
                    float f[kFeat];
                    encode_level(a.G, l, p, f);
#pragma unroll
                    for (int q = 0; q < kFeat; ++q) fq[l * kFeat + q] = f[q];
                }
            }
            for (int r = 0; r < R; ++r) {
                const float* fr = fr_all + r * kLF;
                // x = [fr * fq ; fr + fq]: 16-byte chunks 0-7 the products, 8-15 the sums
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float4 r0 = *reinterpret_cast<const float4*>(fr + 8 * c);
                    const float4 r1 = *reinterpret_cast<const float4*>(fr + 8 * c + 4);
                    const float* q = fq + 8 * c;
                    *reinterpret_cast<uint4*>(A + swz(i, c)) =
                        make_uint4(bf2(r0.x * q[0], r0.y * q[1]), bf2(r0.z * q[2], r0.w * q[3]),
                                   bf2(r1.x * q[4], r1.y * q[5]), bf2(r1.z * q[6], r1.w * q[7]));
                    *reinterpret_cast<uint4*>(A + kAtom + swz(i, c)) =
                        make_uint4(bf2(r0.x + q[0], r0.y + q[1]), bf2(r0.z + q[2], r0.w + q[3]),
                                   bf2(r1.x + q[4], r1.y + q[5]), bf2(r1.z + q[6], r1.w + q[7]));
                }
                proxy_fence();
                tc_fence_before();
                arrive(&a_ready[s]);
                for (int layer = 0; layer < 3; ++layer) {
                    if (!__all_sync(0xffffffffu, wait_bounded(&d_ready[s], nd & 1u, abort_flag))) goto done;
                    ++nd;
                    tc_fence_after();
                    const float* bias = vec + layer * kHid;
                    float acc = 0.0f;
#pragma unroll
                    for (int c0 = 0; c0 < kHid; c0 += 32) {
                        float h[32];
                        tmem_ld32(taddr + (uint32_t)c0, h);
#pragma unroll
                        for (int j = 0; j < 32; ++j) h[j] = fmaxf(h[j] + bias[c0 + j], 0.0f);
                        if (layer < 2) {  // next layer's operand: columns c0..c0+31
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int c = (c0 >> 3) + q;  // 16-byte chunk of the 256-byte row
                                *reinterpret_cast<uint4*>(A + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) =
                                    make_uint4(bf2(h[8 * q], h[8 * q + 1]), bf2(h[8 * q + 2], h[8 * q + 3]),
                                               bf2(h[8 * q + 4], h[8 * q + 5]), bf2(h[8 * q + 6], h[8 * q + 7]));
                            }
                        } else {  // output layer on the BF16-rounded h3
#pragma unroll
                            for (int j = 0; j < 32; j += 2) {
                                const float2 hv = unbf2(bf2(h[j], h[j + 1]));
                                acc = fmaf(vec[3 * kHid + c0 + j], hv.x,
                                           fmaf(vec[3 * kHid + c0 + j + 1], hv.y, acc));
                            }
                        }
                    }
                    if (layer < 2) {
                        proxy_fence();
                        tc_fence_before();
                        arrive(&a_ready[s]);
                    } else if (v < a.N) {
                        const float o = acc + b4;
                        a.out[(int64_t)r * a.N + v] =
                            a.measure == 0 ? tanhf(o) : (o > 20.f ? o : log1pf(expf(o)));
                    }
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

cudaError_t launch_infer_tc(ndf_model* m, const int64_t* d_refs, int R, float* out) {
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
    a.w = m->wbf;
    a.params = m->params;
    a.offb1 = m->L.b1;
    a.offb2 = m->L.b2;
    a.offb3 = m->L.b3;
    a.offw4 = m->L.w4;
    a.offb4 = m->L.b4;
    a.N = m->X * m->Y * m->Z;
    a.X = m->X;
    a.Y = m->Y;
    a.Z = m->Z;
    a.measure = m->measure;
    a.status = ctx->flag.as<unsigned>() + 1;
    const int64_t tiles = (a.N + kTile - 1) / kTile;
    int64_t grid = ctx->sm_count;  // one persistent CTA per SM, two tiles in flight each
    if (grid > (tiles + 1) / 2) grid = (tiles + 1) / 2;
    if (grid < 1) grid = 1;
    for (int r0 = 0; r0 < R; r0 += kMaxRefsPerLaunch) {
        a.refs = d_refs + r0;
        a.R = R - r0 < kMaxRefsPerLaunch ? R - r0 : kMaxRefsPerLaunch;
        a.out = out + (int64_t)r0 * a.N;
        infer_tc_kernel<<<(unsigned)grid, kTcThreads, kTcSmem, ctx->stream>>>(a);
        ctx->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ndf

// The dense NDF's MLP (Sec. 4.1, Eq. 3 training) on the 5th-generation tensor
// cores: forward, data gradient and weight gradient of the three 128 x 128 ReLU
// layers, BF16 operands with FP32 accumulation in TMEM.
//
// Layout of the activations: the merged input x is [B][128] (row-major, written by
// the encoding kernel); the kernels here write the layer inputs and the
// pre-activation gradients TRANSPOSED, feature-major [128][Bs] (Bs = B rounded up
// to 8), because a thread owns one sample: for each feature a warp stores 32
// consecutive samples (64 contiguous bytes), and the transposed matrices are the
// K-major operands of the weight gradient, whose K is the batch.
//
//   forward (per 128-sample tile): A = x rows -> layer 1 -> ReLU -> layer 2 -> ...;
//     writes x^T, h1^T, h2^T, h3^T (training), the output layer and L1 loss terms.
//   data gradient (per tile): dz3 = dL/do * w4 * [h3 > 0]; dz2 = (dz3 W3) * [h2 > 0];
//     dz1 = (dz2 W2) * [h1 > 0]; dx = dz1 W1 (FP32); writes dz3^T, dz2^T, dz1^T, dx.
//     The B operands are the transposed weights W^T ([in][out]).
//   weight gradient: dW_l = dz_l^T . h_(l-1) = sum over the batch, as a GEMM with
//     M = N = 128 and K = the batch: A = dz_l^T, B = h_(l-1)^T, both K-major, loaded
//     by TMA (128-byte swizzle) into a ring; each CTA sums one chunk of the batch in
//     TMEM and writes its partial 128 x 128 FP32 tile; a second kernel adds the
//     chunks in order (deterministic), and the bias and output-layer gradients are
//     row sums of the transposed matrices.
// The forward and data-gradient kernels follow the structure of the volume decoder
// (ndf_decode_tc.cu): one persistent CTA per SM, two 128-row slots (warps 0-3, 4-7)
// whose epilogues overlap the other slot's MMAs, warp 8 allocating TMEM and issuing
// tcgen05.mma (M = N = K = 128 per layer).  All waits are bounded.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "ndf_net.h"
#include "tc_common.cuh"

namespace ndf {

namespace {

using namespace tc;

constexpr int kTile = 128;
constexpr int kThreads = 288;  // 8 epilogue warps + 1 MMA warp
// shared memory: three 128 x 128 weight matrices (2 atoms each), one 2-atom operand
// per slot, bias / output-weight vectors, barriers
constexpr uint32_t kOffW = 0, kOffSlot = 6 * kAtom, kSlotBytes = 2 * kAtom;
constexpr uint32_t kOffVec = kOffSlot + 2 * kSlotBytes;
constexpr uint32_t kOffBar = kOffVec + 4 * kHid * 4;
constexpr uint32_t kSmem = kOffBar + 256 + 1024;

__device__ __forceinline__ float out_act(int measure, float o) {
    return measure == 0 ? tanhf(o) : (o > 20.0f ? o : log1pf(expf(o)));
}
__device__ __forceinline__ float out_dact(int measure, float o) {
    if (measure == 0) {
        const float t = tanhf(o);
        return 1.0f - t * t;
    }
    return 1.0f / (1.0f + expf(-o));
}

__device__ __forceinline__ __nv_bfloat16 bf(float v) { return __float2bfloat16_rn(v); }

// the three weight matrices ([rows][128] BF16, rows = MMA N) into the swizzled K-major layout
__device__ __forceinline__ void load_weights_sw(unsigned char* smem, const __nv_bfloat16* w) {
    for (int i = threadIdx.x; i < 3 * kHid * 16; i += blockDim.x) {
        const int l = i / (kHid * 16), row = (i >> 4) % kHid, c = i & 15;
        const uint32_t o = (uint32_t)(2 * l + (c >> 3)) * kAtom + swz(row, c & 7);
        *reinterpret_cast<uint4*>(smem + kOffW + o) =
            reinterpret_cast<const uint4*>(w + ((size_t)l * kHid + row) * kHid)[c];
    }
}

// the MMA issuer of both kernels: for each operand a slot announces, one layer
// (eight K = 16 steps over two atoms) against the weight matrix of that step of
// the slot's three-step sequence (order[0..2]), committed to the slot's barrier
__device__ void mma_loop(unsigned char* smem, uint32_t tmem, uint64_t* a_ready, uint64_t* d_ready,
                         int64_t tiles, int64_t step, const int (&order)[3],
                         volatile int* abort_flag) {
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) |
                           ((uint32_t)(kTile >> 4) << 24);
    int64_t left[2];
    for (int s = 0; s < 2; ++s) {
        const int64_t t0 = (int64_t)blockIdx.x * 2 + s;
        left[s] = t0 < tiles ? ((tiles - 1 - t0) / step + 1) * 3 : 0;
    }
    int layer[2] = {0, 0};
    uint32_t na[2] = {0, 0};
    const uint32_t sw = smem_u32(smem + kOffW);
    uint32_t polls = 0;
    uint64_t t0 = 0;
    while ((left[0] > 0 || left[1] > 0) && !*abort_flag) {
        bool progressed = false;
        for (int s = 0; s < 2; ++s) {
            if (left[s] == 0 || !try_wait(&a_ready[s], na[s] & 1u)) continue;
            progressed = true;
            ++na[s];
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + kOffSlot + s * kSlotBytes);
            const uint32_t wl = sw + (uint32_t)(2 * order[layer[s]]) * kAtom;
            const uint32_t d = tmem + (uint32_t)(s * 128);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
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
        } else if ((polls & 1023u) == 0u) {
            const uint64_t t = global_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kWaitNs) *abort_flag = 1;
        }
    }
}

// writes 32 FP32 values of row i, columns c0.., as BF16 into the slot's operand
__device__ __forceinline__ void put_operand(unsigned char* A, int i, int c0, const float (&h)[32]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = (c0 >> 3) + q;
        *reinterpret_cast<uint4*>(A + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) =
            make_uint4(bf2(h[8 * q], h[8 * q + 1]), bf2(h[8 * q + 2], h[8 * q + 3]),
                       bf2(h[8 * q + 4], h[8 * q + 5]), bf2(h[8 * q + 6], h[8 * q + 7]));
    }
}

// prologue shared by both kernels: barriers, TMEM (2 slots x 128 columns)
__device__ __forceinline__ uint32_t setup(unsigned char* smem, uint64_t* bars, uint32_t* tmem_slot,
                                          volatile int* abort_flag) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&bars[s], 128);     // a_ready: the slot's 128 threads
            mbar_init(&bars[2 + s], 1);   // d_ready: the MMA commit
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
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *tmem_slot;
}

__device__ __forceinline__ void teardown(uint32_t tmem, volatile int* abort_flag, unsigned* status) {
    if (*abort_flag && threadIdx.x == 0) report(status, kDevTimeout);
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                     : "memory");
    }
}

}  // namespace

struct MlpTcArgs {
    const __nv_bfloat16* w;  // [3][128][128]: W ([out][in], forward) or W^T ([in][out], backward)
    const float* params;     // FP32 master: biases, w4, b4
    int64_t off_b[3], off_w4, off_b4;
    int64_t B, Bs;           // samples; row pitch of the transposed matrices (B rounded to 8)
    const __nv_bfloat16* x;  // [B][128] merged input
    __nv_bfloat16* hT;       // [4][128][Bs]: x^T, h1^T, h2^T, h3^T
    __nv_bfloat16* dzT;      // [3][128][Bs]: dz1^T, dz2^T, dz3^T
    float* dx;               // [B][128]
    float* o;                // [B] pre-activation output (training)
    float* dout;             // [B] dL/do
    const float* target;     // [B] (training) or null
    float* y;                // [B] output (inference) or null
    double* loss;            // sum |y - t|
    int measure;
    unsigned* status;
};

template <bool TRAIN>
__global__ void __launch_bounds__(kThreads, 1) mlp_fwd_tc_kernel(const MlpTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* vec = reinterpret_cast<float*>(smem + kOffVec);  // b1, b2, b3, w4
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    load_weights_sw(smem, a.w);
    for (int i = threadIdx.x; i < 4 * kHid; i += blockDim.x)
        vec[i] = a.params[(i < 3 * kHid ? a.off_b[i / kHid] : a.off_w4) + (i % kHid)];
    const uint32_t tmem = setup(smem, bars, tmem_slot, abort_flag);
    const int64_t tiles = (a.B + kTile - 1) / kTile;
    const int64_t step = (int64_t)gridDim.x * 2;
    double loss_acc = 0.0;
    if (warp == 8) {
        if (lane == 0) {
            const int order[3] = {0, 1, 2};
            mma_loop(smem, tmem, bars, bars + 2, tiles, step, order, abort_flag);
        }
    } else {
        const int s = warp >> 2;
        const int i = (warp & 3) * 32 + lane;
        unsigned char* A = smem + kOffSlot + s * kSlotBytes;
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(s * 128);
        const float b4 = a.params[a.off_b4];
        uint32_t nd = 0;
        for (int64_t t = (int64_t)blockIdx.x * 2 + s; t < tiles; t += step) {
            const int64_t b = t * kTile + i;
            const bool in = b < a.B;
            // the sample's merged input (zero rows past B) into the operand, and x^T
            const uint4* xr = reinterpret_cast<const uint4*>(a.x + (in ? b : 0) * kIn);
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const uint4 u = in ? xr[c] : make_uint4(0, 0, 0, 0);
                *reinterpret_cast<uint4*>(A + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) = u;
                if (TRAIN && in) {
                    const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const __nv_bfloat162 p = *reinterpret_cast<const __nv_bfloat162*>(&uu[q]);
                        a.hT[(int64_t)(8 * c + 2 * q) * a.Bs + b] = p.x;
                        a.hT[(int64_t)(8 * c + 2 * q + 1) * a.Bs + b] = p.y;
                    }
                }
            }
            proxy_fence();
            tc_fence_before();
            arrive(&bars[s]);
            for (int layer = 0; layer < 3; ++layer) {
                if (!__all_sync(0xffffffffu, wait_bounded(&bars[2 + s], nd & 1u, abort_flag))) goto done;
                ++nd;
                tc_fence_after();
                const float* bias = vec + layer * kHid;
                float acc = 0.0f;
                __nv_bfloat16* hl = a.hT + (int64_t)(layer + 1) * kHid * a.Bs;
#pragma unroll
                for (int c0 = 0; c0 < kHid; c0 += 32) {
                    float h[32];
                    tmem_ld32(taddr + (uint32_t)c0, h);
#pragma unroll
                    for (int j = 0; j < 32; ++j) h[j] = fmaxf(h[j] + bias[c0 + j], 0.0f);
                    if (TRAIN && in) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) hl[(int64_t)(c0 + j) * a.Bs + b] = bf(h[j]);
                    }
                    if (layer < 2) {
                        put_operand(A, i, c0, h);
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
                    arrive(&bars[s]);
                } else if (in) {
                    const float o = acc + b4;
                    const float y = out_act(a.measure, o);
                    if (TRAIN) {
                        a.o[b] = o;
                        const float e = y - a.target[b];
                        loss_acc += fabs((double)e);
                        const float sg = e > 0.0f ? 1.0f : (e < 0.0f ? -1.0f : 0.0f);
                        a.dout[b] = sg / (float)a.B * out_dact(a.measure, o);
                    } else {
                        a.y[b] = y;
                    }
                }
            }
        }
    }
done:
    if (TRAIN && warp < 8) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
        if (lane == 0 && loss_acc != 0.0) atomicAdd(a.loss, loss_acc);
    }
    teardown(tmem, abort_flag, a.status);
}

__global__ void __launch_bounds__(kThreads, 1) mlp_bwd_tc_kernel(const MlpTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* w4 = reinterpret_cast<float*>(smem + kOffVec);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    load_weights_sw(smem, a.w);  // W^T: rows = inputs of each layer
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) w4[i] = a.params[a.off_w4 + i];
    const uint32_t tmem = setup(smem, bars, tmem_slot, abort_flag);
    const int64_t tiles = (a.B + kTile - 1) / kTile;
    const int64_t step = (int64_t)gridDim.x * 2;
    if (warp == 8) {
        if (lane == 0) {
            const int order[3] = {2, 1, 0};  // W3^T, W2^T, W1^T
            mma_loop(smem, tmem, bars, bars + 2, tiles, step, order, abort_flag);
        }
    } else {
        const int s = warp >> 2;
        const int i = (warp & 3) * 32 + lane;
        unsigned char* A = smem + kOffSlot + s * kSlotBytes;
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(s * 128);
        uint32_t nd = 0;
        for (int64_t t = (int64_t)blockIdx.x * 2 + s; t < tiles; t += step) {
            const int64_t b = t * kTile + i;
            const bool in = b < a.B;
            const int64_t bb = in ? b : 0;
            // dz3 = dL/do * w4 * [h3 > 0]; the 32 mask values of a chunk are loaded
            // (read-only path) before any store, so their latencies overlap
            {
                const float d = in ? a.dout[b] : 0.0f;
                const __nv_bfloat16* h3 = a.hT + (int64_t)3 * kHid * a.Bs;
                __nv_bfloat16* z3 = a.dzT + (int64_t)2 * kHid * a.Bs;
#pragma unroll
                for (int c0 = 0; c0 < kHid; c0 += 32) {
                    float g[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) g[j] = __bfloat162float(__ldg(h3 + (int64_t)(c0 + j) * a.Bs + bb));
#pragma unroll
                    for (int j = 0; j < 32; ++j) g[j] = (in && g[j] > 0.0f) ? d * w4[c0 + j] : 0.0f;
                    if (in) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) z3[(int64_t)(c0 + j) * a.Bs + b] = bf(g[j]);
                    }
                    put_operand(A, i, c0, g);
                }
            }
            proxy_fence();
            tc_fence_before();
            arrive(&bars[s]);
            for (int layer = 2; layer >= 0; --layer) {  // the MMA multiplied by W_(layer+1)^T
                if (!__all_sync(0xffffffffu, wait_bounded(&bars[2 + s], nd & 1u, abort_flag))) goto done;
                ++nd;
                tc_fence_after();
#pragma unroll
                for (int c0 = 0; c0 < kHid; c0 += 32) {
                    float g[32];
                    tmem_ld32(taddr + (uint32_t)c0, g);
                    if (layer > 0) {  // through the ReLU of h_layer: dz_layer
                        const __nv_bfloat16* hp = a.hT + (int64_t)layer * kHid * a.Bs;
                        __nv_bfloat16* zp = a.dzT + (int64_t)(layer - 1) * kHid * a.Bs;
                        float hv[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) hv[j] = __bfloat162float(__ldg(hp + (int64_t)(c0 + j) * a.Bs + bb));
#pragma unroll
                        for (int j = 0; j < 32; ++j) g[j] = (in && hv[j] > 0.0f) ? g[j] : 0.0f;
                        if (in) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) zp[(int64_t)(c0 + j) * a.Bs + b] = bf(g[j]);
                        }
                        put_operand(A, i, c0, g);
                    } else if (in) {  // dx, FP32
                        float4* d = reinterpret_cast<float4*>(a.dx + b * kIn + c0);
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            d[q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
                    }
                }
                if (layer > 0) {
                    proxy_fence();
                    tc_fence_before();
                    arrive(&bars[s]);
                }
            }
        }
    }
done:
    teardown(tmem, abort_flag, a.status);
}

// ---------------------------------------------------------------- weight gradient
constexpr int kWgStages = 6;
constexpr uint32_t kWgTile = 128 * 128;          // one 128-row x 128-byte tile (64 samples)
constexpr uint32_t kWgStage = 2 * kWgTile;       // A and B
constexpr uint32_t kWgSmem = kWgStages * kWgStage + 256 + 1024;

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// part[l][chunk][o][i] = sum over the chunk's samples b of A_l[o][b] * B_l[i][b] for
// the three layers at once (blockIdx.y = l; A_l = dz_l^T, B_l = h_(l-1)^T, [128][Bs]
// BF16 each; 6 warps: TMA producer, MMA issuer, four epilogue warps)
__global__ void __launch_bounds__(192, 1)
    mlp_wgrad_tc_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                        const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
                        const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2,
                        int64_t B, int64_t chunk, float* __restrict__ part_all, unsigned* status) {
    const int layer = blockIdx.y;
    const CUtensorMap* mA = layer == 0 ? &mA0 : (layer == 1 ? &mA1 : &mA2);
    const CUtensorMap* mB = layer == 0 ? &mB0 : (layer == 1 ? &mB1 : &mB2);
    float* part = part_all + (int64_t)layer * kMlpMaxChunks * kHid * kHid;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kWgStages * kWgStage);
    uint64_t* empty = full + kWgStages;
    uint64_t* acc_full = empty + kWgStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        *abort_flag = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t k0 = (int64_t)blockIdx.x * chunk;
    const int64_t k1 = k0 + chunk < B ? k0 + chunk : B;
    const int nk = (int)((k1 - k0 + 63) / 64);  // 64 samples (128 bytes) per stage
    if (warp == 0) {
        if (lane == 0) {  // ---- TMA producer
            for (int ks = 0; ks < nk; ++ks) {
                const int st = ks % kWgStages;
                const uint32_t ph = (uint32_t)(ks / kWgStages) & 1u;
                if (!wait_bounded(&empty[st], ph ^ 1u, abort_flag)) break;
                unsigned char* p = smem + st * kWgStage;
                mbar_expect_tx(&full[st], kWgStage);
                const int x = (int)(k0 + 64 * ks);
                tma_2d(p, mA, x, 0, &full[st]);
                tma_2d(p + kWgTile, mB, x, 0, &full[st]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer: D[o][i] += A[o][k] B[i][k]
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);
            for (int ks = 0; ks < nk; ++ks) {
                const int st = ks % kWgStages;
                const uint32_t ph = (uint32_t)(ks / kWgStages) & 1u;
                if (!wait_bounded(&full[st], ph, abort_flag)) break;
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + st * kWgStage);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma(tmem, desc_sw128(sa) + (uint64_t)(kk * 2),
                           desc_sw128(sa + kWgTile) + (uint64_t)(kk * 2), idesc,
                           (ks > 0 || kk > 0) ? 1u : 0u);
                tc_commit(&empty[st]);
            }
            tc_commit(acc_full);
        }
    } else {  // ---- epilogue: warps 2..5, TMEM lane quarter warp % 4
        const int q = warp & 3;
        const int o = q * 32 + lane;
        float* dst = part + (int64_t)blockIdx.x * kHid * kHid + (int64_t)o * kHid;
        if (__all_sync(0xffffffffu, nk > 0 && wait_bounded(acc_full, 0u, abort_flag))) {
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
            for (int c0 = 0; c0 < kHid; c0 += 32) {
                float v[32];
                tmem_ld32(taddr + (uint32_t)c0, v);
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    *reinterpret_cast<float4*>(dst + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
        } else if (nk == 0) {
            for (int c = 0; c < kHid; ++c) dst[c] = 0.0f;
        }
    }
    if (*abort_flag && threadIdx.x == 0) report(status, kDevTimeout);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u)
                     : "memory");
    }
}

// grad[W_l][o][i] += sum over the chunks, in order (blockIdx.y = l)
__global__ void wgrad_reduce_kernel(const float* __restrict__ part_all, int chunks, float* __restrict__ grad,
                                    int64_t offW0, int64_t offW1, int64_t offW2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kHid * kHid) return;
    const int l = blockIdx.y;
    const float* part = part_all + (int64_t)l * kMlpMaxChunks * kHid * kHid;
    float s = 0.0f;
    for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * kHid * kHid + e];
    grad[(l == 0 ? offW0 : (l == 1 ? offW1 : offW2)) + e] += s;
}

// row sums in two fixed-order passes: CTA (r, z) of 256 threads sums slice z of
// row r of rows[r][Bs] (B used; times scale[b] if given) in eight-sample (16-byte)
// groups into part[z][r]; row_sums_finish adds the slices in order into out[r].
constexpr int kRowSplit = 8;
constexpr int kVecParts = 64;

__global__ void __launch_bounds__(256)
    row_sums_kernel(const __nv_bfloat16* __restrict__ rows, int64_t Bs, int64_t B,
                    const float* __restrict__ scale, float* __restrict__ part) {
    __shared__ float red[8];
    const __nv_bfloat16* p = rows + (int64_t)blockIdx.x * Bs;
    const int64_t groups = (B + 7) / 8;  // Bs is a multiple of 8: groups are 16-byte aligned
    const int64_t per = (groups + kRowSplit - 1) / kRowSplit;
    const int64_t g0 = (int64_t)blockIdx.y * per, g1 = g0 + per < groups ? g0 + per : groups;
    float s = 0.0f;
    for (int64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(p) + g);
        const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 v = unbf2(uu[q]);
            const int64_t b = 8 * g + 2 * q;  // the pitch's padding past B is never written:
            if (b < B) s = fmaf(v.x, scale ? scale[b] : 1.0f, s);  // skipped, not multiplied
            if (b + 1 < B) s = fmaf(v.y, scale ? scale[b + 1] : 1.0f, s);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void row_sums_finish(const float* __restrict__ part, int nrows, float* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    float t = 0.0f;
    for (int z = 0; z < kRowSplit; ++z) t += part[z * nrows + r];
    out[r] += t;
}

// part[blockIdx.x] = sum of a fixed slice of v (fixed order), for vec_sum_finish
__global__ void __launch_bounds__(256) vec_sum_kernel(const float* __restrict__ v, int64_t n,
                                                       float* __restrict__ part) {
    __shared__ float red[8];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * per, i1 = i0 + per < n ? i0 + per : n;
    float s = 0.0f;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void vec_sum_finish(const float* __restrict__ part, int n, float* __restrict__ out) {
    float t = 0.0f;
    for (int i = 0; i < n; ++i) t += part[i];
    *out += t;
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// [128][Bs] BF16 matrix with B columns used: 128-row x 64-column (128-byte) boxes,
// 128-byte swizzle; columns past B read as zero
static bool map_transposed(CUtensorMap* m, const __nv_bfloat16* base, int64_t B, int64_t Bs) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)B, (cuuint64_t)kHid};
    cuuint64_t strides[1] = {(cuuint64_t)Bs * 2};
    cuuint32_t box[2] = {64, 128};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static MlpTcArgs tc_args(ndf_model* m, int64_t B) {
    MlpTcArgs a;
    a.params = m->params;
    a.off_b[0] = m->L.b1;
    a.off_b[1] = m->L.b2;
    a.off_b[2] = m->L.b3;
    a.off_w4 = m->L.w4;
    a.off_b4 = m->L.b4;
    a.B = B;
    a.Bs = (B + 7) & ~int64_t(7);
    a.x = m->work.x;
    a.hT = m->work.hT;
    a.dzT = m->work.dzT;
    a.dx = m->work.dx;
    a.o = m->work.o;
    a.dout = m->work.dout;
    a.target = nullptr;
    a.y = nullptr;
    a.loss = m->work.loss;
    a.measure = m->measure;
    a.status = m->ctx->flag.as<unsigned>() + 1;
    return a;
}

static cudaError_t set_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_tc_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_fwd_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kWgSmem);
    if (e == cudaSuccess) done = true;
    return e;
}

static unsigned persistent_tiles(ndf_ctx* ctx, int64_t B) {
    const int64_t tiles = (B + kTile - 1) / kTile;
    int64_t grid = ctx->sm_count;
    if (grid > (tiles + 1) / 2) grid = (tiles + 1) / 2;
    return (unsigned)(grid < 1 ? 1 : grid);
}

cudaError_t mlp_tc_forward(ndf_model* m, int64_t B, const float* target, float* y) {
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    MlpTcArgs a = tc_args(m, B);
    a.w = m->wbf;
    a.target = target;
    a.y = y;
    cudaStream_t s = m->ctx->stream;
    if (target) mlp_fwd_tc_kernel<true><<<persistent_tiles(m->ctx, B), kThreads, kSmem, s>>>(a);
    else mlp_fwd_tc_kernel<false><<<persistent_tiles(m->ctx, B), kThreads, kSmem, s>>>(a);
    m->ctx->launches++;
    return cudaGetLastError();
}

cudaError_t mlp_tc_backward(ndf_model* m, int64_t B) {
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    ndf_ctx* ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    MlpTcArgs a = tc_args(m, B);
    a.w = m->wtbf;
    mlp_bwd_tc_kernel<<<persistent_tiles(ctx, B), kThreads, kSmem, s>>>(a);
    ctx->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // weight gradients, the three layers in one launch: about one CTA per SM, each
    // summing a chunk of whole 64-sample stages of one layer
    int64_t chunks = ctx->sm_count / 3;
    if (chunks < 1) chunks = 1;
    int64_t chunk = (B + chunks - 1) / chunks;
    chunk = (chunk + 63) / 64 * 64;
    chunks = (B + chunk - 1) / chunk;
    if (chunks > kMlpMaxChunks - 1) {  // the last partial tile holds the row-sum slices
        chunk = ((B + kMlpMaxChunks - 2) / (kMlpMaxChunks - 1) + 63) / 64 * 64;
        chunks = (B + chunk - 1) / chunk;
    }
    const int64_t Bs = a.Bs;
    // the row-sum slices use the last partial tile of the weight gradients, which no
    // layer's chunks reach (chunks <= kMlpMaxChunks - 1 by construction above)
    float* rpart = m->work.wpart + ((size_t)3 * kMlpMaxChunks - 1) * kHid * kHid;
    const int64_t offW[3] = {m->L.W1, m->L.W2, m->L.W3};
    const int64_t offb[3] = {m->L.b1, m->L.b2, m->L.b3};
    CUtensorMap mA[3], mB[3];
    for (int l = 0; l < 3; ++l)
        if (!map_transposed(&mA[l], m->work.dzT + (size_t)l * kHid * Bs, B, Bs) ||
            !map_transposed(&mB[l], m->work.hT + (size_t)l * kHid * Bs, B, Bs))
            return cudaErrorUnknown;
    mlp_wgrad_tc_kernel<<<dim3((unsigned)chunks, 3), 192, kWgSmem, s>>>(
        mA[0], mA[1], mA[2], mB[0], mB[1], mB[2], B, chunk, m->work.wpart, a.status);
    wgrad_reduce_kernel<<<dim3(kHid * kHid / 256, 3), 256, 0, s>>>(m->work.wpart, (int)chunks, m->grad,
                                                                  offW[0], offW[1], offW[2]);
    ctx->launches += 2;
    for (int l = 0; l < 3; ++l) {
        row_sums_kernel<<<dim3(kHid, kRowSplit), 256, 0, s>>>(m->work.dzT + (size_t)l * kHid * Bs,
                                                              Bs, B, nullptr, rpart);
        row_sums_finish<<<1, kHid, 0, s>>>(rpart, kHid, m->grad + offb[l]);
        ctx->launches += 2;
    }
    // output layer: dw4 = sum_b dout[b] h3[b], db4 = sum_b dout[b]
    row_sums_kernel<<<dim3(kHid, kRowSplit), 256, 0, s>>>(m->work.hT + (size_t)3 * kHid * Bs, Bs, B,
                                                          m->work.dout, rpart);
    row_sums_finish<<<1, kHid, 0, s>>>(rpart, kHid, m->grad + m->L.w4);
    vec_sum_kernel<<<kVecParts, 256, 0, s>>>(m->work.dout, B, rpart);
    vec_sum_finish<<<1, 1, 0, s>>>(rpart, kVecParts, m->grad + m->L.b4);
    ctx->launches += 4;
    return cudaGetLastError();
}

}  // namespace ndf

// The dense NDF's MLP (Sec. 4.1, Eq. 3 training) on the 5th-generation tensor
// cores: the three 128 x 128 ReLU layers and the output layer, BF16 operands with
// FP32 accumulation in TMEM.
//
// Training (mlp_train_tc_kernel): one persistent kernel per step does, for each
// 128-sample tile, the forward pass, the L1 loss and its output gradient, the data
// gradients and the weight gradients, without writing activations to global memory.
//   Shared memory: W1..W3 (BF16, [out][in], 128-byte-swizzled K-major atoms, 96 KB)
//   and four tile buffers of the same layout, X (the merged input), H1, H2 and DZ
//   (the pre-activation gradient of the layer being processed), 32 KB each.
//   TMEM (512 columns): a working accumulator (layer outputs, data gradients) and the
//   CTA's weight-gradient sums dW1..dW3, accumulated over its tiles.
//   Every buffer serves two ways: as the K-major A operand ([sample][feature]) of a
//   forward or data-gradient product, and read MN-major (features contiguous, the
//   samples as K) as an operand of the weight gradient dW_l = dz_l^T h_(l-1); the
//   weight tiles are the K-major B of the forward and, read MN-major, the B of the
//   data gradient dh = dz W.
//   Per tile:  z1 = X W1^T, h1 = relu(z1 + b1) -> H1;  z2 -> H2;  z3 -> h3, the
//     output o = w4 . h3 + b4 (on the BF16 h3), dL/do, dz3 = dL/do w4 [h3 > 0] -> DZ;
//     dh2 = DZ W3 and dW3 += DZ^T H2;  dz2 = dh2 [h2 > 0] -> DZ;  dh1 = DZ W2 and
//     dW2 += DZ^T H1;  dz1 -> DZ;  dx = DZ W1 (to global, FP32) and dW1 += DZ^T X.
//   The bias and output-layer gradients are column sums of the BF16 DZ (and of
//   dL/do times the BF16 h3): each warp sums its own 32 rows in a fixed order and
//   keeps the sums across the CTA's tiles.  At the end each CTA writes its dW tiles
//   and column sums, and two small kernels add them over the CTAs in order, so the
//   gradient is deterministic.
//   Warps 0-7 are the epilogue: warp w owns rows 32 (w % 4) .. + 31 of the tile (its
//   TMEM lane quarter) and columns 64 (w / 4) .. + 63; warp 8 allocates TMEM and
//   issues the MMAs.
// Inference (mlp_fwd_tc_kernel, the model's forward call) runs the forward alone in
// the structure of the volume decoder (ndf_decode_tc.cu): two 128-row slots whose
// epilogues overlap the other slot's MMAs.  All waits are bounded.
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
            if (left[s] == 0 || !test_wait(&a_ready[s], na[s] & 1u)) continue;
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


// ---------------------------------------------------------------- training
constexpr int kTrainThreads = 288;  // 8 epilogue warps + 1 MMA warp
constexpr uint32_t kOffX = 6 * kAtom, kOffH1 = 8 * kAtom, kOffH2 = 10 * kAtom, kOffDZ = 12 * kAtom;
constexpr uint32_t kOffXch = 14 * kAtom;                // [2][128] half-row output dot products
constexpr uint32_t kOffTBar = kOffXch + 2 * kHid * 4;
constexpr uint32_t kTrainSmem = kOffTBar + 64 + 1024;
constexpr int kColSums = 5;                              // db1, db2, db3, dw4, db4 (first entry)

constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);  // FP32 = BF16 x BF16, M = N = 128
constexpr uint32_t kIdescBMn = kIdesc | (1u << 16);              // B read MN-major
constexpr uint32_t kIdescABMn = kIdesc | (1u << 15) | (1u << 16); // A and B read MN-major

// a two-atom tile read MN-major: 64 consecutive features per 128-byte row, the next
// 64 in the second atom (leading byte offset), 8-row groups of K 1024 bytes apart
__device__ __forceinline__ uint64_t desc_sw128_mn(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kAtom >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// D = A B^T over K = 128 (features): both tiles K-major
__device__ __forceinline__ void mma_fwd(uint32_t d, uint32_t a, uint32_t b) {
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t at = (uint32_t)(kk >> 2) * kAtom;
        tc_mma(d, desc_sw128(a + at) + (uint64_t)((kk & 3) * 2), desc_sw128(b + at) + (uint64_t)((kk & 3) * 2),
               kIdesc, kk > 0 ? 1u : 0u);
    }
}
// D = A W over K = 128 (the outputs of W): A K-major, the weight tile read MN-major
__device__ __forceinline__ void mma_dgrad(uint32_t d, uint32_t a, uint32_t w) {
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
        tc_mma(d, desc_sw128(a + (uint32_t)(kk >> 2) * kAtom) + (uint64_t)((kk & 3) * 2),
               desc_sw128_mn(w + (uint32_t)kk * 2048u), kIdescBMn, kk > 0 ? 1u : 0u);
}
// D (+)= A^T B over K = 128 (the tile's samples): both tiles read MN-major
__device__ __forceinline__ void mma_wgrad(uint32_t d, uint32_t a, uint32_t b, bool first) {
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
        tc_mma(d, desc_sw128_mn(a + (uint32_t)kk * 2048u), desc_sw128_mn(b + (uint32_t)kk * 2048u),
               kIdescABMn, (first && kk == 0) ? 0u : 1u);
}

// s += the sums over rows 32 q .. 32 q + 31 of the BF16 columns 2 lane, 2 lane + 1 of
// one atom (64 columns); rows in order
__device__ __forceinline__ void colsum(const unsigned char* atom, int q, int lane, float (&s)[2]) {
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
        const int row = 32 * q + r;
        const float2 v = unbf2(*reinterpret_cast<const uint32_t*>(atom + swz(row, lane >> 2) + (lane & 3) * 4));
        a0 += v.x;
        a1 += v.y;
    }
    s[0] += a0;
    s[1] += a1;
}
// the same, each row weighted by its lane's value d (the row's dL/do)
__device__ __forceinline__ void colsum_scaled(const unsigned char* atom, int q, int lane, float d,
                                              float (&s)[2]) {
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
        const int row = 32 * q + r;
        const float dr = __shfl_sync(0xffffffffu, d, r);
        const float2 v = unbf2(*reinterpret_cast<const uint32_t*>(atom + swz(row, lane >> 2) + (lane & 3) * 4));
        a0 = fmaf(dr, v.x, a0);
        a1 = fmaf(dr, v.y, a1);
    }
    s[0] += a0;
    s[1] += a1;
}

}  // namespace

struct MlpTrainArgs {
    const __nv_bfloat16* w;  // [3][128][128] W ([out][in])
    const float* params;     // FP32 master: biases, w4, b4
    int64_t off_b[3], off_w4, off_b4;
    int64_t B;
    const __nv_bfloat16* x;  // [B][128] merged input
    const float* target;     // [B]
    float* dx;               // [B][128] input gradient
    float* wpart;            // [3][gridDim.x][128][128] the CTAs' weight-gradient tiles
    float* cpart;            // [gridDim.x][4][kColSums][128] the CTAs' column sums per row quarter
    double* loss;            // sum |y - t|
    int measure;
    unsigned* status;
};

__global__ void __launch_bounds__(kTrainThreads, 1) mlp_train_tc_kernel(const MlpTrainArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* xch = reinterpret_cast<float*>(smem + kOffXch);
    // a_ready (the 256 epilogue threads), d_ready (the MMA commit), and per row quarter
    // the exchange of the two half-row output dot products (its two warps)
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffTBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 6);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    load_weights_sw(smem, a.w);
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 256);
        mbar_init(&bars[1], 1);
        for (int qq = 0; qq < 4; ++qq) mbar_init(&bars[2 + qq], 64);
        *abort_flag = 0;
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t tiles = (a.B + kTile - 1) / kTile;
    const uint32_t sW = smem_u32(smem + kOffW);
    const uint32_t sIn[3] = {smem_u32(smem + kOffX), smem_u32(smem + kOffH1), smem_u32(smem + kOffH2)};
    const uint32_t sDZ = smem_u32(smem + kOffDZ);
    if (warp == 8) {
        if (lane == 0) {  // ---- MMA issuer: six products per tile, each on its epilogue's signal
            uint32_t na = 0;
            bool first = true;
            for (int64_t t = blockIdx.x; t < tiles && !*abort_flag; t += gridDim.x) {
                for (int l = 0; l < 3; ++l) {  // z_(l+1) = h_l W_(l+1)^T
                    if (!wait_bounded(&bars[0], na & 1u, abort_flag)) break;
                    ++na;
                    tc_fence_after();
                    mma_fwd(tmem, sIn[l], sW + (uint32_t)(2 * l) * kAtom);
                    tc_commit(&bars[1]);
                }
                for (int l = 2; l >= 0 && !*abort_flag; --l) {  // dh_l = dz_(l+1) W_(l+1); dW_(l+1) += dz^T h_l
                    if (!wait_bounded(&bars[0], na & 1u, abort_flag)) break;
                    ++na;
                    tc_fence_after();
                    mma_dgrad(tmem, sDZ, sW + (uint32_t)(2 * l) * kAtom);
                    mma_wgrad(tmem + (uint32_t)(128 * (l + 1)), sDZ, sIn[l], first);
                    tc_commit(&bars[1]);
                }
                first = false;
            }
        }
    } else {  // ---- epilogue
        const int q = warp & 3, hh = warp >> 2;
        const int i = q * 32 + lane;  // row of the tile
        const int cb = hh * 64;       // first column of this warp's half
        const uint32_t trow = (uint32_t)(q * 32) << 16;
        const uint32_t twork = tmem + trow + (uint32_t)cb;
        unsigned char* X = smem + kOffX;
        unsigned char* H[2] = {smem + kOffH1, smem + kOffH2};
        unsigned char* DZ = smem + kOffDZ;
        unsigned char* DZh = DZ + hh * kAtom;  // this half's atom of DZ
        const float* w4 = a.params + a.off_w4;
        const float b4 = a.params[a.off_b4];
        float cs[4][2] = {};  // column sums (db1, db2, db3, dw4) of columns cb + 2 lane, + 1
        float sb4 = 0.0f;
        double loss_acc = 0.0;
        uint32_t nd = 0, nx = 0;
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
            const int64_t b = t * kTile + i;
            const bool in = b < a.B;
            const float tgt = in ? __ldg(a.target + b) : 0.0f;  // used at the output layer
            {  // this half of the sample's merged input -> X (zero rows past B)
                const uint4* xr = reinterpret_cast<const uint4*>(a.x + (in ? b : 0) * kIn) + hh * 8;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint4 u = in ? __ldg(xr + c) : make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4*>(X + hh * kAtom + swz(i, c)) = u;
                }
            }
            proxy_fence();
            tc_fence_before();
            arrive(&bars[0]);
            for (int l = 0; l < 2; ++l) {  // h1, h2
                if (!__all_sync(0xffffffffu, wait_bounded(&bars[1], nd & 1u, abort_flag))) goto done;
                ++nd;
                tc_fence_after();
                const float* bias = a.params + a.off_b[l];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    float v[32];
                    tmem_ld32(twork + (uint32_t)(32 * k), v);
                    const float4* bb = reinterpret_cast<const float4*>(bias + cb + 32 * k);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 bv = __ldg(bb + j);
                        v[4 * j] = fmaxf(v[4 * j] + bv.x, 0.0f);
                        v[4 * j + 1] = fmaxf(v[4 * j + 1] + bv.y, 0.0f);
                        v[4 * j + 2] = fmaxf(v[4 * j + 2] + bv.z, 0.0f);
                        v[4 * j + 3] = fmaxf(v[4 * j + 3] + bv.w, 0.0f);
                    }
                    put_operand(H[l], i, cb + 32 * k, v);
                }
                proxy_fence();
                tc_fence_before();
                arrive(&bars[0]);
            }
            {  // h3, the output, dL/do, dz3
                if (!__all_sync(0xffffffffu, wait_bounded(&bars[1], nd & 1u, abort_flag))) goto done;
                ++nd;
                tc_fence_after();
                const float* bias = a.params + a.off_b[2];
                uint32_t hb[32];  // BF16 h3 of this half, packed pairs
                float part = 0.0f;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    float v[32];
                    tmem_ld32(twork + (uint32_t)(32 * k), v);
                    const float4* bb = reinterpret_cast<const float4*>(bias + cb + 32 * k);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 bv = __ldg(bb + j);
                        hb[16 * k + 2 * j] = bf2(fmaxf(v[4 * j] + bv.x, 0.0f), fmaxf(v[4 * j + 1] + bv.y, 0.0f));
                        hb[16 * k + 2 * j + 1] =
                            bf2(fmaxf(v[4 * j + 2] + bv.z, 0.0f), fmaxf(v[4 * j + 3] + bv.w, 0.0f));
                    }
                    const float2* wp = reinterpret_cast<const float2*>(w4 + cb + 32 * k);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float2 hv = unbf2(hb[16 * k + j]);
                        const float2 wv = __ldg(wp + j);
                        part = fmaf(wv.x, hv.x, fmaf(wv.y, hv.y, part));
                    }
                }
                // the BF16 h3 into DZ for the output-weight column sums
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    *reinterpret_cast<uint4*>(DZh + swz(i, c)) =
                        make_uint4(hb[4 * c], hb[4 * c + 1], hb[4 * c + 2], hb[4 * c + 3]);
                xch[hh * kHid + i] = part;
                arrive(&bars[2 + q]);  // the two warps of this row quarter
                if (!__all_sync(0xffffffffu, wait_bounded(&bars[2 + q], nx & 1u, abort_flag))) goto done;
                ++nx;
                const float o = xch[i] + xch[kHid + i] + b4;
                float dout = 0.0f;
                if (in) {
                    const float y = out_act(a.measure, o);
                    const float e = y - tgt;
                    if (hh == 0) loss_acc += fabs((double)e);
                    const float sg = e > 0.0f ? 1.0f : (e < 0.0f ? -1.0f : 0.0f);
                    dout = sg / (float)a.B * out_dact(a.measure, o);
                }
                __syncwarp();
                colsum_scaled(DZh, q, lane, dout, cs[3]);
                if (hh == 0) {
                    float d = dout;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
                    sb4 += d;
                }
                __syncwarp();
                // dz3 = dL/do * w4 * [h3 > 0]
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint32_t g[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const float2 hv = unbf2(hb[4 * c + p]);
                        const float2 wv = __ldg(reinterpret_cast<const float2*>(w4 + cb + 8 * c + 2 * p));
                        g[p] = bf2(hv.x > 0.0f ? dout * wv.x : 0.0f, hv.y > 0.0f ? dout * wv.y : 0.0f);
                    }
                    *reinterpret_cast<uint4*>(DZh + swz(i, c)) = make_uint4(g[0], g[1], g[2], g[3]);
                }
                __syncwarp();
                colsum(DZh, q, lane, cs[2]);
                proxy_fence();
                tc_fence_before();
                arrive(&bars[0]);
            }
            {  // the next tile's input rows into L2 while the backward runs
                const int64_t bn = (t + gridDim.x) * kTile + i;
                if (bn < a.B)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.x + bn * kIn + hh * 64));
            }
            for (int l = 1; l >= 0; --l) {  // dz2 = dh2 [h2 > 0], dz1 = dh1 [h1 > 0]
                if (!__all_sync(0xffffffffu, wait_bounded(&bars[1], nd & 1u, abort_flag))) goto done;
                ++nd;
                tc_fence_after();
                const unsigned char* Hm = H[l] + hh * kAtom;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    float v[32];
                    tmem_ld32(twork + (uint32_t)(32 * k), v);
#pragma unroll
                    for (int cq = 0; cq < 4; ++cq) {
                        const uint4 u = *reinterpret_cast<const uint4*>(Hm + swz(i, 4 * k + cq));
                        const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const float2 hv = unbf2(uu[p]);
                            const int j = 8 * cq + 2 * p;
                            v[j] = hv.x > 0.0f ? v[j] : 0.0f;
                            v[j + 1] = hv.y > 0.0f ? v[j + 1] : 0.0f;
                        }
                    }
                    put_operand(DZ, i, cb + 32 * k, v);
                }
                __syncwarp();
                colsum(DZh, q, lane, cs[l]);
                proxy_fence();
                tc_fence_before();
                arrive(&bars[0]);
            }
            {  // dx = dz1 W1
                if (!__all_sync(0xffffffffu, wait_bounded(&bars[1], nd & 1u, abort_flag))) goto done;
                ++nd;
                tc_fence_after();
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    float v[32];
                    tmem_ld32(twork + (uint32_t)(32 * k), v);
                    if (in) {
                        float4* d = reinterpret_cast<float4*>(a.dx + b * kIn + cb + 32 * k);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            d[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    }
                }
            }
        }
        {  // the CTA's weight-gradient tiles (rows of this quarter, columns of this half)
           // and column sums; every MMA has completed (the last wait above)
#pragma unroll 1
        for (int l = 0; l < 3; ++l) {
            float* dst = a.wpart + ((int64_t)l * gridDim.x + blockIdx.x) * kHid * kHid + (int64_t)i * kHid + cb;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                float v[32];
                tmem_ld32(tmem + trow + (uint32_t)(128 * (l + 1) + cb + 32 * k), v);
                float4* d = reinterpret_cast<float4*>(dst + 32 * k);
#pragma unroll
                for (int j = 0; j < 8; ++j) d[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
        }
        float* cp = a.cpart + ((int64_t)blockIdx.x * 4 + q) * kColSums * kHid;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            cp[s * kHid + cb + 2 * lane] = cs[s][0];
            cp[s * kHid + cb + 2 * lane + 1] = cs[s][1];
        }
        if (hh == 0 && lane == 0) cp[4 * kHid] = sb4;
        }
    done:
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
        if (lane == 0 && loss_acc != 0.0) atomicAdd(a.loss, loss_acc);
    }
    if (*abort_flag && threadIdx.x == 0) report(a.status, kDevTimeout);
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                     : "memory");
    }
}

// grad[W_l][o][i] += the CTAs' tiles, in order (blockIdx.y = l)
__global__ void wgrad_reduce_kernel(const float* __restrict__ wpart, int parts, float* __restrict__ grad,
                                    int64_t offW0, int64_t offW1, int64_t offW2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kHid * kHid) return;
    const int l = blockIdx.y;
    const float* part = wpart + (int64_t)l * parts * kHid * kHid;
    float s = 0.0f;
    for (int c = 0; c < parts; ++c) s += part[(int64_t)c * kHid * kHid + e];
    grad[(l == 0 ? offW0 : (l == 1 ? offW1 : offW2)) + e] += s;
}

// grad[b1 | b2 | b3 | w4][c] and grad[b4] += the column sums of the CTAs' row quarters:
// CTA (c, s) of 128 threads, thread k adding parts k, k + 128, ... in order, then a
// fixed tree over the threads (the same order every step)
__global__ void __launch_bounds__(128)
    colsum_reduce_kernel(const float* __restrict__ cpart, int parts, float* __restrict__ grad, int64_t ob1,
                         int64_t ob2, int64_t ob3, int64_t ow4, int64_t ob4) {
    __shared__ float red[4];
    const int c = blockIdx.x, s = blockIdx.y, k = threadIdx.x;
    if (s == 4 && c > 0) return;  // db4: the first entry only
    float t = 0.0f;
    for (int p = k; p < parts; p += 128) t += cpart[((int64_t)p * kColSums + s) * kHid + c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if ((k & 31) == 0) red[k >> 5] = t;
    __syncthreads();
    if (k == 0) {
        const int64_t off = s == 0 ? ob1 : (s == 1 ? ob2 : (s == 2 ? ob3 : (s == 3 ? ow4 : ob4)));
        grad[off + c] += (red[0] + red[1]) + (red[2] + red[3]);
    }
}

// ---------------------------------------------------------------- inference forward
struct MlpTcArgs {
    const __nv_bfloat16* w;  // [3][128][128] W ([out][in])
    const float* params;     // FP32 master: biases, w4, b4
    int64_t off_b[3], off_w4, off_b4;
    int64_t B;
    const __nv_bfloat16* x;  // [B][128] merged input
    float* y;                // [B] output
    int measure;
    unsigned* status;
};

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
            // the sample's merged input (zero rows past B) into the operand
            const uint4* xr = reinterpret_cast<const uint4*>(a.x + (in ? b : 0) * kIn);
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const uint4 u = in ? xr[c] : make_uint4(0, 0, 0, 0);
                *reinterpret_cast<uint4*>(A + (uint32_t)(c >> 3) * kAtom + swz(i, c & 7)) = u;
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
#pragma unroll
                for (int c0 = 0; c0 < kHid; c0 += 32) {
                    float h[32];
                    tmem_ld32(taddr + (uint32_t)c0, h);
#pragma unroll
                    for (int j = 0; j < 32; ++j) h[j] = fmaxf(h[j] + bias[c0 + j], 0.0f);
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
                    a.y[b] = out_act(a.measure, acc + b4);
                }
            }
        }
    }
done:
    teardown(tmem, abort_flag, a.status);
}

// ---------------------------------------------------------------- host side
static cudaError_t set_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kTrainSmem);
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t mlp_tc_forward(ndf_model* m, int64_t B, float* y) {
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    MlpTcArgs a;
    a.w = m->wbf;
    a.params = m->params;
    a.off_b[0] = m->L.b1;
    a.off_b[1] = m->L.b2;
    a.off_b[2] = m->L.b3;
    a.off_w4 = m->L.w4;
    a.off_b4 = m->L.b4;
    a.B = B;
    a.x = m->work.x;
    a.y = y;
    a.measure = m->measure;
    a.status = m->ctx->flag.as<unsigned>() + 1;
    const int64_t tiles = (B + kTile - 1) / kTile;
    int64_t grid = m->ctx->sm_count;
    if (grid > (tiles + 1) / 2) grid = (tiles + 1) / 2;
    if (grid < 1) grid = 1;
    mlp_fwd_tc_kernel<<<(unsigned)grid, kThreads, kSmem, m->ctx->stream>>>(a);
    m->ctx->launches++;
    return cudaGetLastError();
}

cudaError_t mlp_tc_train(ndf_model* m, int64_t B, const float* target) {
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    ndf_ctx* ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    MlpTrainArgs a;
    a.w = m->wbf;
    a.params = m->params;
    a.off_b[0] = m->L.b1;
    a.off_b[1] = m->L.b2;
    a.off_b[2] = m->L.b3;
    a.off_w4 = m->L.w4;
    a.off_b4 = m->L.b4;
    a.B = B;
    a.x = m->work.x;
    a.target = target;
    a.dx = m->work.dx;
    a.wpart = m->work.wpart;
    a.cpart = m->work.cpart;
    a.loss = m->work.loss;
    a.measure = m->measure;
    a.status = ctx->flag.as<unsigned>() + 1;
    const int64_t tiles = (B + kTile - 1) / kTile;
    int64_t grid = ctx->sm_count < kMlpMaxParts ? ctx->sm_count : kMlpMaxParts;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    mlp_train_tc_kernel<<<(unsigned)grid, kTrainThreads, kTrainSmem, s>>>(a);
    wgrad_reduce_kernel<<<dim3(kHid * kHid / 256, 3), 256, 0, s>>>(m->work.wpart, (int)grid, m->grad,
                                                                  m->L.W1, m->L.W2, m->L.W3);
    colsum_reduce_kernel<<<dim3(kHid, kColSums), 128, 0, s>>>(m->work.cpart, (int)grid * 4, m->grad, m->L.b1,
                                                              m->L.b2, m->L.b3, m->L.w4, m->L.b4);
    ctx->launches += 3;
    return cudaGetLastError();
}

}  // namespace ndf

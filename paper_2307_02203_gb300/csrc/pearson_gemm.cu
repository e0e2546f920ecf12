// Batched multi-reference Pearson volumes (Sec. 3.1, Eq. 1) as a
// standardised-data GEMM on the 5th-generation tensor cores.
//
// With z_{m,v} = (y_{m,v} - mu_v) / sqrt(S_v), Eq. 1 becomes a plain inner
// product, r(ref, v) = sum_m z_{m,ref} z_{m,v}, so R reference volumes are
//   C[v][r] = sum_m Zt[v][m] * Zr[r][m]       (A = Zt: N x K, B = Zr: R x K, both K-major)
// where Zt is the standardised field stored vertex-major (members contiguous,
// zero-padded to Kp) and Zr holds the R reference rows of Zt.
//
// Precisions (error against FP64 is reported by the tests and the benchmark):
//   TF32    z rounded to TF32 once, tcgen05.mma kind::tf32, FP32 accumulate.
//   BF16x3  z = hi + lo with hi = bf16(z), lo = bf16(z - hi);
//           C = hi*hi' + hi*lo' + lo*hi' (kind::f16, bf16 inputs), FP32 accumulate.
//   FP32    one exact CUDA-core Pearson volume per reference (no tensor cores).
//
// GEMM kernel (one persistent CTA per SM, 6 warps):
//   warp 0      TMA producer: 128-vertex x 128-byte A tiles and Rpad x 128-byte
//               B tiles, 128B swizzle, into an S-stage shared-memory ring.
//   warp 1      allocates TMEM; one elected lane issues tcgen05.mma (M=128,
//               N=Rpad) into a double-buffered FP32 accumulator and commits to
//               the ring / accumulator mbarriers.
//   warps 2..5  epilogue: tcgen05.ld 32 lanes x 32 columns at a time, clamp,
//               coalesced stores out[r][v] (one warp = 32 consecutive vertices).
// The path is HBM-bound at R = 64 (about 33 flop per byte of Zt), so the ring
// keeps ~190 KB of loads in flight per SM.  No cluster multicast is used.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <vector>

#include "device_common.cuh"
#include "ndf_internal.h"

namespace ndf {

constexpr int kTileV = 128;       // vertices per tile (MMA M)
constexpr int kMaxR = 256;        // references per GEMM launch (MMA N <= 256)
constexpr int kGemmThreads = 192; // 6 warps
constexpr int kSmemBudget = 200 * 1024;

// ---------------------------------------------------------------- standardised copies
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// field [M][N] -> zt [N][Kp] (TF32) or hi/lo [N][Kp] (BF16); zero padding m >= M
template <bool BF16>
__global__ void __launch_bounds__(256)
    standardize_transpose_kernel(const float* __restrict__ field, int M, int64_t N, int Kp,
                                 const double* __restrict__ mean,
                                 const double* __restrict__ inv_norm, void* __restrict__ out_hi,
                                 void* __restrict__ out_lo) {
    __shared__ float tile[32][33];
    const int m0 = blockIdx.x * 32;
    const int64_t v0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int64_t v = v0 + tx;
    double mu = 0.0, s = 0.0;
    if (v < N) {
        mu = mean[v];
        s = inv_norm[v];
    }
    for (int r = ty; r < 32; r += 8) {
        const int m = m0 + r;
        float z = 0.0f;
        if (m < M && v < N) z = (float)(((double)field[(int64_t)m * N + v] - mu) * s);
        tile[r][tx] = z;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t vv = v0 + r;
        if (vv >= N) continue;
        const float z = tile[tx][r];
        const int64_t o = vv * Kp + m0 + tx;
        if (BF16) {
            __nv_bfloat16 h = __float2bfloat16_rn(z);
            __nv_bfloat16 l = __float2bfloat16_rn(z - __bfloat162float(h));
            static_cast<__nv_bfloat16*>(out_hi)[o] = h;
            static_cast<__nv_bfloat16*>(out_lo)[o] = l;
        } else {
            static_cast<float*>(out_hi)[o] = to_tf32(z);
        }
    }
}

// rows of the standardised copy at the reference vertices -> [Rpad][Kp], zero rows r >= R
__global__ void gather_rows_kernel(const unsigned char* __restrict__ src, int64_t row_bytes,
                                   const int64_t* __restrict__ rows, int R, int Rpad,
                                   unsigned char* __restrict__ dst) {
    const int r = blockIdx.x;
    const uint4* s = r < R ? reinterpret_cast<const uint4*>(src + rows[r] * row_bytes) : nullptr;
    uint4* d = reinterpret_cast<uint4*>(dst + (int64_t)r * row_bytes);
    for (int64_t i = threadIdx.x; i < row_bytes / 16; i += blockDim.x)
        d[i] = s ? s[i] : make_uint4(0, 0, 0, 0);
    (void)Rpad;
}

// ---------------------------------------------------------------- tcgen05 / TMA helpers
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused, swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity,
                                              volatile int* abort_flag) {
    uint32_t addr = smem_u32(bar);
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < kWaitPolls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 255) == 255 && *abort_flag) return false;
        if ((i & 1023u) == 1023u) {  // and at most kWaitNs of wall time
            const uint64_t t = global_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kWaitNs) break;
        }
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct GemmArgs {
    int64_t N;         // vertices
    int R, Rpad;       // references, padded to a multiple of 32
    int k_stages;      // Kp / elements per 128-byte row
    int stages;        // smem ring depth
    uint32_t a_bytes;  // one A tile (per hi/lo copy)
    uint32_t b_bytes;  // one B tile (per hi/lo copy)
    uint32_t idesc;
    uint32_t tmem_cols;
    float* out;        // [R][N]
    unsigned* status;
};

// ---------------------------------------------------------------- GEMM kernel
template <bool SPLIT>  // SPLIT = BF16x3 (hi/lo operands), else TF32
__global__ void __launch_bounds__(kGemmThreads, 1)
    pearson_gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mA2,
                        const __grid_constant__ CUtensorMap mB, const __grid_constant__ CUtensorMap mB2,
                        const GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned ring
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t copies = SPLIT ? 2u : 1u;
    const uint32_t stage_bytes = copies * (g.a_bytes + g.b_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)g.stages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + g.stages;
    uint64_t* acc_full = bars + 2 * g.stages;
    uint64_t* acc_empty = acc_full + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < g.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        *abort_flag = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int64_t ntiles = (g.N + kTileV - 1) / kTileV;
    if (warp == 0) {
        if (lane == 0) {  // ---- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                for (int ks = 0; ks < g.k_stages; ++ks) {
                    if (!wait_or_abort(&empty[stage], phase ^ 1u, abort_flag)) goto done;
                    unsigned char* st = smem + (size_t)stage * stage_bytes;
                    mbar_expect_tx(&full[stage], stage_bytes);
                    const int x = ks * (SPLIT ? 64 : 32);
                    tma_load_2d(st, &mA, x, (int)(t * kTileV), &full[stage]);
                    tma_load_2d(st + g.a_bytes, &mB, x, 0, &full[stage]);
                    if (SPLIT) {
                        tma_load_2d(st + g.a_bytes + g.b_bytes, &mA2, x, (int)(t * kTileV),
                                    &full[stage]);
                        tma_load_2d(st + 2 * g.a_bytes + g.b_bytes, &mB2, x, 0, &full[stage]);
                    }
                    if (++stage == g.stages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer
            int stage = 0;
            uint32_t phase = 0;
            int local = 0;
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++local) {
                const int b = local & 1;
                const uint32_t use = (uint32_t)(local >> 1);
                if (!wait_or_abort(&acc_empty[b], (use & 1u) ^ 1u, abort_flag)) goto done;
                fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(b * g.Rpad);
                for (int ks = 0; ks < g.k_stages; ++ks) {
                    if (!wait_or_abort(&full[stage], phase, abort_flag)) goto done;
                    fence_after();
                    unsigned char* st = smem + (size_t)stage * stage_bytes;
                    const uint64_t a_hi = sw128_desc(smem_u32(st));
                    const uint64_t b_hi = sw128_desc(smem_u32(st + g.a_bytes));
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {  // 4 x 32 bytes of K per 128-byte row
                        const uint32_t acc = (ks > 0 || kk > 0) ? 1u : 0u;
                        const uint64_t adv = (uint64_t)(kk * 2);  // 32 B >> 4
                        if (SPLIT) {
                            const uint64_t a_lo = sw128_desc(smem_u32(st + g.a_bytes + g.b_bytes));
                            const uint64_t b_lo =
                                sw128_desc(smem_u32(st + 2 * g.a_bytes + g.b_bytes));
                            mma_f16(d_tmem, a_hi + adv, b_hi + adv, g.idesc, acc);
                            mma_f16(d_tmem, a_hi + adv, b_lo + adv, g.idesc, 1u);
                            mma_f16(d_tmem, a_lo + adv, b_hi + adv, g.idesc, 1u);
                        } else {
                            mma_tf32(d_tmem, a_hi + adv, b_hi + adv, g.idesc, acc);
                        }
                    }
                    mma_commit(&empty[stage]);
                    if (++stage == g.stages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                mma_commit(&acc_full[b]);
            }
        }
    } else {  // ---- epilogue warps 2..5: TMEM lane quarter = warp % 4
        const int q = warp & 3;
        int local = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++local) {
            const int b = local & 1;
            const uint32_t use = (uint32_t)(local >> 1);
            if (!wait_or_abort(&acc_full[b], use & 1u, abort_flag)) break;
            fence_after();
            const int64_t v = t * kTileV + q * 32 + lane;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * g.Rpad);
            for (int c0 = 0; c0 < g.Rpad; c0 += 32) {
                float val[32];
                tmem_ld32(taddr + (uint32_t)c0, val);
                if (v < g.N) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int r = c0 + j;
                        if (r < g.R) {
                            float x = fminf(1.0f, fmaxf(-1.0f, val[j]));
                            __stcs(g.out + (int64_t)r * g.N + v, x);
                        }
                    }
                }
            }
            fence_before();
            mbar_arrive(&acc_empty[b]);
        }
    }
done:
    if (*abort_flag && threadIdx.x == 0) report(g.status, kDevTimeout);
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(g.tmem_cols)
                     : "memory");
    }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D K-major map: rows x Kp elements, box = box_rows x 128 bytes, 128B swizzle
static bool make_map(CUtensorMap* m, const void* base, bool bf16, int64_t rows, int Kp,
                     int box_rows) {
    auto enc = get_encoder();
    if (!enc) return false;
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Builds the standardised copy of a field for one precision (once per field).
static ndf_status ensure_standardized(ndf_ctx* ctx, Field& f, bool bf16) {
    if (bf16 ? (f.z_hi != nullptr) : (f.z_tf32 != nullptr)) return NDF_OK;
    const int Kp = (int)((f.M + 63) / 64 * 64);
    const size_t esz = bf16 ? 2 : 4;
    const size_t bytes = (size_t)f.N * (size_t)Kp * esz;
    void* hi = nullptr;
    void* lo = nullptr;
    cudaError_t e = cudaMalloc(&hi, bytes);
    if (e == cudaSuccess && bf16) e = cudaMalloc(&lo, bytes);
    if (e != cudaSuccess) {
        if (hi) cudaFree(hi);
        return cuda_fail(ctx, e, "standardised copy allocation");
    }
    dim3 grid((unsigned)(Kp / 32), (unsigned)((f.N + 31) / 32));
    if (bf16)
        standardize_transpose_kernel<true><<<grid, 256, 0, ctx->stream>>>(
            f.data, (int)f.M, f.N, Kp, f.mean, f.inv_norm, hi, lo);
    else
        standardize_transpose_kernel<false><<<grid, 256, 0, ctx->stream>>>(
            f.data, (int)f.M, f.N, Kp, f.mean, f.inv_norm, hi, nullptr);
    ctx->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(hi);
        if (lo) cudaFree(lo);
        return cuda_fail(ctx, e, "standardisation launch");
    }
    f.Kp = Kp;
    if (bf16) {
        f.z_hi = hi;
        f.z_lo = lo;
    } else {
        f.z_tf32 = hi;
    }
    return NDF_OK;
}

static ndf_status gemm_chunk(ndf_ctx* ctx, const Field& rf, const Field& qf, bool bf16,
                             const int64_t* d_refs, int R, float* out) {
    const int Rpad = (R + 31) / 32 * 32;
    const int Kp = qf.Kp;
    const size_t esz = bf16 ? 2 : 4;
    const int64_t row_bytes = (int64_t)Kp * (int64_t)esz;
    cudaError_t e = ctx->zr.reserve((size_t)(bf16 ? 2 : 1) * (size_t)Rpad * (size_t)row_bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reference rows");
    unsigned char* zr = ctx->zr.as<unsigned char>();
    unsigned char* zr_lo = zr + (size_t)Rpad * (size_t)row_bytes;
    gather_rows_kernel<<<Rpad, 256, 0, ctx->stream>>>(
        static_cast<const unsigned char*>(bf16 ? rf.z_hi : rf.z_tf32), row_bytes, d_refs, R, Rpad,
        zr);
    ctx->launches++;
    if (bf16) {
        gather_rows_kernel<<<Rpad, 256, 0, ctx->stream>>>(
            static_cast<const unsigned char*>(rf.z_lo), row_bytes, d_refs, R, Rpad, zr_lo);
        ctx->launches++;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "reference gather");

    CUtensorMap mA, mA2, mB, mB2;
    const void* a_hi = bf16 ? qf.z_hi : qf.z_tf32;
    const void* a_lo = bf16 ? qf.z_lo : qf.z_tf32;
    if (!make_map(&mA, a_hi, bf16, qf.N, Kp, kTileV) || !make_map(&mA2, a_lo, bf16, qf.N, Kp, kTileV) ||
        !make_map(&mB, zr, bf16, Rpad, Kp, Rpad) ||
        !make_map(&mB2, bf16 ? zr_lo : zr, bf16, Rpad, Kp, Rpad))
        return fail(ctx, NDF_ERR_CUDA, "tensor map encoding failed");

    GemmArgs g;
    g.N = qf.N;
    g.R = R;
    g.Rpad = Rpad;
    g.k_stages = Kp / (bf16 ? 64 : 32);
    g.a_bytes = kTileV * 128;
    g.b_bytes = (uint32_t)Rpad * 128;
    const uint32_t stage_bytes = (bf16 ? 2u : 1u) * (g.a_bytes + g.b_bytes);
    g.stages = (int)((kSmemBudget - 2048) / stage_bytes);
    if (g.stages > 8) g.stages = 8;
    if (g.stages < 2) return fail(ctx, NDF_ERR_ARG, "too many references for one GEMM tile");
    const uint32_t fmt = bf16 ? 1u : 2u;  // A/B type: BF16 (kind::f16) / TF32 (kind::tf32)
    g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(Rpad >> 3) << 17) |
              ((uint32_t)(kTileV >> 4) << 24);
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * Rpad)) cols <<= 1;
    g.tmem_cols = cols;
    g.out = out;
    g.status = ctx->flag.as<unsigned>() + 1;
    const size_t smem = 1024 + (size_t)g.stages * stage_bytes + 256;
    const int64_t ntiles = (qf.N + kTileV - 1) / kTileV;
    int grid = ctx->sm_count;
    if (grid > ntiles) grid = (int)ntiles;
    if (bf16) {
        e = cudaFuncSetAttribute(pearson_gemm_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            pearson_gemm_kernel<true><<<grid, kGemmThreads, smem, ctx->stream>>>(mA, mA2, mB, mB2, g);
    } else {
        e = cudaFuncSetAttribute(pearson_gemm_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            pearson_gemm_kernel<false><<<grid, kGemmThreads, smem, ctx->stream>>>(mA, mA2, mB, mB2, g);
    }
    ctx->launches++;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pearson gemm launch");
    return NDF_OK;
}

}  // namespace ndf

using namespace ndf;

extern "C" ndf_status ndf_pearson_batch(ndf_ctx* ctx, int ref_field, int query_field,
                                        const int64_t* ref_idx, int R, ndf_precision prec,
                                        float* out) {
    if (!ctx) return NDF_ERR_ARG;
    if (!ref_idx || R < 1) return fail(ctx, NDF_ERR_ARG, "need R >= 1 reference indices");
    const Field *rf, *qf;
    ndf_status st = check_pair(ctx, ref_field, query_field, 0, &rf, &qf);
    if (st != NDF_OK) return st;
    for (int i = 0; i < R; ++i)
        if (ref_idx[i] < 0 || ref_idx[i] >= rf->N)
            return fail(ctx, NDF_ERR_ARG, "ref_idx[%d] out of range", i);
    if (prec != NDF_PREC_FP32 && prec != NDF_PREC_TF32 && prec != NDF_PREC_BF16X3)
        return fail(ctx, NDF_ERR_ARG, "unknown precision %d", (int)prec);
    cudaSetDevice(ctx->device);
    const size_t bytes = sizeof(float) * (size_t)R * (size_t)qf->N;
    void* dev_out;
    bool is_host;
    if ((st = resolve_out(ctx, out, bytes, &dev_out, &is_host)) != NDF_OK) return st;
    float* o = static_cast<float*>(dev_out);
    if (prec == NDF_PREC_FP32) {
        for (int i = 0; i < R; ++i) {
            cudaError_t e = launch_pearson(ctx, *rf, *qf, ref_idx[i], o + (size_t)i * qf->N);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "pearson launch");
        }
        return finish_out(ctx, out, dev_out, bytes, is_host);
    }
    const bool bf16 = prec == NDF_PREC_BF16X3;
    Field& rfm = ctx->fields[ref_field];
    Field& qfm = ctx->fields[query_field];
    if ((st = ensure_standardized(ctx, rfm, bf16)) != NDF_OK) return st;
    if ((st = ensure_standardized(ctx, qfm, bf16)) != NDF_OK) return st;
    cudaError_t e = ctx->refidx.reserve(sizeof(int64_t) * (size_t)R);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->refidx.ptr, ref_idx, sizeof(int64_t) * (size_t)R,
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reference index upload");
    const int64_t* d_refs = ctx->refidx.as<int64_t>();
    for (int r0 = 0; r0 < R; r0 += kMaxR) {
        const int rc = R - r0 < kMaxR ? R - r0 : kMaxR;
        if ((st = gemm_chunk(ctx, rfm, qfm, bf16, d_refs + r0, rc, o + (size_t)r0 * qf->N)) !=
            NDF_OK)
            return st;
    }
    // the host-to-device copy of ref_idx above is from pageable memory, so it has
    // completed before return; the device buffer stays valid until the next call
    return finish_out(ctx, out, dev_out, bytes, is_host);
}

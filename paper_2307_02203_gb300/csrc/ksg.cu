// KSG mutual-information volume: algorithm 1 of the k-NN estimator cited in
// Sec. 3.2 (timed on the CPU in Sec. 6.2, Table 1), for the reference vertex
// against every vertex of the query field.
//
// Per pair (x = reference column, y = query column, M joint samples):
//   d_ij  = max(|x_i - x_j|, |y_i - y_j|)           FP32, exactly rounded
//   eps_i = k-th smallest d_ij over j != i
//         = (k+1)-th smallest over all j (the self distance 0 is always the smallest)
//   nx_i  = #{j != i : |x_i - x_j| < eps_i},  ny_i likewise
//   I     = psi(k) + psi(M) - (1/M) sum_i [psi(nx_i + 1) + psi(ny_i + 1)]   (FP64)
//
// GPU design:
//   stage   one CTA sorts the reference column once per launch (values + member ids).
//   volume  persistent CTAs walk tiles of VT query vertices.  A tile's y columns
//           are loaded once (coalesced across the VT vertices of each member row).
//           For each vertex the CTA builds the joint points in x-sorted order in a
//           doubled, padded shared array; thread t owns the 4 consecutive sorted
//           points 4t..4t+3 (and 4(t+T).. for M > 4T) and visits every other point exactly once, outward in
//           x-order (nearest in x first, wrapping through the doubled array), so
//           the running top-(k+1) distances in registers tighten early and the
//           insert branch is rare.  Insertion is a branch-free min/max network.
//           Counts: binary search in the sorted x (shared by all pairs) and in the
//           query column's sorted copy (sorted once per field); the search
//           predicates are the same FP32 |difference| < eps tests, which are
//           monotone in sorted order.  The digamma sum is FP64, block-reduced.
#include <float.h>
#include <limits.h>
#include <math.h>

#include "device_common.cuh"
#include "ksg_common.cuh"
#include "ndf_internal.h"

namespace ndf {

constexpr int kKsgPts = 4;  // sorted points owned by one thread

__host__ __device__ __forceinline__ int padi(int i) { return i + (i >> 2); }  // bank-conflict padding

// ---------------------------------------------------------------- stage (a2)
__global__ void __launch_bounds__(1024) ksg_stage_kernel(const float* __restrict__ field, int M,
                                                          int64_t N, int64_t ref,
                                                          float* __restrict__ xs_out,
                                                          int* __restrict__ perm_out) {
    __shared__ float key[kKsgMaxM];
    __shared__ int val[kKsgMaxM];
    int n2 = 1;
    while (n2 < M) n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        key[i] = i < M ? field[(int64_t)i * N + ref] : FLT_MAX;
        val[i] = i < M ? i : INT_MAX;
    }
    __syncthreads();
    for (int kk = 2; kk <= n2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    bool up = (i & kk) == 0;
                    float a = key[i], b = key[l];
                    int va = val[i], vb = val[l];
                    bool gt = (a > b) || (a == b && va > vb);
                    if (gt == up) {
                        key[i] = b; key[l] = a;
                        val[i] = vb; val[l] = va;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        xs_out[i] = key[i];
        perm_out[i] = val[i];
    }
}

__device__ __forceinline__ unsigned long long pack_f2(float2 v) {
    return ((unsigned long long)__float_as_uint(v.y) << 32) | __float_as_uint(v.x);
}

// (a.x - b.x, a.y - b.y), each rounded to nearest like a scalar FP32 subtract
__device__ __forceinline__ float2 sub_f32x2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return make_float2(__uint_as_float((unsigned)d), __uint_as_float((unsigned)(d >> 32)));
}

struct KsgArgs {
    const float* field;  // query field [M][N]
    const float* sorted; // the query field's columns sorted ascending [M][N]
    int M;
    int k;
    int n2;              // power of two >= M
    int VT;              // vertices per tile
    int64_t N;
    int64_t v_begin, v_end;
    const float* xs;     // sorted reference values [M]
    const int* perm;     // member of each sorted position [M]
    const double* psi;   // psi(n), n <= M + 1
    float* out;          // out[v - v_begin]
    double* dbg_mi;      // debug (single vertex) outputs, may be null
    float* dbg_eps;
    int32_t* dbg_nx;
    int32_t* dbg_ny;
};

// shared-memory carve-up (bytes) for a given M and VT
struct KsgSmem {
    size_t xs, perm, ytile, ystile, pts, red, total;
    __host__ __device__ KsgSmem(int M, int n2, int VT) {
        size_t o = 0;
        red = o; o += 32 * sizeof(double);
        xs = o; o += sizeof(float) * (size_t)M;
        perm = o; o += sizeof(int) * (size_t)M;
        o = (o + 15) & ~size_t(15);
        ytile = o; o += sizeof(float) * (size_t)M * (size_t)VT;
        ystile = o; o += sizeof(float) * (size_t)M * (size_t)VT;
        o = (o + 15) & ~size_t(15);
        pts = o; o += sizeof(float2) * (size_t)(padi(2 * M) + 4);
        total = o;
        (void)n2;
    }
};

// ---------------------------------------------------------------- volume (a4-a6)
constexpr int kKsgMaxThreads = 512;

template <int K1>
__global__ void __launch_bounds__(kKsgMaxThreads) ksg_volume_kernel(KsgArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const KsgSmem L(A.M, A.n2, A.VT);
    double* red = reinterpret_cast<double*>(smem + L.red);
    float* xs = reinterpret_cast<float*>(smem + L.xs);
    int* perm = reinterpret_cast<int*>(smem + L.perm);
    float* ytile = reinterpret_cast<float*>(smem + L.ytile);
    float2* pts = reinterpret_cast<float2*>(smem + L.pts);
    float* ystile = reinterpret_cast<float*>(smem + L.ystile);

    const int M = A.M, T = blockDim.x, tid = threadIdx.x;
    const int64_t N = A.N;
    for (int i = tid; i < M; i += T) {
        xs[i] = A.xs[i];
        perm[i] = A.perm[i];
    }
    const double psi_k = A.psi[A.k], psi_M = A.psi[M];

    const int64_t nv = A.v_end - A.v_begin;
    const int64_t ntiles = (nv + A.VT - 1) / A.VT;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t vt0 = A.v_begin + tile * A.VT;
        const int vcount = (int)(A.v_end - vt0 < A.VT ? A.v_end - vt0 : A.VT);
        __syncthreads();  // previous tile's readers are done with ytile
        for (int idx = tid; idx < M * A.VT; idx += T) {
            int m = idx / A.VT, p = idx - m * A.VT;
            ytile[p * M + m] = p < vcount ? __ldcs(A.field + (int64_t)m * N + vt0 + p) : 0.0f;
            ystile[p * M + m] = p < vcount ? __ldcs(A.sorted + (int64_t)m * N + vt0 + p) : 0.0f;
        }
        for (int p = 0; p < vcount; ++p) {
            const float* ycol = ytile + p * M;
            const float* ys = ystile + p * M;  // the column, sorted (for n_y)
            __syncthreads();  // tiles ready / previous pair done with pts
            for (int s = tid; s < M; s += T) {
                float2 q = make_float2(xs[s], ycol[perm[s]]);
                pts[padi(s)] = q;
                pts[padi(s + M)] = q;
            }
            __syncthreads();

            double acc = 0.0;
            for (int base = 0; base < M; base += kKsgPts * T) {
                const int b0 = base + kKsgPts * tid;
                const int n_own = M - b0 >= kKsgPts ? kKsgPts : (M - b0 > 0 ? M - b0 : 0);
                const int R = (M - n_own + 1) >> 1, Lc = (M - n_own) >> 1;
                // ---- joint k-NN: top-(k+1) distances (self included) per owned point.
                // Per candidate: one packed FP32 subtract gives (dx, dy) for a point,
                // d = max(|dx|, |dy|) is one min/max, and the threshold test moves to
                // the FMA pipe as u = d - t (exactly negative iff d < t: no flush to
                // zero); the 4 tests merge with a min tree into one compare.
                unsigned long long P[kKsgPts];
                float px[kKsgPts], py[kKsgPts];
                float a[kKsgPts][K1];
#pragma unroll
                for (int q = 0; q < kKsgPts; ++q) {
                    // a missing point sits at +inf: its distances are +inf, never inserted
                    float2 pq = q < n_own ? pts[padi(b0 + q)] : make_float2(INFINITY, INFINITY);
                    px[q] = pq.x;
                    py[q] = pq.y;
                    P[q] = pack_f2(pq);
#pragma unroll
                    for (int j = 0; j < K1; ++j) a[q][j] = FLT_MAX;
                }
                auto visit = [&](float2 c) {
                    const unsigned long long C = pack_f2(c);
                    float d[kKsgPts], u[kKsgPts];
#pragma unroll
                    for (int q = 0; q < kKsgPts; ++q) {
                        const float2 dd = sub_f32x2(P[q], C);
                        d[q] = fmaxf(fabsf(dd.x), fabsf(dd.y));
                        u[q] = d[q] - a[q][K1 - 1];
                    }
                    if (fminf(fminf(u[0], u[1]), fminf(u[2], u[3])) < 0.0f) {
#pragma unroll
                        for (int q = 0; q < kKsgPts; ++q) topk_insert<K1>(a[q], d[q]);
                    }
                };
                if (n_own > 0) {
#pragma unroll
                    for (int c = 0; c < kKsgPts; ++c)
                        if (c < n_own) visit(pts[padi(b0 + c)]);
                    const int rb = b0 + n_own - 1, lb = b0 + M;
                    for (int o = 1; o <= R; ++o) {
                        visit(pts[padi(rb + o)]);
                        if (o <= Lc) visit(pts[padi(lb - o)]);
                    }
                }
                // ---- marginal counts and the digamma sum
#pragma unroll
                for (int q = 0; q < kKsgPts; ++q) {
                    if (q < n_own) {
                        const float e = a[q][K1 - 1];
                        const int self = e > 0.0f ? 1 : 0;
                        const int cx = count_within(xs, M, px[q], e) - self;
                        const int cy = count_within(ys, M, py[q], e) - self;
                        acc += A.psi[cx + 1] + A.psi[cy + 1];
                        if (A.dbg_eps) {
                            const int mi = perm[b0 + q];
                            A.dbg_eps[mi] = e;
                            A.dbg_nx[mi] = cx;
                            A.dbg_ny[mi] = cy;
                        }
                    }
                }
            }
            const double tot = block_sum(acc, red);
            if (tid == 0) {
                const double mi = psi_k + psi_M - tot / (double)M;
                const int64_t v = vt0 + p;
                A.out[v - A.v_begin] = (float)mi;
                if (A.dbg_mi) *A.dbg_mi = mi;
            }
        }
    }
}

template <int K1>
static cudaError_t launch_ksg_k(ndf_ctx* ctx, const KsgArgs& A, int threads, size_t smem,
                                int64_t ntiles) {
    cudaError_t e = cudaFuncSetAttribute(ksg_volume_kernel<K1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ksg_volume_kernel<K1>, threads,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)ctx->sm_count * per_sm;
    if (grid > ntiles) grid = ntiles;
    ksg_volume_kernel<K1><<<(unsigned)grid, threads, smem, ctx->stream>>>(A);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_ksg(ndf_ctx* ctx, const Field& rf, const Field& qf, int64_t ref_idx, int k,
                       int64_t v_begin, int64_t v_end, float* out, double* dbg_mi, float* dbg_eps,
                       int32_t* dbg_nx, int32_t* dbg_ny) {
    const int M = (int)rf.M;
    cudaError_t e = ctx->stage_x.reserve(sizeof(float) * (size_t)M);
    if (e == cudaSuccess) e = ctx->stage_perm.reserve(sizeof(int) * (size_t)M);
    if (e != cudaSuccess) return e;
    ksg_stage_kernel<<<1, 1024, 0, ctx->stream>>>(rf.data, M, rf.N, ref_idx,
                                                   ctx->stage_x.as<float>(),
                                                   ctx->stage_perm.as<int>());
    ctx->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    KsgArgs A;
    A.field = qf.data;
    A.sorted = qf.sorted;
    A.M = M;
    A.k = k;
    A.n2 = 1;
    while (A.n2 < M) A.n2 <<= 1;
    A.N = qf.N;
    A.v_begin = v_begin;
    A.v_end = v_end;
    A.xs = ctx->stage_x.as<float>();
    A.perm = ctx->stage_perm.as<int>();
    A.psi = ctx->psi.as<double>();
    A.out = out;
    A.dbg_mi = dbg_mi;
    A.dbg_eps = dbg_eps;
    A.dbg_nx = dbg_nx;
    A.dbg_ny = dbg_ny;
    int threads = ((M + kKsgPts - 1) / kKsgPts + 31) / 32 * 32;
    if (threads > kKsgMaxThreads) threads = kKsgMaxThreads;
    // vertices per tile: up to 8, bounded by a ~96 KB shared-memory budget
    int VT = 8;
    while (VT > 1 && KsgSmem(M, A.n2, VT).total > 96 * 1024) VT >>= 1;
    A.VT = VT;
    size_t smem = KsgSmem(M, A.n2, VT).total;
    int64_t ntiles = (v_end - v_begin + VT - 1) / VT;
    switch (k + 1) {
        case 2: return launch_ksg_k<2>(ctx, A, threads, smem, ntiles);
        case 3: return launch_ksg_k<3>(ctx, A, threads, smem, ntiles);
        case 4: return launch_ksg_k<4>(ctx, A, threads, smem, ntiles);
        case 5: return launch_ksg_k<5>(ctx, A, threads, smem, ntiles);
        case 6: return launch_ksg_k<6>(ctx, A, threads, smem, ntiles);
        case 7: return launch_ksg_k<7>(ctx, A, threads, smem, ntiles);
        case 8: return launch_ksg_k<8>(ctx, A, threads, smem, ntiles);
        case 9: return launch_ksg_k<9>(ctx, A, threads, smem, ntiles);
        case 10: return launch_ksg_k<10>(ctx, A, threads, smem, ntiles);
        case 11: return launch_ksg_k<11>(ctx, A, threads, smem, ntiles);
        case 12: return launch_ksg_k<12>(ctx, A, threads, smem, ntiles);
        case 13: return launch_ksg_k<13>(ctx, A, threads, smem, ntiles);
        case 14: return launch_ksg_k<14>(ctx, A, threads, smem, ntiles);
        case 15: return launch_ksg_k<15>(ctx, A, threads, smem, ntiles);
        case 16: return launch_ksg_k<16>(ctx, A, threads, smem, ntiles);
        case 17: return launch_ksg_k<17>(ctx, A, threads, smem, ntiles);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ndf

// KSG mutual information (algorithm 1 of the estimator cited in Sec. 3.2), exact
// pruned search, for one or many reference vertices.
//
// Same estimator and the same FP32 arithmetic as the brute-force kernel; only
// the candidates that cannot change the result are skipped.  With the joint
// points in order of the reference value x, a point's candidates are scanned
// outward on each side, and a side stops at the first candidate whose x-gap
// fl(x_j - x_i) (non-negative in sorted order, equal to |fl(x_i - x_j)|)
// reaches the current (k+1)-th smallest distance: every later candidate on that
// side has a gap at least as large, hence a max-norm distance at least as large,
// and an insert needs a strictly smaller one.  The threshold only shrinks, so
// the rule stays valid and eps_i is exactly the brute-force value.
//
// Scan lengths differ a lot between points (the sparse tails of the x
// distribution scan far), so points are handed to threads dynamically from a
// shared counter.  The marginal counts and the digamma sum run afterwards as a
// separate, evenly split phase.  The query column's sorted copy (for n_y) comes
// from the field's sorted columns (sorted once per field); G references share
// each loaded column tile, so one launch covers R references: work items are
// (reference group, vertex tile).
#include <float.h>
#include <limits.h>

#include "device_common.cuh"
#include "ksg_common.cuh"
#include "ndf_internal.h"

namespace ndf {

// one CTA per reference: sorted reference values and their member ids
__global__ void __launch_bounds__(1024)
    ksg_stage_multi_kernel(const float* __restrict__ field, int M, int64_t N,
                           const int64_t* __restrict__ refs, float* __restrict__ xs_all,
                           int* __restrict__ perm_all) {
    __shared__ float key[kKsgMaxM];
    __shared__ int val[kKsgMaxM];
    const int64_t ref = refs[blockIdx.x];
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
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & kk) == 0;
                    const float a = key[i], b = key[l];
                    const int va = val[i], vb = val[l];
                    const bool gt = (a > b) || (a == b && va > vb);
                    if (gt == up) {
                        key[i] = b; key[l] = a;
                        val[i] = vb; val[l] = va;
                    }
                }
            }
            __syncthreads();
        }
    }
    float* xs = xs_all + (int64_t)blockIdx.x * M;
    int* pm = perm_all + (int64_t)blockIdx.x * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        xs[i] = key[i];
        pm[i] = val[i];
    }
}

struct KsgPArgs {
    const float* field;  // query field [M][N]
    const float* sorted; // its columns sorted ascending [M][N]
    int M, k, n2, VT, G, R;
    int64_t N, v_begin, v_end;
    const float* xs_all; // [R][M] sorted reference values
    const int* perm_all; // [R][M] member id of each sorted position
    const double* psi;
    float* out;          // out[r * out_stride + (v - v_begin)]
    int64_t out_stride;
    double* dbg_mi;      // debug outputs for (reference 0, vertex v_begin), may be null
    float* dbg_eps;
    int32_t* dbg_nx;
    int32_t* dbg_ny;
    unsigned long long* evals;  // distance evaluations performed, may be null
};

struct KsgPSmem {
    size_t red, next, xsg, permg, ytile, ystile, pts, eps, total;
    __host__ __device__ KsgPSmem(int M, int n2, int VT, int G) {
        size_t o = 0;
        red = o; o += 33 * sizeof(double);
        next = o; o += 16;
        xsg = o; o += sizeof(float) * (size_t)M * G;
        permg = o; o += sizeof(int) * (size_t)M * G;
        o = (o + 15) & ~size_t(15);
        ytile = o; o += sizeof(float) * (size_t)M * VT;
        ystile = o; o += sizeof(float) * (size_t)M * VT;
        (void)n2;
        o = (o + 15) & ~size_t(15);
        pts = o; o += sizeof(float2) * (size_t)M;
        eps = o; o += sizeof(float) * (size_t)M;
        total = o;
    }
};

constexpr int kKsgPThreads = 256;

template <int K1>
__global__ void __launch_bounds__(kKsgPThreads) ksg_pruned_kernel(KsgPArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const KsgPSmem L(A.M, A.n2, A.VT, A.G);
    double* red = reinterpret_cast<double*>(smem + L.red);
    int* next = reinterpret_cast<int*>(smem + L.next);
    float* xsg = reinterpret_cast<float*>(smem + L.xsg);
    int* permg = reinterpret_cast<int*>(smem + L.permg);
    float* ytile = reinterpret_cast<float*>(smem + L.ytile);
    float* ystile = reinterpret_cast<float*>(smem + L.ystile);
    float2* pts = reinterpret_cast<float2*>(smem + L.pts);
    float* eps = reinterpret_cast<float*>(smem + L.eps);

    const int M = A.M, T = blockDim.x, tid = threadIdx.x;
    const int64_t N = A.N;
    const int64_t nv = A.v_end - A.v_begin;
    const int64_t tiles = (nv + A.VT - 1) / A.VT;
    const int groups = (A.R + A.G - 1) / A.G;
    const double psi_k = A.psi[A.k], psi_M = A.psi[M];
    unsigned long long my_evals = 0;
    int loaded_group = -1;

    for (int64_t item = blockIdx.x; item < (int64_t)groups * tiles; item += gridDim.x) {
        const int group = (int)(item / tiles);
        const int64_t tile = item % tiles;
        const int r0 = group * A.G;
        const int gcount = A.R - r0 < A.G ? A.R - r0 : A.G;
        const int64_t vt0 = A.v_begin + tile * A.VT;
        const int vcount = (int)(A.v_end - vt0 < A.VT ? A.v_end - vt0 : A.VT);
        __syncthreads();  // the previous item is done with every shared buffer
        if (group != loaded_group) {
            for (int i = tid; i < gcount * M; i += T) {
                xsg[i] = A.xs_all[(int64_t)r0 * M + i];
                permg[i] = A.perm_all[(int64_t)r0 * M + i];
            }
            loaded_group = group;
        }
        for (int idx = tid; idx < M * A.VT; idx += T) {
            const int m = idx / A.VT, p = idx - m * A.VT;
            ytile[p * M + m] = p < vcount ? __ldcs(A.field + (int64_t)m * N + vt0 + p) : 0.0f;
            ystile[p * M + m] = p < vcount ? __ldcs(A.sorted + (int64_t)m * N + vt0 + p) : 0.0f;
        }
        for (int p = 0; p < vcount; ++p) {
            const float* ycol = ytile + p * M;
            __syncthreads();
            const float* ys = ystile + p * M;  // the column, sorted (for n_y)
            for (int g = 0; g < gcount; ++g) {
                const float* xs = xsg + (size_t)g * M;
                const int* perm = permg + (size_t)g * M;
                for (int s = tid; s < M; s += T) pts[s] = make_float2(xs[s], ycol[perm[s]]);
                if (tid == 0) *next = T;
                __syncthreads();
                // ---- phase 1: eps of every point.  One flat loop: each pass either
                // visits one candidate of the lane's point or, when both sides of
                // that point have stopped, records eps and takes the next point from
                // the shared counter, so lanes never wait for a warp-mate's long
                // scan.  Points are handed out from both ends of the x order first
                // (the sparse tails scan longest), the middle last.
                {
                    auto point_of = [M](int t) { return (t & 1) ? M - 1 - (t >> 1) : (t >> 1); };
                    int t = tid;
                    int s = t < M ? point_of(t) : M;
                    float a[K1];
                    float2 me = make_float2(0.0f, 0.0f);
                    int jr = 0, jl = 0;
                    bool on_r = false, on_l = false, tog = false;
                    auto start = [&](int q) {
                        a[0] = 0.0f;  // the point itself
#pragma unroll
                        for (int j = 1; j < K1; ++j) a[j] = FLT_MAX;
                        me = pts[q];
                        jr = q + 1;
                        jl = q - 1;
                        on_r = jr < M;
                        on_l = jl >= 0;
                    };
                    if (t < M) start(s);
                    while (t < M) {
                        if (on_r || on_l) {
                            const bool right = on_r && (!on_l || tog);
                            tog = !tog;
                            const float2 c = pts[right ? jr : jl];
                            const float gap = right ? c.x - me.x : me.x - c.x;
                            if (gap >= a[K1 - 1]) {
                                if (right) on_r = false;
                                else on_l = false;
                            } else {
                                const float d = fmaxf(gap, fabsf(c.y - me.y));
                                if (d < a[K1 - 1]) topk_insert<K1>(a, d);
                                ++my_evals;
                                if (right) on_r = ++jr < M;
                                else on_l = --jl >= 0;
                            }
                        } else {
                            eps[s] = a[K1 - 1];
                            t = atomicAdd(next, 1);
                            if (t < M) {
                                s = point_of(t);
                                start(s);
                            }
                        }
                    }
                }
                __syncthreads();
                // ---- phase 2: marginal counts and the digamma sum
                double acc = 0.0;
                const bool dbg = A.dbg_eps && r0 + g == 0 && p == 0 && tile == 0;
                for (int q = tid; q < M; q += T) {
                    const float e = eps[q];
                    const int self = e > 0.0f ? 1 : 0;
                    const float2 me = pts[q];
                    const int cx = count_within(xs, M, me.x, e) - self;
                    const int cy = count_within(ys, M, me.y, e) - self;
                    acc += A.psi[cx + 1] + A.psi[cy + 1];
                    if (dbg) {
                        const int mi = perm[q];
                        A.dbg_eps[mi] = e;
                        A.dbg_nx[mi] = cx;
                        A.dbg_ny[mi] = cy;
                    }
                }
                const double tot = block_sum(acc, red);
                if (tid == 0) {
                    const double mi = psi_k + psi_M - tot / (double)M;
                    const int64_t v = vt0 + p;
                    A.out[(int64_t)(r0 + g) * A.out_stride + (v - A.v_begin)] = (float)mi;
                    if (dbg && A.dbg_mi) *A.dbg_mi = mi;
                }
                __syncthreads();  // pts / eps are rebuilt for the next reference
            }
        }
    }
    if (A.evals) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_evals += __shfl_xor_sync(0xffffffffu, my_evals, o);
        if ((tid & 31) == 0) atomicAdd(A.evals, my_evals);
    }
}

template <int K1>
static cudaError_t launch_pruned_k(ndf_ctx* ctx, const KsgPArgs& A, size_t smem, int64_t items) {
    cudaError_t e = cudaFuncSetAttribute(ksg_pruned_kernel<K1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ksg_pruned_kernel<K1>, kKsgPThreads,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)ctx->sm_count * per_sm;
    if (grid > items) grid = items;
    ksg_pruned_kernel<K1><<<(unsigned)grid, kKsgPThreads, smem, ctx->stream>>>(A);
    ctx->launches++;
    return cudaGetLastError();
}

// Pruned KSG for R references (device ids in d_refs) over query vertices
// [v_begin, v_end): out[r * out_stride + (v - v_begin)].  G references share a
// CTA (one y sort per vertex), VT vertices per tile.
cudaError_t launch_ksg_pruned(ndf_ctx* ctx, const Field& rf, const Field& qf, const int64_t* d_refs,
                              int R, int k, int64_t v_begin, int64_t v_end, float* out,
                              int64_t out_stride, int G, int VT, double* dbg_mi, float* dbg_eps,
                              int32_t* dbg_nx, int32_t* dbg_ny, unsigned long long* evals) {
    const int M = (int)rf.M;
    cudaError_t e = ctx->stage_x.reserve(sizeof(float) * (size_t)M * (size_t)R);
    if (e == cudaSuccess) e = ctx->stage_perm.reserve(sizeof(int) * (size_t)M * (size_t)R);
    if (e != cudaSuccess) return e;
    ksg_stage_multi_kernel<<<R, 1024, 0, ctx->stream>>>(rf.data, M, rf.N, d_refs,
                                                         ctx->stage_x.as<float>(),
                                                         ctx->stage_perm.as<int>());
    ctx->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    KsgPArgs A;
    A.field = qf.data;
    A.sorted = qf.sorted;
    A.M = M;
    A.k = k;
    A.n2 = 1;
    while (A.n2 < M) A.n2 <<= 1;
    if (G < 1) G = 1;
    if (G > R) G = R;
    if (VT < 1) VT = 1;
    // keep the shared-memory footprint within ~110 KB (two CTAs per SM)
    while (G > 1 && KsgPSmem(M, A.n2, VT, G).total > 110 * 1024) G >>= 1;
    while (VT > 1 && KsgPSmem(M, A.n2, VT, G).total > 110 * 1024) VT >>= 1;
    A.G = G;
    A.VT = VT;
    A.R = R;
    A.N = qf.N;
    A.v_begin = v_begin;
    A.v_end = v_end;
    A.xs_all = ctx->stage_x.as<float>();
    A.perm_all = ctx->stage_perm.as<int>();
    A.psi = ctx->psi.as<double>();
    A.out = out;
    A.out_stride = out_stride;
    A.dbg_mi = dbg_mi;
    A.dbg_eps = dbg_eps;
    A.dbg_nx = dbg_nx;
    A.dbg_ny = dbg_ny;
    A.evals = evals;
    const size_t smem = KsgPSmem(M, A.n2, VT, G).total;
    const int64_t items = (int64_t)((R + G - 1) / G) * ((v_end - v_begin + VT - 1) / VT);
    switch (k + 1) {
        case 2: return launch_pruned_k<2>(ctx, A, smem, items);
        case 3: return launch_pruned_k<3>(ctx, A, smem, items);
        case 4: return launch_pruned_k<4>(ctx, A, smem, items);
        case 5: return launch_pruned_k<5>(ctx, A, smem, items);
        case 6: return launch_pruned_k<6>(ctx, A, smem, items);
        case 7: return launch_pruned_k<7>(ctx, A, smem, items);
        case 8: return launch_pruned_k<8>(ctx, A, smem, items);
        case 9: return launch_pruned_k<9>(ctx, A, smem, items);
        case 10: return launch_pruned_k<10>(ctx, A, smem, items);
        case 11: return launch_pruned_k<11>(ctx, A, smem, items);
        case 12: return launch_pruned_k<12>(ctx, A, smem, items);
        case 13: return launch_pruned_k<13>(ctx, A, smem, items);
        case 14: return launch_pruned_k<14>(ctx, A, smem, items);
        case 15: return launch_pruned_k<15>(ctx, A, smem, items);
        case 16: return launch_pruned_k<16>(ctx, A, smem, items);
        case 17: return launch_pruned_k<17>(ctx, A, smem, items);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ndf

using namespace ndf;

extern "C" ndf_status ndf_ksg_autotune(ndf_ctx* ctx, int ref_field, int query_field, int k,
                                       int* best_group, int* best_tile) {
    if (!ctx) return NDF_ERR_ARG;
    const Field *rf, *qf;
    ndf_status st = check_pair(ctx, ref_field, query_field, 0, &rf, &qf);
    if (st != NDF_OK) return st;
    if (k < 1 || k >= rf->M || k > kKsgMaxK || rf->M > kKsgMaxM)
        return fail(ctx, NDF_ERR_ARG, "bad k or M");
    cudaSetDevice(ctx->device);
    if ((st = ensure_psi_table(ctx, rf->M + 1)) != NDF_OK) return st;
    cudaError_t es = ensure_sorted_columns(ctx, ctx->fields[query_field]);
    if (es != cudaSuccess) return cuda_fail(ctx, es, "sorted columns");
    // sample: 8 references spread over the grid, the first 32768 query vertices
    const int R = 8;
    const int64_t nv = qf->N < 32768 ? qf->N : 32768;
    int64_t refs[R];
    for (int i = 0; i < R; ++i) refs[i] = (int64_t)((double)(i + 0.5) / R * (double)(rf->N - 1));
    float* out = nullptr;
    int64_t* d_refs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(float) * (size_t)R * (size_t)nv);
    if (e == cudaSuccess) e = cudaMalloc(&d_refs, sizeof refs);
    if (e == cudaSuccess) e = cudaMemcpy(d_refs, refs, sizeof refs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int cand[][2] = {{1, 4}, {1, 8}, {2, 8}, {4, 4}, {4, 8}, {8, 4}, {8, 8}};
    float best = 3.4e38f;
    int bg = ctx->ksg_group, bt = ctx->ksg_tile;
    for (const auto& c : cand) {
        if (e != cudaSuccess) break;
        // warm-up, then timed
        e = launch_ksg_pruned(ctx, *rf, *qf, d_refs, R, k, 0, nv, out, nv, c[0], c[1], nullptr,
                              nullptr, nullptr, nullptr, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
        if (e == cudaSuccess)
            e = launch_ksg_pruned(ctx, *rf, *qf, d_refs, R, k, 0, nv, out, nv, c[0], c[1], nullptr,
                                  nullptr, nullptr, nullptr, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) {
            best = ms;
            bg = c[0];
            bt = c[1];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (d_refs) cudaFree(d_refs);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ksg autotune");
    ctx->ksg_group = bg;
    ctx->ksg_tile = bt;
    if (best_group) *best_group = bg;
    if (best_tile) *best_tile = bt;
    return NDF_OK;
}

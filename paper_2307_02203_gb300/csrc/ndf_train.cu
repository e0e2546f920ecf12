// Neural dependence field: model calls, training (Sec. 4.3, Eq. 3), volume
// decoding (Sec. 5) and model files.
//
// Training set: (reference vertex, query vertex, target) triples whose targets
// come from this library's exact estimators.  They are generated in groups: a
// group draws Rg reference vertices and Qg query vertices (uniform, seeded),
// gathers the Qg query columns once into a compact member-major block, and runs
// the Pearson or KSG kernel for each reference over that block, so every group
// yields Rg x Qg uniform pairs without re-reading scattered columns.
// Training: passes over the triples in an affine-bijective order that changes
// every pass, Adam, L1 loss, learning rate x0.1 after `patience` passes without
// improvement of the pass loss (Sec. 4.3), stopping after `max_decays` decays or
// `max_passes` passes.
// Decoding: the tensor-core kernel of ndf_decode_tc.cu, which encodes every
// query vertex once per launch and forms the merged input [f_r*f_q ; f_r+f_q]
// for each reference of the launch in its layer-1 operand.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <vector>

#include "device_common.cuh"
#include "ndf_net.h"

namespace ndf {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float axis_pos(int64_t i, int64_t n) {
    return n > 1 ? -1.0f + 2.0f * (float)i / (float)(n - 1) : 0.0f;
}

__device__ __forceinline__ void vertex_pos(int64_t v, int64_t X, int64_t Y, int64_t Z, float* p) {
    const int64_t x = v % X, y = (v / X) % Y, z = v / (X * Y);
    p[0] = axis_pos(x, X);
    p[1] = axis_pos(y, Y);
    p[2] = axis_pos(z, Z);
}

static uint64_t host_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t host_rand(uint64_t key, uint64_t i) {
    return host_mix(key + (i + 1) * 0x9e3779b97f4a7c15ULL);
}

// gather the query columns of one group: out[m][q] = field[m][verts[q]]
__global__ void gather_columns_kernel(const float* __restrict__ field, int64_t M, int64_t N,
                                      const int64_t* __restrict__ verts, int64_t Q,
                                      float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M * Q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / Q, q = i % Q;
        out[i] = field[m * N + verts[q]];
    }
}

// batch positions and targets from the triple arrays through the bijection
// j = (a * (base + i) + c) mod T
__global__ void make_batch_kernel(const int32_t* __restrict__ vref, const int32_t* __restrict__ vq,
                                  const float* __restrict__ tgt, int64_t T, uint64_t a, uint64_t c,
                                  int64_t base, int64_t B, int64_t X, int64_t Y, int64_t Z,
                                  float* __restrict__ pr, float* __restrict__ pq,
                                  float* __restrict__ target) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const uint64_t j = (a * (uint64_t)(base + i) + c) % (uint64_t)T;  // a, i < T <= 2^31
    vertex_pos(vref[j], X, Y, Z, pr + 3 * i);
    vertex_pos(vq[j], X, Y, Z, pq + 3 * i);
    target[i] = tgt[j];
}

// ---------------------------------------------------------------- continuous samples (Sec. 4.3)
// Member columns at continuous positions: out[m][i] = trilinear sample of member m
// at pos[i].  FP32 with the rounding of every step fixed (no contraction), so
// that the CPU oracle reproduces the columns bit for bit:
//   u = ((p + 1) * 0.5) * (n - 1) clamped to [0, n - 1], i0 = min(floor(u), n - 2)
//   (0 for n = 1), w = u - i0, lerp(a, b, w) = a * (1 - w) + b * w along x, y, z.
__device__ __forceinline__ void interp_axis(float p, int64_t n, int64_t& i0, int64_t& i1, float& w) {
    float u = __fmul_rn(__fmul_rn(__fadd_rn(p, 1.0f), 0.5f), (float)(n - 1));
    u = fminf(fmaxf(u, 0.0f), (float)(n - 1));
    const int64_t f = (int64_t)floorf(u);
    i0 = n > 1 ? (f < n - 2 ? f : n - 2) : 0;
    w = __fsub_rn(u, (float)i0);
    i1 = i0 + 1 < n - 1 ? i0 + 1 : n - 1;
}

__device__ __forceinline__ float lerp_rn(float a, float b, float t) {
    return __fadd_rn(__fmul_rn(a, __fsub_rn(1.0f, t)), __fmul_rn(b, t));
}

__global__ void interp_columns_kernel(const float* __restrict__ field, int64_t M, int64_t X,
                                      int64_t Y, int64_t Z, const float* __restrict__ pos,
                                      int64_t n, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t x0, x1, y0, y1, z0, z1;
    float wx, wy, wz;
    interp_axis(pos[3 * i + 0], X, x0, x1, wx);
    interp_axis(pos[3 * i + 1], Y, y0, y1, wy);
    interp_axis(pos[3 * i + 2], Z, z0, z1, wz);
    const int64_t N = X * Y * Z;
    const int64_t o000 = (z0 * Y + y0) * X + x0, o100 = (z0 * Y + y0) * X + x1;
    const int64_t o010 = (z0 * Y + y1) * X + x0, o110 = (z0 * Y + y1) * X + x1;
    const int64_t o001 = (z1 * Y + y0) * X + x0, o101 = (z1 * Y + y0) * X + x1;
    const int64_t o011 = (z1 * Y + y1) * X + x0, o111 = (z1 * Y + y1) * X + x1;
    for (int64_t m = blockIdx.y; m < M; m += gridDim.y) {
        const float* f = field + m * N;
        const float c00 = lerp_rn(__ldg(f + o000), __ldg(f + o100), wx);
        const float c10 = lerp_rn(__ldg(f + o010), __ldg(f + o110), wx);
        const float c01 = lerp_rn(__ldg(f + o001), __ldg(f + o101), wx);
        const float c11 = lerp_rn(__ldg(f + o011), __ldg(f + o111), wx);
        out[m * n + i] = lerp_rn(lerp_rn(c00, c10, wy), lerp_rn(c01, c11, wy), wz);
    }
}

// Pearson r of column i of a against column i of b (Eq. 1), both blocks [M][n]
// with their FP64 means and 1/sqrt(S); FP64 accumulation, clamped to [-1, 1].
__global__ void pearson_paired_kernel(const float* __restrict__ a, const double* __restrict__ ma,
                                      const double* __restrict__ sa, const float* __restrict__ b,
                                      const double* __restrict__ mb, const double* __restrict__ sb,
                                      int64_t M, int64_t n, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double mua = ma[i], mub = mb[i];
    double acc = 0.0;
    for (int64_t m = 0; m < M; ++m)
        acc = fma((double)__ldg(a + m * n + i) - mua, (double)__ldg(b + m * n + i) - mub, acc);
    const double r = acc * sa[i] * sb[i];
    out[i] = (float)fmin(1.0, fmax(-1.0, r));
}

// batch positions and targets from continuous triples through the bijection
__global__ void make_batch_pos_kernel(const float* __restrict__ pref, const float* __restrict__ pq,
                                      const float* __restrict__ tgt, int64_t T, uint64_t a,
                                      uint64_t c, int64_t base, int64_t B, float* __restrict__ pr,
                                      float* __restrict__ pqo, float* __restrict__ target) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const uint64_t j = (a * (uint64_t)(base + i) + c) % (uint64_t)T;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        pr[3 * i + d] = pref[3 * j + d];
        pqo[3 * i + d] = pq[3 * j + d];
    }
    target[i] = tgt[j];
}

// n triples (p_ref, p_q, R(p_ref, p_q)) at uniform random positions in [-1,1]^3
// (Sec. 4.3), written to device arrays pref[n][3], pq[n][3], target[n].  Pairs
// are independent; the estimators run on the interpolated columns, pair by pair.
cudaError_t sample_triples_dev(ndf_ctx* ctx, const Field& rf, const Field& qf, int measure, int k,
                               int64_t n, uint64_t seed, float* pref, float* pq, float* target,
                               SampleScratch& sc) {
    const int64_t M = rf.M;
    const int64_t chunk = std::min<int64_t>(n, 65536);
    cudaError_t e = sc.reserve(M, chunk);
    if (e != cudaSuccess) return e;
    const uint64_t key = host_mix(seed ^ 0x434f4e54504f5353ULL);
    std::vector<float> hp((size_t)chunk * 6);
    int* d_flag = ctx->flag.as<int>();
    for (int64_t c0 = 0; c0 < n && e == cudaSuccess; c0 += chunk) {
        const int64_t nc = std::min(chunk, n - c0);
        // 24-bit uniform grid on [-1, 1): exact in FP32
        for (int64_t i = 0; i < nc * 6; ++i)
            hp[(size_t)i] = (float)((double)(host_rand(key, (uint64_t)(c0 * 6 + i)) >> 40) *
                                        (2.0 / 16777216.0) - 1.0);
        std::vector<float> hr((size_t)nc * 3), hq((size_t)nc * 3);
        for (int64_t i = 0; i < nc; ++i)
            for (int d = 0; d < 3; ++d) {
                hr[(size_t)(3 * i + d)] = hp[(size_t)(6 * i + d)];
                hq[(size_t)(3 * i + d)] = hp[(size_t)(6 * i + 3 + d)];
            }
        e = cudaMemcpyAsync(pref + 3 * c0, hr.data(), (size_t)nc * 12, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pq + 3 * c0, hq.data(), (size_t)nc * 12, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) break;
        const dim3 grid((unsigned)((nc + 127) / 128), (unsigned)std::min<int64_t>(M, 64));
        interp_columns_kernel<<<grid, 128, 0, ctx->stream>>>(rf.data, M, rf.X, rf.Y, rf.Z,
                                                             pref + 3 * c0, nc, sc.ca);
        interp_columns_kernel<<<grid, 128, 0, ctx->stream>>>(qf.data, M, qf.X, qf.Y, qf.Z,
                                                             pq + 3 * c0, nc, sc.cb);
        ctx->launches += 2;
        Field fa, fb;
        fa.live = fb.live = true;
        fa.M = fb.M = M;
        fa.Z = fb.Z = fa.Y = fb.Y = 1;
        fa.X = fb.X = fa.N = fb.N = nc;
        fa.data = sc.ca;
        fb.data = sc.cb;
        if (measure == NDF_MEASURE_PEARSON) {
            fa.mean = sc.ma;
            fa.inv_norm = sc.sa;
            fb.mean = sc.mb;
            fb.inv_norm = sc.sb;
            e = cudaMemsetAsync(d_flag, 0, 4, ctx->stream);
            if (e == cudaSuccess) e = launch_field_stats(ctx, fa, 0, nc, d_flag);
            if (e == cudaSuccess) e = launch_field_stats(ctx, fb, 0, nc, d_flag);
            if (e == cudaSuccess) {
                pearson_paired_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, ctx->stream>>>(
                    sc.ca, sc.ma, sc.sa, sc.cb, sc.mb, sc.sb, M, nc, target + c0);
                ctx->launches++;
                e = cudaGetLastError();
            }
        } else {
            fb.sorted = sc.cb_sorted;
            e = launch_sort_columns(ctx, fb, 0, nc, ctx->stream);
            if (e == cudaSuccess)
                e = launch_ksg(ctx, fa, fb, nullptr, 0, (int)nc, k, 0, nc, target + c0, 0, true, 1, 1,
                               nullptr, nullptr, nullptr, nullptr, nullptr, 1, nullptr, true);
        }
        // the host position buffers and the column blocks are reused by the next chunk
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    return e;
}

// Sum of the training targets (FP64, one atomic per block), for the MI network's
// initial output bias.
__global__ void __launch_bounds__(256) target_sum_kernel(const float* __restrict__ t, int64_t n,
                                                         double* __restrict__ sum) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s += (double)t[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += part[w];
        atomicAdd(sum, b);
    }
}

// b4 = softplus^-1(max(mean target, 1e-3)) = log(expm1(.)): the untrained MI network
// then predicts about the mean target instead of softplus(0) = 0.69
__global__ void softplus_bias_kernel(const double* __restrict__ sum, int64_t n, float* __restrict__ b4) {
    const double mean = fmax(*sum / (double)n, 1e-3);
    *b4 = (float)log(expm1(mean));
}

// ---------------------------------------------------------------- decoding (Sec. 5)
// All R references in tcgen05 launches of up to 64 references each: every query
// vertex is encoded once per launch, the references enter through the layer-1
// operand (ndf_decode_tc.cu).
cudaError_t model_infer(ndf_model* m, const int64_t* d_refs, int R, float* out) {
    return launch_infer_tc(m, d_refs, R, out);
}

}  // namespace ndf

using namespace ndf;

// ---------------------------------------------------------------- C ABI
extern "C" {

void ndf_train_cfg_default(ndf_train_cfg* c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->res[0] = 32;
    c->res[1] = 64;
    c->res[2] = 128;
    c->res[3] = 256;
    c->n_triples = int64_t(1) << 26;
    c->batch = int64_t(1) << 18;
    c->refs_per_group = 128;
    c->queries_per_group = 8192;
    c->max_passes = 50;
    c->patience = 5;
    c->max_decays = 2;
    c->lr = 3e-4f;
    c->beta1 = 0.9f;
    c->beta2 = 0.999f;
    c->eps = 1e-8f;
    c->seed = 20230705ULL;
    c->time_budget_s = 0.0;
    c->continuous = 0;
    c->hash_tf32 = 1;
}

ndf_status ndf_model_create(ndf_ctx* ctx, const int res[4], int measure, uint64_t seed, int64_t X,
                            int64_t Y, int64_t Z, ndf_model** out) {
    if (!ctx || !res || !out) return NDF_ERR_ARG;
    if (X < 1 || Y < 1 || Z < 1 || X * Y * Z > (int64_t(1) << 31))
        return fail(ctx, NDF_ERR_ARG, "grid dimensions out of range");
    cudaSetDevice(ctx->device);
    cudaError_t e = net_set_attributes();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel attributes");
    ndf_model* m = nullptr;
    ndf_status st = model_alloc(ctx, res, measure, X, Y, Z, &m);
    if (st != NDF_OK) return st;
    e = model_init_params(m, seed);
    if (e != cudaSuccess) {
        model_free(m);
        return cuda_fail(ctx, e, "parameter initialisation");
    }
    *out = m;
    return NDF_OK;
}

void ndf_model_free(ndf_model* m) {
    if (!m) return;
    cudaSetDevice(m->ctx->device);
    cudaStreamSynchronize(m->ctx->stream);
    model_free(m);
}

int64_t ndf_model_param_count(const ndf_model* m) { return m ? m->L.total : 0; }

ndf_status ndf_model_get_params(ndf_model* m, float* out) {
    if (!m || !out) return NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    cudaError_t e = cudaMemcpyAsync(out, m->params, (size_t)m->L.total * 4, cudaMemcpyDefault,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "parameter copy");
    return NDF_OK;
}

ndf_status ndf_model_set_params(ndf_model* m, const float* in) {
    if (!m || !in) return NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    cudaError_t e = cudaMemcpyAsync(m->params, in, (size_t)m->L.total * 4, cudaMemcpyDefault,
                                    ctx->stream);
    if (e == cudaSuccess) e = model_refresh_bf16(m);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "parameter upload");
    return NDF_OK;
}

// stage host-or-device positions/targets into device buffers of the work area
static ndf_status stage_batch(ndf_model* m, const float* pr, const float* pq, const float* target,
                              int64_t B, const float** dpr, const float** dpq, const float** dt) {
    ndf_ctx* ctx = m->ctx;
    ndf_status st = ensure_work(m, B);
    if (st != NDF_OK) return st;
    cudaError_t e = cudaSuccess;
    if (pointer_kind(pr) == PTR_DEVICE) {
        *dpr = pr;
    } else {
        e = cudaMemcpyAsync(m->work.pos, pr, (size_t)B * 12, cudaMemcpyHostToDevice, ctx->stream);
        *dpr = m->work.pos;
    }
    if (e == cudaSuccess) {
        if (pointer_kind(pq) == PTR_DEVICE) {
            *dpq = pq;
        } else {
            e = cudaMemcpyAsync(m->work.pos + 3 * B, pq, (size_t)B * 12, cudaMemcpyHostToDevice,
                                ctx->stream);
            *dpq = m->work.pos + 3 * B;
        }
    }
    if (e == cudaSuccess && target) {
        if (pointer_kind(target) == PTR_DEVICE) {
            *dt = target;
        } else {
            e = cudaMemcpyAsync(m->work.target, target, (size_t)B * 4, cudaMemcpyHostToDevice,
                                ctx->stream);
            *dt = m->work.target;
        }
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch upload");
    return NDF_OK;
}

ndf_status ndf_model_step(ndf_model* m, const float* p_ref, const float* p_query,
                          const float* target, int64_t B, float lr, int update, double* loss_out,
                          float* grad_out) {
    if (!m || !p_ref || !p_query || !target || B < 1) return NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    cudaSetDevice(ctx->device);
    const float *dpr, *dpq, *dt;
    ndf_status st = stage_batch(m, p_ref, p_query, target, B, &dpr, &dpq, &dt);
    if (st != NDF_OK) return st;
    cudaError_t e = cudaMemsetAsync(m->work.loss, 0, 8, ctx->stream);
    if (e == cudaSuccess)
        e = model_step(m, dpr, dpq, dt, B, lr, 0.9f, 0.999f, 1e-8f, update != 0, grad_out != nullptr);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, m->grad, (size_t)m->L.total * 4, cudaMemcpyDefault,
                            ctx->stream);
    double loss = 0.0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&loss, m->work.loss, 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "network step");
    if (loss_out) *loss_out = loss / (double)B;
    return NDF_OK;
}

ndf_status ndf_model_forward(ndf_model* m, const float* p_ref, const float* p_query, int64_t B,
                             float* out) {
    if (!m || !p_ref || !p_query || !out || B < 1) return NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    cudaSetDevice(ctx->device);
    const float *dpr, *dpq, *dt = nullptr;
    ndf_status st = stage_batch(m, p_ref, p_query, nullptr, B, &dpr, &dpq, &dt);
    if (st != NDF_OK) return st;
    void* dev_out;
    bool is_host;
    if ((st = resolve_out(ctx, out, (size_t)B * 4, &dev_out, &is_host)) != NDF_OK) return st;
    cudaError_t e = model_forward(m, dpr, dpq, B, static_cast<float*>(dev_out));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "network forward");
    return finish_out(ctx, out, dev_out, (size_t)B * 4, is_host);
}

ndf_status ndf_infer_batch(ndf_model* m, const int64_t* ref_idx, int R, float* out) {
    if (!m || !ref_idx || R < 1 || !out) return m ? fail(m->ctx, NDF_ERR_ARG, "bad arguments") : NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    const int64_t N = m->X * m->Y * m->Z;
    for (int i = 0; i < R; ++i)
        if (ref_idx[i] < 0 || ref_idx[i] >= N) return fail(ctx, NDF_ERR_ARG, "ref_idx out of range");
    cudaSetDevice(ctx->device);
    const size_t bytes = (size_t)R * (size_t)N * 4;
    void* dev_out;
    bool is_host;
    ndf_status st = resolve_out(ctx, out, bytes, &dev_out, &is_host);
    if (st != NDF_OK) return st;
    cudaError_t e = ctx->refidx.reserve(sizeof(int64_t) * (size_t)R);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->refidx.ptr, ref_idx, sizeof(int64_t) * (size_t)R,
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = model_infer(m, ctx->refidx.as<int64_t>(), R, static_cast<float*>(dev_out));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "network decoding");
    return finish_out(ctx, out, dev_out, bytes, is_host);
}

ndf_status ndf_infer(ndf_model* m, int64_t ref_idx, float* out) {
    return ndf_infer_batch(m, &ref_idx, 1, out);
}

ndf_status ndf_model_info(const ndf_model* m, ndf_model_info_t* info) {
    if (!m || !info) return NDF_ERR_ARG;
    memset(info, 0, sizeof *info);
    info->measure = m->measure;
    for (int l = 0; l < kLevels; ++l) info->res[l] = m->L.res[l];
    info->X = m->X;
    info->Y = m->Y;
    info->Z = m->Z;
    info->param_count = m->L.total;
    info->grid_params = m->L.n_grid;
    // inference footprint: BF16 grid + BF16 weights + FP32 biases/output layer
    info->network_bytes = m->L.n_grid * 2 + (int64_t)3 * kHid * kHid * 2 * 2 + (m->L.total - m->L.W1) * 4;
    info->training_bytes = m->L.total * 4 * 4 + m->L.n_grid * 2;
    info->adam_steps = m->t;
    info->passes = m->passes;
    info->last_loss = m->last_loss;
    info->n_triples = m->n_triples;
    info->gen_seconds = m->gen_seconds;
    info->train_seconds = m->train_seconds;
    return NDF_OK;
}

ndf_status ndf_sample_triples(ndf_ctx* ctx, int ref_field, int query_field, int measure, int k,
                              int64_t n, uint64_t seed, float* pref, float* pq, float* target) {
    if (!ctx) return NDF_ERR_ARG;
    if (!pref || !pq || !target) return fail(ctx, NDF_ERR_ARG, "null pointer");
    const Field *rf, *qf;
    ndf_status st = check_pair(ctx, ref_field, query_field, 0, &rf, &qf);
    if (st != NDF_OK) return st;
    if (measure != NDF_MEASURE_PEARSON && measure != NDF_MEASURE_MI_KSG)
        return fail(ctx, NDF_ERR_ARG, "unknown measure %d", measure);
    if (measure == NDF_MEASURE_MI_KSG && (k < 1 || k >= rf->M || k > kKsgMaxK || rf->M > kKsgMaxM))
        return fail(ctx, NDF_ERR_ARG, "bad k or M for the KSG targets");
    if (n < 1 || n > (int64_t(1) << 31)) return fail(ctx, NDF_ERR_ARG, "need 1 <= n <= 2^31");
    cudaSetDevice(ctx->device);
    if (measure == NDF_MEASURE_MI_KSG && (st = ensure_psi_table(ctx, rf->M + 1)) != NDF_OK) return st;
    void *dr, *dq, *dt;
    bool hr, hq, ht;
    // device staging for host outputs: three context buffers would alias, so use one
    const size_t bp = sizeof(float) * 3 * (size_t)n, bt = sizeof(float) * (size_t)n;
    const bool any_host = pointer_kind(pref) != PTR_DEVICE || pointer_kind(pq) != PTR_DEVICE ||
                          pointer_kind(target) != PTR_DEVICE;
    float* stage = nullptr;
    if (any_host) {
        cudaError_t e = cudaMalloc(&stage, 2 * bp + bt);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sampler staging");
    }
    hr = pointer_kind(pref) != PTR_DEVICE;
    hq = pointer_kind(pq) != PTR_DEVICE;
    ht = pointer_kind(target) != PTR_DEVICE;
    dr = hr ? (void*)stage : (void*)pref;
    dq = hq ? (void*)(stage + 3 * n) : (void*)pq;
    dt = ht ? (void*)(stage + 6 * n) : (void*)target;
    SampleScratch sc;
    cudaError_t e = sample_triples_dev(ctx, *rf, *qf, measure, k, n, seed, (float*)dr, (float*)dq,
                                       (float*)dt, sc);
    if (e == cudaSuccess && hr) e = cudaMemcpyAsync(pref, dr, bp, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && hq) e = cudaMemcpyAsync(pq, dq, bp, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && ht) e = cudaMemcpyAsync(target, dt, bt, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    sc.release();
    if (stage) cudaFree(stage);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "continuous sampling");
    return check_device_status(ctx);
}

// ---- training (Sec. 4.3)
ndf_status ndf_train(ndf_ctx* ctx, int ref_field, int query_field, int measure, int k,
                     const ndf_train_cfg* cfg_in, ndf_model** out) {
    if (!ctx || !out) return NDF_ERR_ARG;
    ndf_train_cfg cfg;
    if (cfg_in) cfg = *cfg_in;
    else ndf_train_cfg_default(&cfg);
    const Field *rf, *qf;
    ndf_status st = check_pair(ctx, ref_field, query_field, 0, &rf, &qf);
    if (st != NDF_OK) return st;
    if (measure != NDF_MEASURE_PEARSON && measure != NDF_MEASURE_MI_KSG)
        return fail(ctx, NDF_ERR_ARG, "unknown measure %d", measure);
    if (measure == NDF_MEASURE_MI_KSG &&
        (k < 1 || k >= rf->M || k > kKsgMaxK || rf->M > kKsgMaxM))
        return fail(ctx, NDF_ERR_ARG, "bad k or M for the KSG targets");
    if (cfg.n_triples < 1 || cfg.batch < 1 || cfg.refs_per_group < 1 || cfg.queries_per_group < 1 ||
        cfg.max_passes < 1 || cfg.n_triples > (int64_t(1) << 31))
        return fail(ctx, NDF_ERR_ARG, "bad training configuration");
    cudaSetDevice(ctx->device);
    const int64_t N = qf->N, M = qf->M;
    const int64_t Qg = cfg.queries_per_group < N ? cfg.queries_per_group : N;
    const int64_t Rg = cfg.refs_per_group;
    const int64_t T = cfg.n_triples;
    ndf_model* m = nullptr;
    if ((st = ndf_model_create(ctx, cfg.res, measure, cfg.seed, qf->X, qf->Y, qf->Z, &m)) != NDF_OK)
        return st;
    auto bail = [&](ndf_status s) {
        ndf_model_free(m);
        return s;
    };
    if (measure == NDF_MEASURE_MI_KSG) {
        if ((st = ensure_psi_table(ctx, M + 1)) != NDF_OK) return bail(st);
        cudaError_t es = ensure_sorted_columns(ctx, ctx->fields[query_field]);
        if (es != cudaSuccess) return bail(cuda_fail(ctx, es, "sorted columns"));
    }

    // ---- training triples: grid vertex pairs, or (continuous) uniform random
    // positions with trilinear samples, renewed every pass (Sec. 4.3)
    const bool cont = cfg.continuous != 0;
    auto t0 = std::chrono::steady_clock::now();
    int32_t *vref = nullptr, *vq = nullptr;
    float *cpref = nullptr, *cpq = nullptr;
    SampleScratch sc;
    float *tgt = nullptr, *block = nullptr, *block_sorted = nullptr, *gtgt = nullptr;
    int64_t *dq = nullptr, *drefs = nullptr;
    cudaError_t e = cudaMalloc(&tgt, (size_t)T * 4);
    if (cont) {
        if (e == cudaSuccess) e = cudaMalloc(&cpref, (size_t)T * 12);
        if (e == cudaSuccess) e = cudaMalloc(&cpq, (size_t)T * 12);
    } else {
        if (e == cudaSuccess) e = cudaMalloc(&vref, (size_t)T * 4);
        if (e == cudaSuccess) e = cudaMalloc(&vq, (size_t)T * 4);
    }
    if (e == cudaSuccess) e = cudaMalloc(&block, (size_t)M * Qg * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dq, (size_t)Qg * 8);
    if (e == cudaSuccess) e = cudaMalloc(&gtgt, (size_t)Rg * Qg * 4);
    if (e == cudaSuccess && measure == NDF_MEASURE_MI_KSG)
        e = cudaMalloc(&block_sorted, (size_t)M * Qg * 4);
    if (e == cudaSuccess) e = cudaMalloc(&drefs, (size_t)Rg * 8);
    Field blk;
    blk.live = true;
    blk.M = M;
    blk.Z = 1;
    blk.Y = 1;
    blk.X = Qg;
    blk.N = Qg;
    blk.data = block;
    blk.sorted = block_sorted;  // gathered from the query field's sorted columns
    if (e == cudaSuccess && measure == NDF_MEASURE_PEARSON) {
        e = cudaMalloc(&blk.mean, (size_t)Qg * 8);
        if (e == cudaSuccess) e = cudaMalloc(&blk.inv_norm, (size_t)Qg * 8);
    }
    auto cleanup_data = [&]() {
        void* ps[] = {vref, vq, tgt, block, block_sorted, dq, gtgt, drefs, blk.mean, blk.inv_norm,
                      cpref, cpq};
        for (void* q : ps)
            if (q) cudaFree(q);
        sc.release();
    };
    if (e != cudaSuccess) {
        cleanup_data();
        return bail(cuda_fail(ctx, e, "training-set buffers"));
    }
    std::vector<int64_t> hq((size_t)Qg), hrefs((size_t)Rg);
    std::vector<int32_t> hr((size_t)(cont ? 0 : T)), hqv((size_t)(cont ? 0 : T));
    const uint64_t key = host_mix(cfg.seed ^ 0x4e44465452414e53ULL);
    int64_t filled = 0, group = 0;
    int* d_flag = ctx->flag.as<int>();
    while (!cont && filled < T && e == cudaSuccess) {
        // queries of this group: Qg distinct-ish uniform vertices, sorted for locality
        for (int64_t q = 0; q < Qg; ++q)
            hq[(size_t)q] = (int64_t)(host_rand(key, (uint64_t)(group * 2 * Qg + q)) % (uint64_t)N);
        std::sort(hq.begin(), hq.end());
        e = cudaMemcpyAsync(dq, hq.data(), (size_t)Qg * 8, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) break;
        gather_columns_kernel<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(qf->data, M, N, dq, Qg, block);
        ctx->launches++;
        if (block_sorted) {
            gather_columns_kernel<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(
                ctx->fields[query_field].sorted, M, N, dq, Qg, block_sorted);
            ctx->launches++;
        }
        if (measure == NDF_MEASURE_PEARSON) {
            e = cudaMemsetAsync(d_flag, 0, 4, ctx->stream);
            if (e == cudaSuccess) e = launch_field_stats(ctx, blk, 0, blk.N, d_flag);
        }
        // reference vertices of this group (as many as the remaining triples need)
        const int64_t rows = std::min<int64_t>(Rg, (T - filled + Qg - 1) / Qg);
        for (int64_t r = 0; r < rows; ++r)
            hrefs[(size_t)r] = (int64_t)(host_rand(key ^ 0xa5a5a5a5ULL, (uint64_t)(group * Rg + r)) %
                                         (uint64_t)rf->N);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(drefs, hrefs.data(), (size_t)rows * 8, cudaMemcpyHostToDevice,
                                ctx->stream);
        if (measure == NDF_MEASURE_PEARSON) {
            for (int64_t r = 0; r < rows && e == cudaSuccess; ++r)
                e = launch_pearson(ctx, *rf, blk, hrefs[(size_t)r], gtgt + r * Qg);
        } else if (e == cudaSuccess) {
            // all references of the group in one launch; each query column is sorted once
            e = launch_ksg(ctx, *rf, blk, drefs, 0, (int)rows, k, 0, Qg, gtgt, Qg,
                           ctx->ksg_algorithm != NDF_KSG_BRUTE, ctx->ksg_group, ctx->ksg_tile,
                           nullptr, nullptr, nullptr, nullptr, nullptr);
        }
        const int64_t take = std::min<int64_t>(T - filled, rows * Qg);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tgt + filled, gtgt, (size_t)take * 4, cudaMemcpyDeviceToDevice,
                                ctx->stream);
        for (int64_t i = 0; i < take; ++i) {
            hr[(size_t)(filled + i)] = (int32_t)hrefs[(size_t)(i / Qg)];
            hqv[(size_t)(filled + i)] = (int32_t)hq[(size_t)(i % Qg)];
        }
        filled += take;
        // the next group's gather overwrites the block: wait for this group's kernels
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        ++group;
    }
    if (e == cudaSuccess && !cont)
        e = cudaMemcpyAsync(vref, hr.data(), (size_t)T * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && !cont)
        e = cudaMemcpyAsync(vq, hqv.data(), (size_t)T * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && cont)
        e = sample_triples_dev(ctx, *rf, *qf, measure, k, T, cfg.seed, cpref, cpq, tgt, sc);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cleanup_data();
        return bail(cuda_fail(ctx, e, "training-set generation"));
    }
    if (e == cudaSuccess && measure == NDF_MEASURE_MI_KSG) {
        // the output bias from the first targets (on continuous samples: the first pass's)
        double* dsum = reinterpret_cast<double*>(ctx->flag.as<unsigned char>() + 64);
        e = cudaMemsetAsync(dsum, 0, sizeof(double), ctx->stream);
        if (e == cudaSuccess) {
            target_sum_kernel<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(tgt, T, dsum);
            softplus_bias_kernel<<<1, 1, 0, ctx->stream>>>(dsum, T, m->params + m->L.b4);
            ctx->launches += 2;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            cleanup_data();
            return bail(cuda_fail(ctx, e, "output bias"));
        }
    }
    auto t1 = std::chrono::steady_clock::now();
    m->gen_seconds = std::chrono::duration<double>(t1 - t0).count();
    m->n_triples = T;

    // ---- passes with Adam and the plateau schedule
    const int64_t B = cfg.batch < T ? cfg.batch : T;
    if ((st = ensure_work(m, B)) != NDF_OK) {
        cleanup_data();
        return bail(st);
    }
    float lr = cfg.lr;
    double best = 1e300;
    int bad = 0, decays = 0;
    double extra_gen = 0.0;
    for (int pass = 0; pass < cfg.max_passes && e == cudaSuccess; ++pass) {
        if (cont && pass > 0) {  // fresh samples every pass
            const auto g0 = std::chrono::steady_clock::now();
            e = sample_triples_dev(ctx, *rf, *qf, measure, k, T, cfg.seed + (uint64_t)pass, cpref,
                                   cpq, tgt, sc);
            extra_gen += std::chrono::duration<double>(std::chrono::steady_clock::now() - g0).count();
            if (e != cudaSuccess) break;
        }
        // a new affine bijection j = a*i + c (mod T) every pass
        uint64_t a = host_rand(key ^ 0x5bd1e995ULL, (uint64_t)pass) % (uint64_t)T;
        if (a == 0) a = 1;
        while (std::gcd(a, (uint64_t)T) != 1) a = (a + 1) % (uint64_t)T == 0 ? 1 : a + 1;
        const uint64_t c = host_rand(key ^ 0x27d4eb2fULL, (uint64_t)pass) % (uint64_t)T;
        e = cudaMemsetAsync(m->work.loss, 0, 8, ctx->stream);
        for (int64_t base = 0; base < T && e == cudaSuccess; base += B) {
            const int64_t b = T - base < B ? T - base : B;
            if (cont)
                make_batch_pos_kernel<<<(unsigned)((b + 255) / 256), 256, 0, ctx->stream>>>(
                    cpref, cpq, tgt, T, a, c, base, b, m->work.pos, m->work.pos + 3 * B,
                    m->work.target);
            else
                make_batch_kernel<<<(unsigned)((b + 255) / 256), 256, 0, ctx->stream>>>(
                    vref, vq, tgt, T, a, c, base, b, m->X, m->Y, m->Z, m->work.pos,
                    m->work.pos + 3 * B, m->work.target);
            ctx->launches++;
            e = model_step(m, m->work.pos, m->work.pos + 3 * B, m->work.target, b, lr, cfg.beta1,
                           cfg.beta2, cfg.eps, true);
            m->steps++;
        }
        double sum = 0.0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&sum, m->work.loss, 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) break;
        const double pass_loss = sum / (double)T;
        m->last_loss = pass_loss;
        m->passes = pass + 1;
        if (pass_loss < best * (1.0 - 1e-4)) {
            best = pass_loss;
            bad = 0;
        } else if (++bad > cfg.patience) {
            lr *= 0.1f;
            bad = 0;
            if (++decays > cfg.max_decays) break;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
        if (cfg.time_budget_s > 0.0 && el > cfg.time_budget_s) break;
    }
    m->train_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count() - extra_gen;
    m->gen_seconds += extra_gen;
    cleanup_data();
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "training"));
    *out = m;
    return NDF_OK;
}

// ---- model files: "NDFMODEL" v1, header, then FP32 params, Adam m and v
struct FileHeader {
    char magic[8];
    int32_t version, measure;
    int32_t res[4];
    int64_t X, Y, Z, total, t;
};

ndf_status ndf_model_save(ndf_model* m, const char* path) {
    if (!m || !path) return NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    const size_t n = (size_t)m->L.total;
    std::vector<float> buf(3 * n);
    cudaError_t e = cudaMemcpyAsync(buf.data(), m->params, n * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf.data() + n, m->m, n * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf.data() + 2 * n, m->v, n * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "model download");
    FileHeader h;
    memcpy(h.magic, "NDFMODEL", 8);
    h.version = 1;
    h.measure = m->measure;
    for (int l = 0; l < 4; ++l) h.res[l] = m->L.res[l];
    h.X = m->X;
    h.Y = m->Y;
    h.Z = m->Z;
    h.total = m->L.total;
    h.t = m->t;
    FILE* f = fopen(path, "wb");
    if (!f) return fail(ctx, NDF_ERR_IO, "cannot open %s", path);
    bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(buf.data(), 4, 3 * n, f) == 3 * n;
    ok = (fclose(f) == 0) && ok;
    return ok ? NDF_OK : fail(ctx, NDF_ERR_IO, "write to %s failed", path);
}

ndf_status ndf_model_load(ndf_ctx* ctx, const char* path, ndf_model** out) {
    if (!ctx || !path || !out) return NDF_ERR_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(ctx, NDF_ERR_IO, "cannot open %s", path);
    FileHeader h;
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, "NDFMODEL", 8) != 0 || h.version != 1) {
        fclose(f);
        return fail(ctx, NDF_ERR_IO, "%s is not an NDF model file", path);
    }
    ndf_model* m = nullptr;
    ndf_status st = ndf_model_create(ctx, h.res, h.measure, 0, h.X, h.Y, h.Z, &m);
    if (st != NDF_OK) {
        fclose(f);
        return st;
    }
    if (m->L.total != h.total) {
        fclose(f);
        ndf_model_free(m);
        return fail(ctx, NDF_ERR_IO, "%s: parameter count mismatch", path);
    }
    const size_t n = (size_t)h.total;
    std::vector<float> buf(3 * n);
    const bool ok = fread(buf.data(), 4, 3 * n, f) == 3 * n;
    fclose(f);
    if (!ok) {
        ndf_model_free(m);
        return fail(ctx, NDF_ERR_IO, "%s is truncated", path);
    }
    cudaError_t e = cudaMemcpyAsync(m->params, buf.data(), n * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->m, buf.data() + n, n * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->v, buf.data() + 2 * n, n * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = model_refresh_bf16(m);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        ndf_model_free(m);
        return cuda_fail(ctx, e, "model upload");
    }
    m->t = h.t;
    *out = m;
    return NDF_OK;
}

}  // extern "C"

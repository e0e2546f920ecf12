// The paper's neural dependence field architecture (Sec. 4.1-4.2, Fig. 2) on the
// GPU: input embedding = [p, Fourier features (Eq. 4), multi-resolution hash-grid
// features], MLP encoder(s) with Snake-family activations, element-wise product
// merge, MLP decoder, tanh / softplus output; L1 loss (Eq. 3) and Adam.
//
// Layout and definitions are those of the FP64 oracle (hash_net_oracle.h):
//   level l: R_l = base_res * 2^l points per axis, corner-aligned on [-1,1]^3,
//            E_l = min(2^T, R_l^3) entries of F features; dense index
//            x + R y + R^2 z when R^3 <= 2^T, else (x * 1 ^ y * 2654435761 ^
//            z * 805459861) mod 2^T (uint32)
//   params:  per encoder: level tables, then layers (W[out][in], b[out]); then
//            the decoder layers.  One encoder (self field, symmetric by
//            construction) or two (cross field: 0 reference, 1 query).
//
// GPU design: activations are feature-major per sample ([B][c] row-major), the
// dense layers are this library's FP32 matrix products (gemm_f32.cu: FP32 for
// parity with the oracle, deterministic weight-gradient sums), and everything
// between them (embedding, bias + activation, merge, output + loss, the
// hash-table scatter of the backward, Adam) is in the kernels below.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <numeric>
#include <vector>

#include "gemm_f32.h"
#include "hash_common.cuh"
#include "ndf_hash_tc.h"
#include "ndf_internal.h"

namespace ndf {

// initial scale of the first encoder layer's weights on the Fourier columns,
// relative to the He-uniform scale of the other weights (see ndf_hash_model_create)
constexpr double kFourierInit = 0.1;

// x0[b][din] = embed(pos[b]) with the tables of one encoder
__global__ void hash_embed_kernel(const float* __restrict__ pos, int64_t B,
                                  const float* __restrict__ enc, EmbedArgs E,
                                  float* __restrict__ x0) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float p[3] = {pos[3 * b], pos[3 * b + 1], pos[3 * b + 2]};
    float* x = x0 + b * E.din;
    embed_point(E, enc, p, [&](int k, float v) { x[k] = v; });
}

// hash-table gradient: scatter dL/d(embedding) of the hash features
__global__ void hash_embed_backward_kernel(const float* __restrict__ pos, int64_t B,
                                           const float* __restrict__ gx, EmbedArgs E,
                                           float* __restrict__ genc) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float p[3] = {pos[3 * b], pos[3 * b + 1], pos[3 * b + 2]};
    const float* g = gx + b * E.din + 3 + 6 * E.L;
    for (int l = 0; l < E.levels; ++l) {
        const Cell cl = level_cell(E, l, p);
        float* tab = genc + E.toff[l];
        for (int f = 0; f < E.F; ++f) {
            const float gv = g[l * E.F + f];
            if (gv == 0.0f) continue;
#pragma unroll
            for (int q = 0; q < 8; ++q) atomicAdd(tab + (int64_t)cl.idx[q] * E.F + f, cl.w[q] * gv);
        }
    }
}

// pre[b][o] += bias[o]; post = act(pre) (or a copy when act < 0)
__global__ void bias_act_kernel(float* __restrict__ pre, const float* __restrict__ bias, int c,
                                int64_t B, int act, float* __restrict__ post) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)c * B) return;
    const float v = pre[i] + bias[i % c];
    pre[i] = v;
    if (post) post[i] = act < 0 ? v : act_f(act, v);
}

__global__ void dact_mul_kernel(float* __restrict__ g, const float* __restrict__ pre, int64_t n,
                                int act) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) g[i] *= dact_f(act, pre[i]);
}

// z from the two latents (d features each, zr broadcast when zr_stride == 0):
// product (the paper's merge), sum, |difference|, or concatenation [zr; zq]
__global__ void merge_kernel(const float* __restrict__ zr, int64_t zr_stride,
                             const float* __restrict__ zq, int d, int64_t B, int mode,
                             float* __restrict__ z) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)d * B) return;
    const int64_t b = i / d, o = i - b * d;
    const float a = zr[b * zr_stride + o], q = zq[i];
    if (mode == NDF_MERGE_CONCAT) {
        z[b * 2 * d + o] = a;
        z[b * 2 * d + d + o] = q;
    } else {
        z[i] = mode == NDF_MERGE_PRODUCT ? a * q : mode == NDF_MERGE_SUM ? a + q : fabsf(a - q);
    }
}

__global__ void merge_backward_kernel(const float* __restrict__ g, const float* __restrict__ zr,
                                      const float* __restrict__ zq, int d, int64_t B, int mode,
                                      float* __restrict__ gr, float* __restrict__ gq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)d * B) return;
    const int64_t b = i / d, o = i - b * d;
    if (mode == NDF_MERGE_CONCAT) {
        gr[i] = g[b * 2 * d + o];
        gq[i] = g[b * 2 * d + d + o];
    } else if (mode == NDF_MERGE_PRODUCT) {
        gr[i] = g[i] * zq[i];
        gq[i] = g[i] * zr[i];
    } else if (mode == NDF_MERGE_SUM) {
        gr[i] = g[i];
        gq[i] = g[i];
    } else {
        const float sg = zr[i] > zq[i] ? 1.0f : (zr[i] < zq[i] ? -1.0f : 0.0f);
        gr[i] = g[i] * sg;
        gq[i] = -g[i] * sg;
    }
}

// y = out_act(raw) (and the L1 loss and its gradient when target != null)
__global__ void out_loss_kernel(const float* __restrict__ raw, const float* __restrict__ target,
                                int64_t B, int measure, float* __restrict__ y,
                                float* __restrict__ graw, double* __restrict__ loss) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < B) {
        const float x = raw[b];
        const float v = out_act(measure, x);
        if (y) y[b] = v;
        if (target) {
            const float d = v - target[b];
            l = fabs((double)d);
            const float sg = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
            float dv;
            if (measure == NDF_MEASURE_PEARSON) {
                dv = 1.0f - v * v;
            } else {
                dv = 1.0f / (1.0f + expf(-x));
            }
            graw[b] = sg / (float)B * dv;
        }
    }
    if (target) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
    }
}

__global__ void hash_adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                 float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                                 float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void fill_kernel(float* __restrict__ p, int64_t n, float v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void vertex_positions_kernel(int64_t v0, int64_t n, int64_t X, int64_t Y, int64_t Z,
                                        float* __restrict__ pos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vertex_position(v0 + i, X, Y, Z, pos + 3 * i);
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace ndf

namespace ndf {

// the tensor-core decoder covers width 128, an embedding of at most 128 inputs
// and the element-wise merges (not concatenation)
static bool hash_tc_eligible(const HashLayout& L) {
    const int nL = L.le + L.ld - 1;
    const int kin = 3 * hash_tc_f8(L.L) + 3 + L.levels * L.F;  // embedding columns in operand order
    return L.c == 128 && kin <= 128 && L.merge != NDF_MERGE_CONCAT && nL >= 1 && nL <= kHashTcMaxLayers;
}

// the query-latent cache needs a latent (an encoder layer) and a decoder layer after it
static bool hash_tc_cache_ok(const HashLayout& L) { return hash_tc_eligible(L) && L.le >= 1 && L.ld >= 2; }

}  // namespace ndf

using namespace ndf;

struct ndf_hash_model {
    ndf_ctx* ctx = nullptr;
    ndf_hash_arch arch{};
    int measure = 0;
    int64_t X = 1, Y = 1, Z = 1;
    HashLayout Ly;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int64_t t = 0;
    // workspace for a batch of up to cap samples, and of the weight-gradient products
    float* gemm_work = nullptr;
    int64_t cap = 0;
    float* ws = nullptr;
    float *x0[2] = {}, *pre_e[2][kHashMaxLayers] = {}, *post_e[2][kHashMaxLayers] = {};
    float *z = nullptr, *pre_d[kHashMaxLayers] = {}, *post_d[kHashMaxLayers] = {};
    float *ga = nullptr, *gb = nullptr, *gr = nullptr, *gq = nullptr;
    float *graw = nullptr, *tgt = nullptr, *pos = nullptr;
    double* loss = nullptr;
    // tensor-core decoding: packed BF16 weight images and biases of the parameter
    // version tc_ver, reference latents, per-axis Fourier features of the decode
    // grid, optional cache of the query latents
    int decode_tc = 0, cache_q = 0;
    int64_t ver = 0, tc_ver = -1, lat_ver = -1;
    unsigned char* tc_w = nullptr;
    float *tc_bias = nullptr, *tc_zr = nullptr, *tc_lat = nullptr, *tc_ftab = nullptr;
    // training record
    int passes = 0;
    double last_loss = 0.0, gen_seconds = 0.0, train_seconds = 0.0;
    int64_t n_triples = 0;
};

namespace ndf {

static cudaError_t hash_workspace(ndf_hash_model* m, int64_t B) {
    if (B <= m->cap) return cudaSuccess;
    if (m->ws) cudaFree(m->ws);
    if (m->gemm_work) cudaFree(m->gemm_work);
    m->ws = nullptr;
    m->gemm_work = nullptr;
    m->cap = 0;
    const HashLayout& L = m->Ly;
    const int64_t c = L.c, wmax = std::max<int64_t>(std::max<int64_t>(L.din, c), L.ddec);
    // loss (2 doubles), x0 x2, encoder pre/post x2 sides, z, decoder pre/post,
    // ga, gb (ping-pong), gr, gq (merge gradients), graw, tgt, positions
    const int64_t floats = 4 + 2 * B * L.din + 2 * 2 * L.le * B * c + B * L.ddec +
                           2 * L.ld * B * c + 2 * B * wmax + 2 * B * L.dlat + 2 * B + 6 * B;
    cudaError_t e = cudaMalloc(&m->ws, sizeof(float) * (size_t)floats);
    if (e != cudaSuccess) return e;
    // partial products of the weight gradients (at most c x wmax per slice) and of the
    // bias gradients
    const int64_t wf = std::max<int64_t>(gemm_f32_tn_work_floats(c, wmax, B), kSplitK * wmax);
    e = cudaMalloc(&m->gemm_work, sizeof(float) * (size_t)wf);
    if (e != cudaSuccess) return e;
    float* o = m->ws;
    auto take = [&](int64_t n) {
        float* r = o;
        o += n;
        return r;
    };
    m->loss = reinterpret_cast<double*>(take(4));
    for (int s = 0; s < 2; ++s) m->x0[s] = take(B * L.din);
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < L.le; ++k) {
            m->pre_e[s][k] = take(B * c);
            m->post_e[s][k] = take(B * c);
        }
    m->z = take(B * L.ddec);
    for (int k = 0; k < L.ld; ++k) {
        m->pre_d[k] = take(B * c);
        m->post_d[k] = take(B * c);
    }
    m->ga = take(B * wmax);
    m->gb = take(B * wmax);
    m->gr = take(B * L.dlat);
    m->gq = take(B * L.dlat);
    m->graw = take(B);
    m->tgt = take(B);
    m->pos = take(6 * B);
    m->cap = B;
    return cudaSuccess;
}

// Activations are sample-major, [B][c]; W is [c_out][c_in].
// Y[B][c_out] = X[B][c_in] W^T
static bool gemm_fwd(ndf_hash_model* m, const float* W, const float* X, float* Y, int c_out,
                     int c_in, int64_t B) {
    return gemm_f32_nt(m->ctx->stream, X, W, Y, B, c_out, c_in) == cudaSuccess;
}

// dX = dY W (when dX is wanted); dW += dY^T X; db += the column sums of dY
static bool gemm_bwd(ndf_hash_model* m, const float* W, const float* X, const float* dY, float* dX,
                     float* dW, float* db, int c_out, int c_in, int64_t B) {
    cudaStream_t s = m->ctx->stream;
    if (dX && gemm_f32_nn(s, dY, W, dX, B, c_in, c_out) != cudaSuccess) return false;
    if (gemm_f32_tn_acc(s, dY, X, dW, c_out, c_in, B, m->gemm_work) != cudaSuccess) return false;
    m->ctx->launches += 5;
    return colsum_f32_acc(s, dY, db, B, c_out, m->gemm_work) == cudaSuccess;
}

// encoder e over the positions pos[B][3]: fills x0 / pre / post of side s
static cudaError_t encode_side(ndf_hash_model* m, int e, int s, const float* pos, int64_t B) {
    const HashLayout& L = m->Ly;
    ndf_ctx* ctx = m->ctx;
    const float* enc = m->params + L.enc_size * e;
    hash_embed_kernel<<<blocks_for(B, 128), 128, 0, ctx->stream>>>(pos, B, enc, embed_args(L),
                                                                   m->x0[s]);
    ctx->launches++;
    const float* in = m->x0[s];
    for (int k = 0; k < L.le; ++k) {
        const int cin = k == 0 ? L.din : L.c;
        if (!gemm_fwd(m, enc + L.ew[k], in, m->pre_e[s][k], L.c, cin, B))
            return cudaErrorUnknown;
        bias_act_kernel<<<blocks_for((int64_t)L.c * B), 256, 0, ctx->stream>>>(
            m->pre_e[s][k], enc + L.eb[k], L.c, B, k < L.le - 1 ? L.act : -1, m->post_e[s][k]);
        ctx->launches++;
        in = m->post_e[s][k];
    }
    return cudaGetLastError();
}

// the latent of side s: the last encoder layer, or the embedding (grid-only)
static const float* latent(const ndf_hash_model* m, int s) {
    return m->Ly.le > 0 ? m->post_e[s][m->Ly.le - 1] : m->x0[s];
}

// decoder over m->z; raw outputs in pre_d[ld-1]
static cudaError_t decode_z(ndf_hash_model* m, int64_t B) {
    const HashLayout& L = m->Ly;
    ndf_ctx* ctx = m->ctx;
    const float* in = m->z;
    for (int k = 0; k < L.ld; ++k) {
        const int cout = k == L.ld - 1 ? 1 : L.c, cin = k == 0 ? L.ddec : L.c;
        if (!gemm_fwd(m, m->params + L.dw[k], in, m->pre_d[k], cout, cin, B))
            return cudaErrorUnknown;
        bias_act_kernel<<<blocks_for((int64_t)cout * B), 256, 0, ctx->stream>>>(
            m->pre_d[k], m->params + L.db[k], cout, B, k < L.ld - 1 ? L.act : -1, m->post_d[k]);
        ctx->launches++;
        in = m->post_d[k];
    }
    return cudaGetLastError();
}

// full forward (and, with target, the L1 loss, gradient into m->grad)
static cudaError_t hash_forward_backward(ndf_hash_model* m, const float* pr, const float* pq,
                                         const float* target, int64_t B, float* y) {
    const HashLayout& L = m->Ly;
    ndf_ctx* ctx = m->ctx;
    const int eq = L.n_enc - 1;
    cudaError_t e = encode_side(m, 0, 0, pr, B);
    if (e == cudaSuccess) e = encode_side(m, eq, 1, pq, B);
    if (e != cudaSuccess) return e;
    const float* zr = latent(m, 0);
    const float* zq = latent(m, 1);
    merge_kernel<<<blocks_for((int64_t)L.dlat * B), 256, 0, ctx->stream>>>(zr, L.dlat, zq, L.dlat, B,
                                                                           L.merge, m->z);
    ctx->launches++;
    if ((e = decode_z(m, B)) != cudaSuccess) return e;
    out_loss_kernel<<<blocks_for(B), 256, 0, ctx->stream>>>(m->pre_d[L.ld - 1], target, B,
                                                             m->measure, y, m->graw, m->loss);
    ctx->launches++;
    if (!target) return cudaGetLastError();
    // ---- backward: decoder (ping-pong ga / gb), merge, then each encoder side
    const float* g = m->graw;  // dL/d(raw output), [1][B]
    float* pp[2] = {m->ga, m->gb};
    int cur = 0;
    for (int k = L.ld - 1; k >= 0; --k) {
        const int cout = k == L.ld - 1 ? 1 : L.c, cin = k == 0 ? L.ddec : L.c;
        const float* in = k == 0 ? m->z : m->post_d[k - 1];
        float* gin = pp[cur];
        if (!gemm_bwd(m, m->params + L.dw[k], in, g, gin, m->grad + L.dw[k], m->grad + L.db[k],
                      cout, cin, B))
            return cudaErrorUnknown;
        if (k > 0) {
            dact_mul_kernel<<<blocks_for((int64_t)L.c * B), 256, 0, ctx->stream>>>(
                gin, m->pre_d[k - 1], (int64_t)L.c * B, L.act);
            ctx->launches++;
        }
        g = gin;
        cur ^= 1;
    }
    merge_backward_kernel<<<blocks_for((int64_t)L.dlat * B), 256, 0, ctx->stream>>>(
        g, zr, zq, L.dlat, B, L.merge, m->gr, m->gq);
    ctx->launches++;
    for (int s = 0; s < 2; ++s) {
        const int enc_i = s == 0 ? 0 : eq;  // a shared encoder accumulates both sides
        const float* enc = m->params + L.enc_size * enc_i;
        float* genc = m->grad + L.enc_size * enc_i;
        const float* gs = s == 0 ? m->gr : m->gq;
        int t = 0;
        for (int k = L.le - 1; k >= 0; --k) {
            const int cin = k == 0 ? L.din : L.c;
            const float* in = k == 0 ? m->x0[s] : m->post_e[s][k - 1];
            float* gin = pp[t];
            if (!gemm_bwd(m, enc + L.ew[k], in, gs, gin, genc + L.ew[k], genc + L.eb[k],
                          L.c, cin, B))
                return cudaErrorUnknown;
            if (k > 0) {
                dact_mul_kernel<<<blocks_for((int64_t)L.c * B), 256, 0, ctx->stream>>>(
                    gin, m->pre_e[s][k - 1], (int64_t)L.c * B, L.act);
                ctx->launches++;
            }
            gs = gin;
            t ^= 1;
        }
        hash_embed_backward_kernel<<<blocks_for(B, 128), 128, 0, ctx->stream>>>(
            s == 0 ? pr : pq, B, gs, embed_args(L), genc);
        ctx->launches++;
    }
    return cudaGetLastError();
}


// ---------------------------------------------------------------- tensor-core decoding
// Packed images: [encoder 0 layers][encoder 1 layers (cross)][decoder hidden layers],
// so that a query-side chain (encoder eq, then the decoder) is contiguous.
static cudaError_t hash_tc_prepare(ndf_hash_model* m) {
    const HashLayout& L = m->Ly;
    const int n = L.n_enc * L.le + L.ld - 1;
    const size_t lb = hash_tc_layer_bytes();
    cudaError_t e = cudaSuccess;
    if (!m->tc_w) {
        e = cudaMalloc(&m->tc_w, lb * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&m->tc_bias, sizeof(float) * 128 * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&m->tc_zr, sizeof(float) * 128 * (size_t)kHashTcMaxRefs);
        const int f8 = hash_tc_f8(L.L);
        const size_t nf = (size_t)(m->X + m->Y + m->Z) * (size_t)f8;
        if (e == cudaSuccess) e = cudaMalloc(&m->tc_ftab, sizeof(float) * std::max<size_t>(nf, 4));
        if (e == cudaSuccess) e = launch_hash_tc_ftab(L.L, f8, m->X, m->Y, m->Z, m->tc_ftab, m->ctx->stream);
        m->ctx->launches++;
        if (e != cudaSuccess) return e;
    }
    if (m->tc_ver == m->ver) return cudaSuccess;
    HashTcPack pk;
    pk.L = L.L;
    pk.f8 = hash_tc_f8(L.L);
    pk.ngrid = L.levels * L.F;
    for (int en = 0; en < L.n_enc; ++en)
        for (int k = 0; k < L.le; ++k) {
            pk.perm[pk.n] = k == 0;
            pk.cin[pk.n] = k == 0 ? L.din : L.c;
            pk.w[pk.n] = L.enc_size * en + L.ew[k];
            pk.b[pk.n] = L.enc_size * en + L.eb[k];
            ++pk.n;
        }
    for (int k = 0; k < L.ld - 1; ++k) {
        pk.perm[pk.n] = k == 0 && L.le == 0;  // grid-only: the merged embedding
        pk.cin[pk.n] = k == 0 ? L.ddec : L.c;
        pk.w[pk.n] = L.dw[k];
        pk.b[pk.n] = L.db[k];
        ++pk.n;
    }
    e = launch_hash_tc_pack(m->params, pk, m->tc_w, m->tc_bias, m->ctx->stream);
    m->ctx->launches++;
    if (e == cudaSuccess) m->tc_ver = m->ver;
    return e;
}

static HashTcArgs hash_tc_base(const ndf_hash_model* m) {
    HashTcArgs a;
    a.E = embed_args(m->Ly);
    a.measure = m->measure;
    a.X = m->X;
    a.Y = m->Y;
    a.Z = m->Z;
    a.status = m->ctx->flag.as<unsigned>() + 1;
    a.ftab = m->tc_ftab;
    a.f8 = hash_tc_f8(m->Ly.L);
    a.foff[0] = 0;
    a.foff[1] = m->X * a.f8;
    a.foff[2] = (m->X + m->Y) * a.f8;
    return a;
}

// CTAs per reference: the SMs shared among the references (the launcher caps it at
// the tile groups there are)
static int hash_tc_ctas(const ndf_hash_model* m, int64_t rows, int R) {
    (void)rows;
    const int c = (m->ctx->sm_count + R - 1) / R;
    return c < 1 ? 1 : c;
}

// encode-only launch: the FP32 latents of encoder `en` for rows vertices
// (vlist when given, else 0 .. rows-1) into lat[rows][128]
static cudaError_t hash_tc_encode(ndf_hash_model* m, int en, const int64_t* vlist, int64_t rows, float* lat) {
    const HashLayout& L = m->Ly;
    HashTcArgs a = hash_tc_base(m);
    a.tables = m->params + L.enc_size * en;
    a.wimg = m->tc_w + hash_tc_layer_bytes() * (size_t)(en * L.le);
    a.bias = m->tc_bias + (size_t)128 * (en * L.le);
    a.nL = L.le;
    a.n_enc = L.le;
    a.merge = -1;
    a.N = rows;
    if (vlist) {
        a.vlist_n = (int)rows;
        for (int64_t i = 0; i < rows; ++i) a.vlist[i] = vlist[i];
    }
    a.lat = lat;
    m->ctx->launches++;
    return launch_hash_tc(a, L.act, hash_tc_ctas(m, rows, 1), 1, m->ctx->stream);
}

// volumes of R <= kHashTcMaxRefs references into out[R][N] (device)
static cudaError_t hash_tc_decode(ndf_hash_model* m, const int64_t* refs, int R, float* out) {
    const HashLayout& L = m->Ly;
    ndf_ctx* ctx = m->ctx;
    const int64_t N = m->X * m->Y * m->Z;
    cudaError_t e = hash_tc_prepare(m);
    if (e != cudaSuccess) return e;
    // reference latents (encoder 0)
    if (L.le == 0) {
        HashTcArgs a = hash_tc_base(m);
        a.tables = m->params;
        a.vlist_n = R;
        for (int i = 0; i < R; ++i) a.vlist[i] = refs[i];
        e = launch_hash_tc_embed_refs(a, m->tc_zr, ctx->stream);
        ctx->launches++;
    } else {
        e = hash_tc_encode(m, 0, refs, R, m->tc_zr);
    }
    if (e != cudaSuccess) return e;
    const int eq = L.n_enc - 1;
    const bool cached = m->cache_q && hash_tc_cache_ok(L);
    if (cached && m->lat_ver != m->ver) {
        if (!m->tc_lat && (e = cudaMalloc(&m->tc_lat, sizeof(float) * 128 * (size_t)N)) != cudaSuccess) return e;
        if ((e = hash_tc_encode(m, eq, nullptr, N, m->tc_lat)) != cudaSuccess) return e;
        m->lat_ver = m->ver;
    }
    HashTcArgs a = hash_tc_base(m);
    a.merge = L.merge;
    a.zr = m->tc_zr;
    a.w_last = m->params + L.dw[L.ld - 1];
    a.b_last = m->params + L.db[L.ld - 1];
    a.N = N;
    a.out = out;
    const int first = cached ? L.n_enc * L.le : eq * L.le;
    a.wimg = m->tc_w + hash_tc_layer_bytes() * (size_t)first;
    a.bias = m->tc_bias + (size_t)128 * first;
    if (cached) {
        a.lat_in = m->tc_lat;
        a.nL = L.ld - 1;
        a.n_enc = 0;
    } else {
        a.tables = m->params + L.enc_size * eq;
        a.nL = L.le + L.ld - 1;
        a.n_enc = L.le;
    }
    ctx->launches++;
    return launch_hash_tc(a, L.act, hash_tc_ctas(m, N, R), R, ctx->stream);
}

// the FP32 path for one reference: the reference encoded once, queries in chunks
static cudaError_t hash_fp32_decode(ndf_hash_model* m, int64_t ref_idx, float* dev_out) {
    ndf_ctx* ctx = m->ctx;
    const HashLayout& L = m->Ly;
    const int64_t N = m->X * m->Y * m->Z;
    const int64_t chunk = std::min<int64_t>(N, 65536);
    cudaError_t e = hash_workspace(m, chunk);
    if (e != cudaSuccess) return e;
    vertex_positions_kernel<<<1, 32, 0, ctx->stream>>>(ref_idx, 1, m->X, m->Y, m->Z, m->pos);
    ctx->launches++;
    e = encode_side(m, 0, 0, m->pos, 1);
    const float* zr = latent(m, 0);
    for (int64_t v0 = 0; v0 < N && e == cudaSuccess; v0 += chunk) {
        const int64_t n = std::min(chunk, N - v0);
        vertex_positions_kernel<<<blocks_for(n), 256, 0, ctx->stream>>>(v0, n, m->X, m->Y, m->Z,
                                                                         m->pos + 3);
        ctx->launches++;
        e = encode_side(m, L.n_enc - 1, 1, m->pos + 3, n);
        if (e != cudaSuccess) break;
        merge_kernel<<<blocks_for((int64_t)L.dlat * n), 256, 0, ctx->stream>>>(
            zr, 0, latent(m, 1), L.dlat, n, L.merge, m->z);
        ctx->launches++;
        if ((e = decode_z(m, n)) != cudaSuccess) break;
        out_loss_kernel<<<blocks_for(n), 256, 0, ctx->stream>>>(m->pre_d[L.ld - 1], nullptr, n, m->measure,
                                                                 dev_out + v0, nullptr, nullptr);
        ctx->launches++;
        e = cudaGetLastError();
    }
    return e;
}
}  // namespace ndf

extern "C" {

void ndf_hash_arch_default(ndf_hash_arch* a) {
    if (!a) return;
    a->levels = 6;
    a->base_res = 16;
    a->log2_table = 22;
    a->feat = 2;
    a->n_freq = 12;
    a->width = 128;
    a->enc_layers = 6;
    a->dec_layers = 6;
    a->act = NDF_ACT_SNAKEALT;
    a->merge = NDF_MERGE_PRODUCT;
}

ndf_status ndf_hash_model_create(ndf_ctx* ctx, const ndf_hash_arch* arch, int measure, int cross,
                                 uint64_t seed, int64_t X, int64_t Y, int64_t Z,
                                 ndf_hash_model** out) {
    if (!ctx || !arch || !out) return NDF_ERR_ARG;
    *out = nullptr;
    if (measure != NDF_MEASURE_PEARSON && measure != NDF_MEASURE_MI_KSG)
        return fail(ctx, NDF_ERR_ARG, "unknown measure %d", measure);
    if (X < 1 || Y < 1 || Z < 1 || X * Y * Z > (int64_t(1) << 31))
        return fail(ctx, NDF_ERR_ARG, "bad decode grid");
    ndf_hash_model* m = new (std::nothrow) ndf_hash_model();
    if (!m) return NDF_ERR_OOM;
    m->ctx = ctx;
    m->arch = *arch;
    m->measure = measure;
    m->X = X;
    m->Y = Y;
    m->Z = Z;
    if (!m->Ly.init(*arch, cross ? 2 : 1)) {
        delete m;
        return fail(ctx, NDF_ERR_ARG, "bad hash-network architecture");
    }
    cudaSetDevice(ctx->device);
    const size_t bytes = sizeof(float) * (size_t)m->Ly.total;
    cudaError_t e = cudaMalloc(&m->params, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, bytes, ctx->stream);
    if (e != cudaSuccess) {
        ndf_hash_model_free(m);
        return cuda_fail(ctx, e, "hash model allocation");
    }
    // initialisation: tables U(-0.1, 0.1), weights U(-sqrt(6/in), sqrt(6/in)), biases 0, and a
    // zero last decoder layer (the untrained field is constant: without it, the sin^2 term
    // of Snake-family activations drifts the output and L1 training collapses it).  The
    // first encoder layer's weights on the Fourier columns start at kFourierInit of that
    // scale: at full scale the frequencies up to 2^(L-1) pi reach every latent feature, the
    // untrained encoder maps positions a cell apart to unrelated latents, the product merge
    // carries no dependence signal, and on a field whose pairs are mostly uncorrelated the
    // L1 loss keeps the network at the constant predictor
    std::vector<float> h((size_t)m->Ly.total, 0.0f);
    uint64_t st = seed * 0x9e3779b97f4a7c15ULL + 0x1234567ULL;
    auto unif = [&]() {
        st += 0x9e3779b97f4a7c15ULL;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    const HashLayout& L = m->Ly;
    for (int e_i = 0; e_i < L.n_enc; ++e_i) {
        const int64_t base = L.enc_size * e_i;
        for (int64_t i = 0; i < L.tables; ++i) h[(size_t)(base + i)] = (float)(0.1 * unif());
        for (int k = 0; k < L.le; ++k) {
            const int64_t cin = k == 0 ? L.din : L.c;
            const double a = sqrt(6.0 / (double)cin);
            for (int64_t i = 0; i < cin * L.c; ++i) {
                const int64_t col = i % cin;  // W[out][in]
                const bool fourier = k == 0 && col >= 3 && col < 3 + 6 * (int64_t)L.L;
                h[(size_t)(base + L.ew[k] + i)] = (float)((fourier ? kFourierInit : 1.0) * a * unif());
            }
        }
    }
    for (int k = 0; k < L.ld - 1; ++k) {
        const int64_t cin = k == 0 ? L.ddec : L.c;
        const double a = sqrt(6.0 / (double)cin);
        for (int64_t i = 0; i < cin * L.c; ++i) h[(size_t)(L.dw[k] + i)] = (float)(a * unif());
    }
    e = cudaMemcpyAsync(m->params, h.data(), bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        ndf_hash_model_free(m);
        return cuda_fail(ctx, e, "hash model initialisation");
    }
    m->decode_tc = hash_tc_eligible(m->Ly) ? 1 : 0;
    *out = m;
    return NDF_OK;
}

void ndf_hash_model_free(ndf_hash_model* m) {
    if (!m) return;
    if (m->ctx) cudaStreamSynchronize(m->ctx->stream);
    void* ps[] = {m->params, m->grad, m->m, m->v, m->ws, m->gemm_work, m->tc_w, m->tc_bias,
                  m->tc_zr, m->tc_lat, m->tc_ftab};
    for (void* q : ps)
        if (q) cudaFree(q);
    delete m;
}

int64_t ndf_hash_model_param_count(const ndf_hash_model* m) { return m ? m->Ly.total : -1; }

ndf_status ndf_hash_model_get_params(ndf_hash_model* m, float* out) {
    if (!m || !out) return NDF_ERR_ARG;
    const size_t bytes = sizeof(float) * (size_t)m->Ly.total;
    cudaError_t e = cudaMemcpyAsync(out, m->params, bytes, cudaMemcpyDefault, m->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->ctx->stream);
    return e == cudaSuccess ? NDF_OK : cuda_fail(m->ctx, e, "hash params download");
}

ndf_status ndf_hash_model_set_params(ndf_hash_model* m, const float* in) {
    if (!m || !in) return NDF_ERR_ARG;
    const size_t bytes = sizeof(float) * (size_t)m->Ly.total;
    cudaError_t e = cudaMemcpyAsync(m->params, in, bytes, cudaMemcpyDefault, m->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->ctx->stream);
    ++m->ver;
    return e == cudaSuccess ? NDF_OK : cuda_fail(m->ctx, e, "hash params upload");
}

// positions / targets / outputs may be host or device; staged through the workspace
// one training step on device batches (no copies, no host synchronisation): the
// summed |error| of the batch accumulates in m->loss
static cudaError_t hash_train_step(ndf_hash_model* m, const float* pr, const float* pq,
                                   const float* target, int64_t B, float lr) {
    ndf_ctx* ctx = m->ctx;
    cudaError_t e = cudaMemsetAsync(m->grad, 0, sizeof(float) * (size_t)m->Ly.total, ctx->stream);
    if (e == cudaSuccess) e = hash_forward_backward(m, pr, pq, target, B, nullptr);
    if (e != cudaSuccess) return e;
    ++m->t;
    ++m->ver;
    const float c1 = 1.0f - powf(0.9f, (float)m->t), c2 = 1.0f - powf(0.999f, (float)m->t);
    hash_adam_kernel<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(m->params, m->grad, m->m, m->v,
                                                                m->Ly.total, lr, 0.9f, 0.999f, 1e-8f,
                                                                c1, c2);
    ctx->launches++;
    return cudaGetLastError();
}

ndf_status ndf_hash_model_step(ndf_hash_model* m, const float* pr, const float* pq,
                               const float* target, int64_t B, float lr, int apply,
                               float* grad_out, double* loss_out) {
    if (!m || !pr || !pq || !target || B < 1) return NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    cudaSetDevice(ctx->device);
    cudaError_t e = hash_workspace(m, B);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hash workspace");
    const size_t pb = sizeof(float) * 3 * (size_t)B;
    e = cudaMemcpyAsync(m->pos, pr, pb, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->pos + 3 * B, pq, pb, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->tgt, target, sizeof(float) * B, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, sizeof(float) * (size_t)m->Ly.total, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, sizeof(double), ctx->stream);
    if (e == cudaSuccess) e = hash_forward_backward(m, m->pos, m->pos + 3 * B, m->tgt, B, nullptr);
    if (e == cudaSuccess && apply) {
        ++m->t;
        ++m->ver;
        const float c1 = 1.0f - powf(0.9f, (float)m->t), c2 = 1.0f - powf(0.999f, (float)m->t);
        hash_adam_kernel<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(
            m->params, m->grad, m->m, m->v, m->Ly.total, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
        ctx->launches++;
        e = cudaGetLastError();
    }
    double l = 0.0;
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, m->grad, sizeof(float) * (size_t)m->Ly.total, cudaMemcpyDefault,
                            ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hash step");
    if (loss_out) *loss_out = l / (double)B;
    return NDF_OK;
}

ndf_status ndf_hash_model_forward(ndf_hash_model* m, const float* pr, const float* pq, int64_t B,
                                  float* out) {
    if (!m || !pr || !pq || !out || B < 1) return NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    cudaSetDevice(ctx->device);
    cudaError_t e = hash_workspace(m, B);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hash workspace");
    const size_t pb = sizeof(float) * 3 * (size_t)B;
    e = cudaMemcpyAsync(m->pos, pr, pb, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->pos + 3 * B, pq, pb, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = hash_forward_backward(m, m->pos, m->pos + 3 * B, nullptr, B, m->graw);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, m->graw, sizeof(float) * B, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? NDF_OK : cuda_fail(ctx, e, "hash forward");
}

// the volume of one reference vertex (tensor-core decoder or the FP32 chain)
ndf_status ndf_hash_infer(ndf_hash_model* m, int64_t ref_idx, float* out) {
    return ndf_hash_infer_batch(m, &ref_idx, 1, out);
}

ndf_status ndf_hash_infer_batch(ndf_hash_model* m, const int64_t* refs, int32_t R, float* out) {
    if (!m || !refs || !out || R < 1) return NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    const int64_t N = m->X * m->Y * m->Z;
    for (int32_t i = 0; i < R; ++i)
        if (refs[i] < 0 || refs[i] >= N) return fail(ctx, NDF_ERR_ARG, "ref_idx out of range");
    cudaSetDevice(ctx->device);
    void* dev_out;
    bool is_host;
    const size_t bytes = sizeof(float) * (size_t)N * (size_t)R;
    ndf_status st = resolve_out(ctx, out, bytes, &dev_out, &is_host);
    if (st != NDF_OK) return st;
    float* o = static_cast<float*>(dev_out);
    cudaError_t e = cudaSuccess;
    if (m->decode_tc) {
        for (int32_t r0 = 0; r0 < R && e == cudaSuccess; r0 += kHashTcMaxRefs)
            e = hash_tc_decode(m, refs + r0, std::min<int32_t>(kHashTcMaxRefs, R - r0), o + (size_t)r0 * N);
    } else {
        for (int32_t r = 0; r < R && e == cudaSuccess; ++r) e = hash_fp32_decode(m, refs[r], o + (size_t)r * N);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hash decode");
    return finish_out(ctx, out, dev_out, bytes, is_host);
}

ndf_status ndf_hash_set_decode(ndf_hash_model* m, int32_t mode, int32_t cache_queries) {
    if (!m) return NDF_ERR_ARG;
    if (mode != NDF_HASH_DECODE_FP32 && mode != NDF_HASH_DECODE_TC)
        return fail(m->ctx, NDF_ERR_ARG, "unknown decode mode %d", mode);
    if (mode == NDF_HASH_DECODE_TC && !hash_tc_eligible(m->Ly))
        return fail(m->ctx, NDF_ERR_ARG,
                    "the tensor-core decoder needs width 128, at most 128 embedding inputs and a "
                    "product / sum / |difference| merge");
    if (cache_queries && (mode != NDF_HASH_DECODE_TC || !hash_tc_cache_ok(m->Ly)))
        return fail(m->ctx, NDF_ERR_ARG,
                    "the query-latent cache needs the tensor-core decoder, an encoder layer and two "
                    "decoder layers");
    m->decode_tc = mode;
    m->cache_q = cache_queries ? 1 : 0;
    if (!m->cache_q && m->tc_lat) {
        cudaStreamSynchronize(m->ctx->stream);
        cudaFree(m->tc_lat);
        m->tc_lat = nullptr;
        m->lat_ver = -1;
    }
    return NDF_OK;
}

int32_t ndf_hash_get_decode(const ndf_hash_model* m) { return m ? m->decode_tc : -1; }

// training on continuous samples renewed every pass (Sec. 4.3)
ndf_status ndf_hash_train(ndf_ctx* ctx, int ref_field, int query_field, int measure, int k,
                          const ndf_hash_arch* arch, const ndf_train_cfg* cfg_in,
                          ndf_hash_model** out) {
    if (!ctx || !arch || !out) return NDF_ERR_ARG;
    ndf_train_cfg cfg;
    if (cfg_in) cfg = *cfg_in;
    else ndf_train_cfg_default(&cfg);
    const Field *rf, *qf;
    ndf_status st = check_pair(ctx, ref_field, query_field, 0, &rf, &qf);
    if (st != NDF_OK) return st;
    if (measure == NDF_MEASURE_MI_KSG && (k < 1 || k >= rf->M || k > kKsgMaxK || rf->M > kKsgMaxM))
        return fail(ctx, NDF_ERR_ARG, "bad k or M for the KSG targets");
    if (cfg.n_triples < 1 || cfg.batch < 1 || cfg.max_passes < 1 || cfg.n_triples > (int64_t(1) << 31))
        return fail(ctx, NDF_ERR_ARG, "bad training configuration");
    ndf_hash_model* m = nullptr;
    if ((st = ndf_hash_model_create(ctx, arch, measure, ref_field != query_field, cfg.seed, qf->X,
                                    qf->Y, qf->Z, &m)) != NDF_OK)
        return st;
    if (measure == NDF_MEASURE_MI_KSG && (st = ensure_psi_table(ctx, rf->M + 1)) != NDF_OK) {
        ndf_hash_model_free(m);
        return st;
    }
    const int64_t T = cfg.n_triples, B = std::min(cfg.batch, T);
    float *pref = nullptr, *pq = nullptr, *tgt = nullptr;
    cudaError_t e = cudaMalloc(&pref, sizeof(float) * 3 * (size_t)T);
    if (e == cudaSuccess) e = cudaMalloc(&pq, sizeof(float) * 3 * (size_t)T);
    if (e == cudaSuccess) e = cudaMalloc(&tgt, sizeof(float) * (size_t)T);
    if (e == cudaSuccess) e = hash_workspace(m, B);
    SampleScratch sc;
    auto cleanup = [&]() {
        if (pref) cudaFree(pref);
        if (pq) cudaFree(pq);
        if (tgt) cudaFree(tgt);
        sc.release();
    };
    const auto t_start = std::chrono::steady_clock::now();
    float lr = cfg.lr;
    double best = 1e300;
    int bad = 0, decays = 0;
    for (int pass = 0; pass < cfg.max_passes && e == cudaSuccess; ++pass) {
        const auto g0 = std::chrono::steady_clock::now();
        e = sample_triples_dev(ctx, *rf, *qf, measure, k, T, cfg.seed + (uint64_t)pass, pref, pq, tgt, sc);
        m->gen_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - g0).count();
        if (e != cudaSuccess) break;
        // the pass's steps run back to back; its summed |error| is read once
        e = cudaMemsetAsync(m->loss, 0, sizeof(double), ctx->stream);
        for (int64_t b0 = 0; b0 < T && e == cudaSuccess; b0 += B)
            e = hash_train_step(m, pref + 3 * b0, pq + 3 * b0, tgt + b0, std::min(B, T - b0), lr);
        double pass_sum = 0.0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&pass_sum, m->loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) break;
        const double pass_loss = pass_sum / (double)T;
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
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (cfg.time_budget_s > 0.0 && el > cfg.time_budget_s) break;
    }
    m->train_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() - m->gen_seconds;
    m->n_triples = T;
    cleanup();
    if (e != cudaSuccess) {
        ndf_hash_model_free(m);
        return cuda_fail(ctx, e, "hash training");
    }
    *out = m;
    return NDF_OK;
}

ndf_status ndf_hash_model_info(const ndf_hash_model* m, int* passes, double* last_loss,
                               double* gen_seconds, double* train_seconds, int64_t* adam_steps) {
    if (!m) return NDF_ERR_ARG;
    if (passes) *passes = m->passes;
    if (last_loss) *last_loss = m->last_loss;
    if (gen_seconds) *gen_seconds = m->gen_seconds;
    if (train_seconds) *train_seconds = m->train_seconds;
    if (adam_steps) *adam_steps = m->t;
    return NDF_OK;
}

}  // extern "C"

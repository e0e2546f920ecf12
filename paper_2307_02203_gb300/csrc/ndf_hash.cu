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
// GPU design: activations are feature-major per sample ([B][c] row-major, which
// is a column-major [c][B] matrix), the dense layers are FP32 cuBLAS GEMMs (plain
// library GEMMs; FP32 for parity with the oracle), and everything between them
// (embedding, bias + activation, merge, output + loss, the hash-table scatter of
// the backward, Adam) is in the kernels below.
#include <cublas_v2.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <numeric>
#include <vector>

#include "ndf_internal.h"

namespace ndf {

constexpr int kHashMaxLevels = 8;
constexpr int kHashMaxLayers = 8;

struct HashLayout {
    int levels = 0, F = 0, L = 0, c = 0, le = 0, ld = 0, n_enc = 0, din = 0, act = 0, logT = 0;
    int merge = 0, dlat = 0, ddec = 0;  // latent width, decoder input width
    int64_t res[kHashMaxLevels] = {}, entries[kHashMaxLevels] = {}, toff[kHashMaxLevels] = {};
    int64_t ew[kHashMaxLayers] = {}, eb[kHashMaxLayers] = {};  // within an encoder
    int64_t dw[kHashMaxLayers] = {}, db[kHashMaxLayers] = {};  // absolute
    int64_t enc_size = 0, tables = 0, total = 0;
    bool init(const ndf_hash_arch& a, int n_enc_) {
        if (a.levels < 1 || a.levels > kHashMaxLevels || a.base_res < 2 || a.log2_table < 1 ||
            a.log2_table > 30 || a.feat < 1 || a.feat > 8 || a.n_freq < 0 || a.n_freq > 20 ||
            a.width < 1 || a.width > 1024 || a.enc_layers < 0 || a.enc_layers > kHashMaxLayers ||
            a.dec_layers < 1 || a.dec_layers > kHashMaxLayers || a.act < 0 || a.act > 2 ||
            a.merge < 0 || a.merge > 3)
            return false;
        if ((int64_t)a.base_res << (a.levels - 1) > (int64_t(1) << 20)) return false;
        levels = a.levels;
        F = a.feat;
        L = a.n_freq;
        c = a.width;
        le = a.enc_layers;
        ld = a.dec_layers;
        n_enc = n_enc_;
        act = a.act;
        logT = a.log2_table;
        merge = a.merge;
        din = 3 + 6 * L + levels * F;
        dlat = le > 0 ? c : din;
        ddec = merge == NDF_MERGE_CONCAT ? 2 * dlat : dlat;
        int64_t o = 0;
        for (int l = 0; l < levels; ++l) {
            res[l] = (int64_t)a.base_res << l;
            const double dense = (double)res[l] * (double)res[l] * (double)res[l];
            const int64_t cap = int64_t(1) << logT;
            entries[l] = dense <= (double)cap ? res[l] * res[l] * res[l] : cap;
            toff[l] = o;
            o += entries[l] * F;
        }
        tables = o;
        for (int k = 0; k < le; ++k) {
            ew[k] = o;
            o += (int64_t)(k == 0 ? din : c) * c;
            eb[k] = o;
            o += c;
        }
        enc_size = o;
        o = enc_size * n_enc;
        for (int k = 0; k < ld; ++k) {
            const int64_t out = k == ld - 1 ? 1 : c, in = k == 0 ? ddec : c;
            dw[k] = o;
            o += out * in;
            db[k] = o;
            o += out;
        }
        total = o;
        return true;
    }
};

// kernel-side copy of what the embedding needs
struct EmbedArgs {
    int levels, F, L, din;
    int res[kHashMaxLevels];
    int64_t entries[kHashMaxLevels], toff[kHashMaxLevels];
    unsigned char dense[kHashMaxLevels];
};

EmbedArgs embed_args(const HashLayout& Ly) {
    EmbedArgs e;
    e.levels = Ly.levels;
    e.F = Ly.F;
    e.L = Ly.L;
    e.din = Ly.din;
    for (int l = 0; l < Ly.levels; ++l) {
        e.res[l] = (int)Ly.res[l];
        e.entries[l] = Ly.entries[l];
        e.toff[l] = Ly.toff[l];
        e.dense[l] = (double)Ly.res[l] * Ly.res[l] * Ly.res[l] <= (double)(int64_t(1) << Ly.logT);
    }
    return e;
}

struct Cell {
    int64_t idx[8];
    float w[8];
};

__device__ __forceinline__ Cell level_cell(const EmbedArgs& E, int l, const float* p) {
    const int R = E.res[l];
    int i0[3];
    float t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = (p[a] + 1.0f) * 0.5f * (float)(R - 1);
        u = fminf(fmaxf(u, 0.0f), (float)(R - 1));
        i0[a] = min((int)floorf(u), R - 2);
        t[a] = u - (float)i0[a];
    }
    Cell c;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int x = i0[0] + (q & 1), y = i0[1] + ((q >> 1) & 1), z = i0[2] + ((q >> 2) & 1);
        if (E.dense[l]) {
            c.idx[q] = (int64_t)x + (int64_t)R * y + (int64_t)R * R * z;
        } else {
            const uint32_t h = (uint32_t)x * 1u ^ (uint32_t)y * 2654435761u ^ (uint32_t)z * 805459861u;
            c.idx[q] = (int64_t)(h % (uint32_t)E.entries[l]);
        }
        c.w[q] = ((q & 1) ? t[0] : 1.0f - t[0]) * (((q >> 1) & 1) ? t[1] : 1.0f - t[1]) *
                 (((q >> 2) & 1) ? t[2] : 1.0f - t[2]);
    }
    return c;
}

// x0[b][din] = embed(pos[b]) with the tables of one encoder
__global__ void hash_embed_kernel(const float* __restrict__ pos, int64_t B,
                                  const float* __restrict__ enc, EmbedArgs E,
                                  float* __restrict__ x0) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float p[3] = {pos[3 * b], pos[3 * b + 1], pos[3 * b + 2]};
    float* x = x0 + b * E.din;
    x[0] = p[0];
    x[1] = p[1];
    x[2] = p[2];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < E.L; ++i) {
            float s, c;
            sincospif(ldexpf(p[j], i), &s, &c);  // sin / cos(2^i pi p_j)
            x[3 + (j * E.L + i) * 2] = s;
            x[3 + (j * E.L + i) * 2 + 1] = c;
        }
    for (int l = 0; l < E.levels; ++l) {
        const Cell cl = level_cell(E, l, p);
        const float* tab = enc + E.toff[l];
        for (int f = 0; f < E.F; ++f) {
            float v = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; ++q) v += cl.w[q] * __ldg(tab + cl.idx[q] * E.F + f);
            x[3 + 6 * E.L + l * E.F + f] = v;
        }
    }
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
            for (int q = 0; q < 8; ++q) atomicAdd(tab + cl.idx[q] * E.F + f, cl.w[q] * gv);
        }
    }
}

__device__ __forceinline__ float act_f(int a, float x) {
    if (a == 0) return fmaxf(x, 0.0f);
    const float s = sinf(x);
    return (a == 1 ? x : 0.5f * x) + s * s;
}
__device__ __forceinline__ float dact_f(int a, float x) {
    if (a == 0) return x > 0.0f ? 1.0f : 0.0f;
    return (a == 1 ? 1.0f : 0.5f) + sinf(2.0f * x);
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

__device__ __forceinline__ float out_act(int measure, float x) {
    return measure == NDF_MEASURE_PEARSON ? tanhf(x) : log1pf(expf(-fabsf(x))) + fmaxf(x, 0.0f);
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
    const int64_t v = v0 + i, x = v % X, y = (v / X) % Y, z = v / (X * Y);
    pos[3 * i] = X > 1 ? -1.0f + 2.0f * (float)x / (float)(X - 1) : 0.0f;
    pos[3 * i + 1] = Y > 1 ? -1.0f + 2.0f * (float)y / (float)(Y - 1) : 0.0f;
    pos[3 * i + 2] = Z > 1 ? -1.0f + 2.0f * (float)z / (float)(Z - 1) : 0.0f;
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

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
    cublasHandle_t blas = nullptr;
    // workspace for a batch of up to cap samples
    int64_t cap = 0;
    float* ws = nullptr;
    float *x0[2] = {}, *pre_e[2][kHashMaxLayers] = {}, *post_e[2][kHashMaxLayers] = {};
    float *z = nullptr, *pre_d[kHashMaxLayers] = {}, *post_d[kHashMaxLayers] = {};
    float *ga = nullptr, *gb = nullptr, *gr = nullptr, *gq = nullptr;
    float *ones = nullptr, *graw = nullptr, *tgt = nullptr, *pos = nullptr;
    double* loss = nullptr;
    // training record
    int passes = 0;
    double last_loss = 0.0, gen_seconds = 0.0, train_seconds = 0.0;
    int64_t n_triples = 0;
};

namespace ndf {

static cudaError_t hash_workspace(ndf_hash_model* m, int64_t B) {
    if (B <= m->cap) return cudaSuccess;
    if (m->ws) cudaFree(m->ws);
    m->ws = nullptr;
    m->cap = 0;
    const HashLayout& L = m->Ly;
    const int64_t c = L.c, wmax = std::max<int64_t>(std::max<int64_t>(L.din, c), L.ddec);
    // loss (2 doubles), x0 x2, encoder pre/post x2 sides, z, decoder pre/post,
    // ga, gb (ping-pong), gr, gq (merge gradients), ones, graw, tgt, positions
    const int64_t floats = 4 + 2 * B * L.din + 2 * 2 * L.le * B * c + B * L.ddec +
                           2 * L.ld * B * c + 2 * B * wmax + 2 * B * L.dlat + 3 * B + 6 * B;
    cudaError_t e = cudaMalloc(&m->ws, sizeof(float) * (size_t)floats);
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
    m->ones = take(B);
    m->graw = take(B);
    m->tgt = take(B);
    m->pos = take(6 * B);
    fill_kernel<<<blocks_for(B), 256, 0, m->ctx->stream>>>(m->ones, B, 1.0f);
    m->cap = B;
    return cudaGetLastError();
}

static bool blas_ok(cublasStatus_t s) { return s == CUBLAS_STATUS_SUCCESS; }

// Y[c_out][B] = W x X[c_in][B] (W row-major [c_out][c_in])
static bool gemm_fwd(cublasHandle_t h, const float* W, const float* X, float* Y, int c_out,
                     int c_in, int64_t B) {
    const float one = 1.0f, zero = 0.0f;
    return blas_ok(cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, c_out, (int)B, c_in, &one, W, c_in, X,
                               c_in, &zero, Y, c_out));
}

// dX = W^T dY; dW += X dY^T; db += dY 1
static bool gemm_bwd(cublasHandle_t h, const float* W, const float* X, const float* dY, float* dX,
                     float* dW, float* db, const float* ones, int c_out, int c_in, int64_t B) {
    const float one = 1.0f, zero = 0.0f;
    if (dX && !blas_ok(cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, c_in, (int)B, c_out, &one, W, c_in,
                                   dY, c_out, &zero, dX, c_in)))
        return false;
    if (!blas_ok(cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, c_in, c_out, (int)B, &one, X, c_in, dY,
                             c_out, &one, dW, c_in)))
        return false;
    return blas_ok(cublasSgemv(h, CUBLAS_OP_N, c_out, (int)B, &one, dY, c_out, ones, 1, &one, db, 1));
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
        if (!gemm_fwd(m->blas, enc + L.ew[k], in, m->pre_e[s][k], L.c, cin, B))
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
        if (!gemm_fwd(m->blas, m->params + L.dw[k], in, m->pre_d[k], cout, cin, B))
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
        if (!gemm_bwd(m->blas, m->params + L.dw[k], in, g, gin, m->grad + L.dw[k], m->grad + L.db[k],
                      m->ones, cout, cin, B))
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
            if (!gemm_bwd(m->blas, enc + L.ew[k], in, gs, gin, genc + L.ew[k], genc + L.eb[k],
                          m->ones, L.c, cin, B))
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
    if (e != cudaSuccess || cublasCreate(&m->blas) != CUBLAS_STATUS_SUCCESS ||
        cublasSetStream(m->blas, ctx->stream) != CUBLAS_STATUS_SUCCESS) {
        ndf_hash_model_free(m);
        return e != cudaSuccess ? cuda_fail(ctx, e, "hash model allocation")
                                : fail(ctx, NDF_ERR_CUDA, "cuBLAS set-up failed");
    }
    // initialisation: tables U(-0.1, 0.1), weights U(-sqrt(6/in), sqrt(6/in)), biases 0, and a
    // zero last decoder layer (the untrained field is constant: without it, the sin^2 term
    // of Snake-family activations drifts the output and L1 training collapses it)
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
            for (int64_t i = 0; i < cin * L.c; ++i) h[(size_t)(base + L.ew[k] + i)] = (float)(a * unif());
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
    *out = m;
    return NDF_OK;
}

void ndf_hash_model_free(ndf_hash_model* m) {
    if (!m) return;
    if (m->ctx) cudaStreamSynchronize(m->ctx->stream);
    void* ps[] = {m->params, m->grad, m->m, m->v, m->ws};
    for (void* q : ps)
        if (q) cudaFree(q);
    if (m->blas) cublasDestroy(m->blas);
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
    return e == cudaSuccess ? NDF_OK : cuda_fail(m->ctx, e, "hash params upload");
}

// positions / targets / outputs may be host or device; staged through the workspace
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

// the volume of one reference vertex: the reference is encoded once, queries in chunks
ndf_status ndf_hash_infer(ndf_hash_model* m, int64_t ref_idx, float* out) {
    if (!m || !out) return NDF_ERR_ARG;
    ndf_ctx* ctx = m->ctx;
    const int64_t N = m->X * m->Y * m->Z;
    if (ref_idx < 0 || ref_idx >= N) return fail(ctx, NDF_ERR_ARG, "ref_idx out of range");
    cudaSetDevice(ctx->device);
    const int64_t chunk = std::min<int64_t>(N, 65536);
    cudaError_t e = hash_workspace(m, chunk);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hash workspace");
    void* dev_out;
    bool is_host;
    ndf_status st = resolve_out(ctx, out, sizeof(float) * (size_t)N, &dev_out, &is_host);
    if (st != NDF_OK) return st;
    const HashLayout& L = m->Ly;
    // the reference latent: side 0 with a batch of one
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
        out_loss_kernel<<<blocks_for(n), 256, 0, ctx->stream>>>(
            m->pre_d[L.ld - 1], nullptr, n, m->measure, static_cast<float*>(dev_out) + v0, nullptr,
            nullptr);
        ctx->launches++;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hash decode");
    return finish_out(ctx, out, dev_out, sizeof(float) * (size_t)N, is_host);
}

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
        double pass_sum = 0.0;
        for (int64_t b0 = 0; b0 < T && e == cudaSuccess; b0 += B) {
            const int64_t nb = std::min(B, T - b0);
            double l = 0.0;
            st = ndf_hash_model_step(m, pref + 3 * b0, pq + 3 * b0, tgt + b0, nb, lr, 1, nullptr, &l);
            if (st != NDF_OK) {
                cleanup();
                ndf_hash_model_free(m);
                return st;
            }
            pass_sum += l * (double)nb;
        }
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

// The hash-grid network's layout and the device functions that its FP32 kernels
// and its tensor-core decoder share: parameter layout, the embedding (Eq. 4 +
// the multi-resolution hash grid), activations, the output non-linearity.
#pragma once

#include <math.h>
#include <stdint.h>

#include "ndf.h"

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

inline EmbedArgs embed_args(const HashLayout& Ly) {
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
    uint32_t idx[8];  // entry index (< 2^30)
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
        if (E.dense[l]) {  // R^3 <= 2^T <= 2^30
            c.idx[q] = (uint32_t)x + (uint32_t)R * ((uint32_t)y + (uint32_t)R * (uint32_t)z);
        } else {
            const uint32_t h = (uint32_t)x * 1u ^ (uint32_t)y * 2654435761u ^ (uint32_t)z * 805459861u;
            c.idx[q] = h & (uint32_t)(E.entries[l] - 1);  // entries = 2^T
        }
        c.w[q] = ((q & 1) ? t[0] : 1.0f - t[0]) * (((q >> 1) & 1) ? t[1] : 1.0f - t[1]) *
                 (((q >> 2) & 1) ? t[2] : 1.0f - t[2]);
    }
    return c;
}


// The embedding of one position (FP32): emit(k, value) for k = 0 .. din-1 in
// order [p_0..2, (sin, cos)(2^i pi p_j) for j < 3, i < L, level features].
// embed_fourier emits the first 3 + 6 L entries, embed_grid the level features.
template <class Emit>
__device__ __forceinline__ void embed_fourier(const EmbedArgs& E, const float* p, Emit&& emit) {
    emit(0, p[0]);
    emit(1, p[1]);
    emit(2, p[2]);
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < E.L; ++i) {
            float s, c;
            sincospif(ldexpf(p[j], i), &s, &c);  // sin / cos(2^i pi p_j)
            emit(3 + (j * E.L + i) * 2, s);
            emit(4 + (j * E.L + i) * 2, c);
        }
}

// grid features of levels [l0, l1): emit(l * F + f, value).  With two features
// per entry, two levels at a time: their 16 corner loads are in flight together.
template <class Emit>
__device__ __forceinline__ void embed_levels(const EmbedArgs& E, const float* __restrict__ tables,
                                             const float* p, int l0, int l1, Emit&& emit) {
    int l = l0;
    if (E.F == 2) {
        for (; l + 1 < l1; l += 2) {
            const Cell ca = level_cell(E, l, p), cb = level_cell(E, l + 1, p);
            const float2* ta = reinterpret_cast<const float2*>(tables + E.toff[l]);
            const float2* tb = reinterpret_cast<const float2*>(tables + E.toff[l + 1]);
            float2 ga[8], gb[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                ga[q] = __ldg(ta + ca.idx[q]);
                gb[q] = __ldg(tb + cb.idx[q]);
            }
            float2 va = make_float2(0.0f, 0.0f), vb = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                va.x += ca.w[q] * ga[q].x;
                va.y += ca.w[q] * ga[q].y;
                vb.x += cb.w[q] * gb[q].x;
                vb.y += cb.w[q] * gb[q].y;
            }
            emit(l * 2, va.x);
            emit(l * 2 + 1, va.y);
            emit(l * 2 + 2, vb.x);
            emit(l * 2 + 3, vb.y);
        }
    }
    for (; l < l1; ++l) {
        const Cell cl = level_cell(E, l, p);
        const float* tab = tables + E.toff[l];
        for (int f = 0; f < E.F; ++f) {
            float v = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; ++q) v += cl.w[q] * __ldg(tab + (int64_t)cl.idx[q] * E.F + f);
            emit(l * E.F + f, v);
        }
    }
}

template <class Emit>
__device__ __forceinline__ void embed_grid(const EmbedArgs& E, const float* __restrict__ tables,
                                           const float* p, Emit&& emit) {
    embed_levels(E, tables, p, 0, E.levels, [&](int g, float v) { emit(3 + 6 * E.L + g, v); });
}

template <class Emit>
__device__ __forceinline__ void embed_point(const EmbedArgs& E, const float* __restrict__ tables,
                                            const float* p, Emit&& emit) {
    embed_fourier(E, p, emit);
    embed_grid(E, tables, p, emit);
}

// vertex v of an X x Y x Z grid -> its vertex-aligned position in [-1,1]^3
__device__ __forceinline__ void vertex_position(int64_t v, int64_t X, int64_t Y, int64_t Z, float* p) {
    const int64_t x = v % X, y = (v / X) % Y, z = v / (X * Y);
    p[0] = X > 1 ? -1.0f + 2.0f * (float)x / (float)(X - 1) : 0.0f;
    p[1] = Y > 1 ? -1.0f + 2.0f * (float)y / (float)(Y - 1) : 0.0f;
    p[2] = Z > 1 ? -1.0f + 2.0f * (float)z / (float)(Z - 1) : 0.0f;
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

__device__ __forceinline__ float out_act(int measure, float x) {
    return measure == NDF_MEASURE_PEARSON ? tanhf(x) : log1pf(expf(-fabsf(x))) + fmaxf(x, 0.0f);
}

}  // namespace ndf

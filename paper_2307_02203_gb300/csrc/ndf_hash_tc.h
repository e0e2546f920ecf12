// Host-side interface of the hash-grid network's tensor-core decoder
// (ndf_hash_tc.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hash_common.cuh"

namespace ndf {

constexpr int kHashTcMaxLayers = 16;  // tensor-core layers of one launch
constexpr int kHashTcMaxRefs = 64;    // vertices listed in the arguments

struct HashTcArgs {
    EmbedArgs E;
    const float* tables = nullptr;        // level tables of the encoder that embeds the rows
    const unsigned char* wimg = nullptr;  // nL weight images, hash_tc_layer_bytes() each
    const float* bias = nullptr;          // [nL][128]
    int nL = 0;                           // tensor-core layers in this launch
    int n_enc = 0;                        // of which the first n_enc are encoder layers
    int merge = -1;                       // ndf_merge; -1: encode-only (latents to lat)
    int measure = 0;
    const float* zr = nullptr;            // [R][128] reference latents (decode)
    const float* w_last = nullptr;        // [128] output layer (decode)
    const float* b_last = nullptr;        // its bias (device scalar)
    const float* lat_in = nullptr;        // [N][128] cached query latents (cached decode)
    const float* ftab = nullptr;          // per-axis Fourier features, FP32 [n][f8] per axis
    int64_t foff[3] = {};                 // offsets of the x, y, z tables in ftab
    int f8 = 0;                           // per-axis Fourier block: 2 L rounded up to 8
    int64_t N = 0, X = 1, Y = 1, Z = 1;   // rows; the grid that maps a vertex to its position
    int vlist_n = 0;                      // > 0: row r is vertex vlist[r] (encode-only)
    int64_t vlist[kHashTcMaxRefs] = {};
    float* out = nullptr;                 // decode: [R][N]
    float* lat = nullptr;                 // encode-only: [N][128] FP32 latents
    unsigned* status = nullptr;
};

// Column order of the embedding in the tensor-core operand: the Fourier features
// of axis j in block [j f8, j f8 + 2 L) (f8 = 2 L rounded up to 8, so that each
// axis block starts on a 16-byte chunk), then the position and the grid features
// from 3 f8 on.  Returns the embedding index (Eq. 4 order: p, Fourier, grid) of
// operand column kp, or -1 for a padding column.
__host__ __device__ inline int hash_tc_emb_source(int kp, int L, int f8, int ngrid) {
    if (kp < 3 * f8) {
        const int j = kp / f8, q = kp - j * f8;
        return q < 2 * L ? 3 + j * 2 * L + q : -1;
    }
    const int u = kp - 3 * f8;
    if (u < 3) return u;
    return u < 3 + ngrid ? 3 + 6 * L + (u - 3) : -1;
}

inline int hash_tc_f8(int L) { return (2 * L + 7) & ~7; }

// the layers to pack: parameter offsets of W[out=128][in=cin] and b[128]; perm:
// the layer's input is the embedding (its columns follow hash_tc_emb_source)
struct HashTcPack {
    int n = 0, L = 0, f8 = 0, ngrid = 0;
    int cin[3 * kHashMaxLayers] = {}, perm[3 * kHashMaxLayers] = {};
    int64_t w[3 * kHashMaxLayers] = {}, b[3 * kHashMaxLayers] = {};
};

size_t hash_tc_layer_bytes();
cudaError_t launch_hash_tc_pack(const float* params, const HashTcPack& pk, unsigned char* wimg,
                                float* bias, cudaStream_t st);
cudaError_t launch_hash_tc_embed_refs(const HashTcArgs& a, float* zr, cudaStream_t st);
// ftab[foff[j] + n * f8 + q] = (sin, cos)(2^(q/2) pi p_j(n)) for q < 2 L, else 0
cudaError_t launch_hash_tc_ftab(int L, int f8, int64_t X, int64_t Y, int64_t Z, float* ftab,
                                cudaStream_t st);
cudaError_t launch_hash_tc(const HashTcArgs& a, int act, int ctas_x, int R, cudaStream_t st);

}  // namespace ndf

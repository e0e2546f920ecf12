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
    int64_t N = 0, X = 1, Y = 1, Z = 1;   // rows; the grid that maps a vertex to its position
    int vlist_n = 0;                      // > 0: row r is vertex vlist[r] (encode-only)
    int64_t vlist[kHashTcMaxRefs] = {};
    float* out = nullptr;                 // decode: [R][N]
    float* lat = nullptr;                 // encode-only: [N][128] FP32 latents
    unsigned* status = nullptr;
};

// the layers to pack: parameter offsets of W[out=128][in=cin] and b[128]
struct HashTcPack {
    int n = 0;
    int cin[3 * kHashMaxLayers] = {};
    int64_t w[3 * kHashMaxLayers] = {}, b[3 * kHashMaxLayers] = {};
};

size_t hash_tc_layer_bytes();
cudaError_t launch_hash_tc_pack(const float* params, const HashTcPack& pk, unsigned char* wimg,
                                float* bias, cudaStream_t st);
cudaError_t launch_hash_tc_embed_refs(const HashTcArgs& a, float* zr, cudaStream_t st);
cudaError_t launch_hash_tc(const HashTcArgs& a, int act, int ctas_x, int R, cudaStream_t st);

}  // namespace ndf

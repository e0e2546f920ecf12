// Neural dependence field (Sec. 4): model state and kernel launchers shared by
// ndf_net.cu (network kernels, model calls) and ndf_train.cu (training data,
// training loop, volume decoding).
#pragma once

#include <cuda_bf16.h>

#include "ndf_internal.h"

namespace ndf {

// Fixed network widths of the tensor-core kernels: 4 dense grid levels x 16
// features = 64 features per position; input [f*f ; f+f] = 128; 3 hidden
// layers of 128; one output.
constexpr int kLevels = 4;
constexpr int kFeat = 16;
constexpr int kLF = kLevels * kFeat;  // 64
constexpr int kIn = 2 * kLF;          // 128
constexpr int kHid = 128;
constexpr int kWStride = kHid + 8;    // padded bf16 row stride of weights in shared memory

// Offsets (in floats) of the flat FP32 parameter vector; same layout as the
// FP64 oracle: grid levels (point-major, 16 features each), W1 [128][128], b1,
// W2, b2, W3, b3, w4 [128], b4.
struct NetLayout {
    int res[kLevels];
    int64_t grid_off[kLevels];
    int64_t n_grid;
    int64_t W1, b1, W2, b2, W3, b3, w4, b4, total;
    void init(const int r[kLevels]);
};

// CTAs of the training kernel whose weight-gradient sums are kept (at most)
constexpr int kMlpMaxParts = 256;

// Per-batch work buffers (grown on demand).
struct NetWork {
    int64_t cap = 0;
    float* fr = nullptr;          // [B][64] reference features
    float* fq = nullptr;          // [B][64] query features
    __nv_bfloat16* x = nullptr;   // [B][128] merged input
    float* wpart = nullptr;       // [3][kMlpMaxParts][128][128] the training CTAs' weight gradients
    float* cpart = nullptr;       // [kMlpMaxParts][4][5][128] their bias / output-layer column sums
    float* dx = nullptr;          // [B][128] input gradient
    float* pos = nullptr;         // [2][B][3] positions (when the caller passes host memory)
    float* target = nullptr;      // [B]
    double* loss = nullptr;       // [1]
    void release();
};

}  // namespace ndf

struct ndf_model {
    ndf_ctx* ctx = nullptr;
    ndf::NetLayout L;
    int measure = 0;           // 0 Pearson (tanh output), 1 MI (softplus output)
    int64_t X = 0, Y = 0, Z = 0;  // ensemble grid the positions refer to
    float* params = nullptr;   // FP32 master [total]
    float* grad = nullptr;     // [total]
    bool grad_zero = true;     // grad is all zero (cleared by the last Adam step or at allocation)
    float* m = nullptr;        // Adam first moment
    float* v = nullptr;        // Adam second moment
    __nv_bfloat16* grid_bf = nullptr;  // bf16 copy of the grid part
    __nv_bfloat16* wbf = nullptr;      // [3][128][128] bf16 W1..W3 ([out][in])
    int64_t t = 0;             // Adam steps taken
    ndf::NetWork work;
    // training record
    double last_loss = 0.0;
    int passes = 0;
    int64_t steps = 0;
    double gen_seconds = 0.0, train_seconds = 0.0;
    int64_t n_triples = 0;
};

namespace ndf {

ndf_status model_alloc(ndf_ctx* ctx, const int res[kLevels], int measure, int64_t X, int64_t Y,
                       int64_t Z, ndf_model** out);
void model_free(ndf_model* m);
cudaError_t model_init_params(ndf_model* m, uint64_t seed);
cudaError_t model_refresh_bf16(ndf_model* m);  // bf16 copies from the FP32 master
ndf_status ensure_work(ndf_model* m, int64_t B);

// One step on a batch of device positions (pr, pq: [B][3]) and targets: loss
// (accumulated in work.loss) and gradients; with update, one Adam step.
// keep_grad: leave this step's gradient in m->grad after the update (a caller reads it)
cudaError_t model_step(ndf_model* m, const float* pr, const float* pq, const float* target,
                       int64_t B, float lr, float beta1, float beta2, float eps, bool update,
                       bool keep_grad = false);
cudaError_t net_set_attributes();
cudaError_t model_forward(ndf_model* m, const float* pr, const float* pq, int64_t B, float* out);

// The MLP on tcgen05 (ndf_mlp_tc.cu), over the merged input in m->work.x: the
// forward alone (y = the network output), and the training pass (the L1 loss sum
// into m->work.loss, the gradients of the three layers and of the output layer
// added into m->grad, the input gradient in m->work.dx).
cudaError_t mlp_tc_forward(ndf_model* m, int64_t B, float* y);
cudaError_t mlp_tc_train(ndf_model* m, int64_t B, const float* target);

// Volume decoding for R references (vertex ids on the device): out[R][N].
cudaError_t model_infer(ndf_model* m, const int64_t* d_refs, int R, float* out);
// tcgen05 decoding of R references (vertex ids on the device): out[R][N]
cudaError_t launch_infer_tc(ndf_model* m, const int64_t* d_refs, int R, float* out);

}  // namespace ndf

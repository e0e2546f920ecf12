/*
 * CPU oracle of the paper's neural dependence field architecture (Sec. 4.1-4.2,
 * Fig. 2): TEST INFRASTRUCTURE ONLY, FP64.
 *
 *   embed(p)  = [p_x, p_y, p_z,
 *                for axis j, frequency i < L: sin(2^i pi p_j), cos(2^i pi p_j)   (Eq. 4),
 *                for level l < levels, feature f < F: trilinear hash-grid feature]
 *   hash grid level l: R_l = base_res * 2^l points per axis, corner-aligned on
 *             [-1,1]^3 (u = (p + 1) / 2 * (R_l - 1), i0 = min(floor(u), R_l - 2));
 *             entries E_l = min(2^T, R_l^3): dense index x + R y + R^2 z when R^3 <= 2^T,
 *             else (x * 1 XOR y * 2654435761 XOR z * 805459861) mod 2^T in uint32
 *   encoder   enc_layers linear layers (first D_in -> width, then width -> width),
 *             activation after every layer but the last; enc_layers = 0 is the
 *             grid-only ablation (Sec. 6.4): the latent is the embedding itself
 *   merge     0: z = enc(p_ref) * enc(p_q) elementwise (the paper's choice), and the
 *             ablations of Sec. 4.1: 1 sum, 2 absolute difference, 3 concatenation
 *             [enc(p_ref); enc(p_q)]; one shared encoder and grid (n_enc = 1, self
 *             fields) or one per variable (n_enc = 2, cross fields: encoder 0 for
 *             the reference, 1 for the query)
 *   decoder   dec_layers linear layers (first |z| -> width, then width -> width,
 *             last -> 1), activation after every layer but the last, then tanh
 *             (Pearson) or softplus (MI)
 *   act       0 ReLU, 1 Snake x + sin^2 x, 2 SnakeAlt x / 2 + sin^2 x
 *   loss      mean |y - target| (L1, Eq. 3)
 * Parameters (flat, in this order): per encoder e: level tables [E_l][F] for
 * l = 0..levels-1, then its layers (W[out][in], b[out]) in order; then the
 * decoder layers (W, b).
 */
#ifndef NDF_HASH_NET_ORACLE_H
#define NDF_HASH_NET_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t levels, base_res, log2_table, feat, n_freq, width, enc_layers, dec_layers;
    int32_t n_enc, measure, act, merge;
} oracle_hash_shape;

int64_t oracle_hash_param_count(const oracle_hash_shape* s);

/* out[B] = network(pr[b], pq[b]).  Returns 0 or -1. */
int oracle_hash_forward(const oracle_hash_shape* s, const double* params, int64_t B,
                        const double* pr, const double* pq, double* out);

/* The same network with BF16 operands: every product of an encoder layer and
 * of a decoder hidden layer takes its weight and its input rounded to BF16
 * (oracle_bf16_round); sums, biases, activations, the merge and the output layer
 * stay FP64.  This is the arithmetic of a BF16 tensor-core decoder (BF16
 * operands, wide accumulation).  Returns 0 or -1. */
int oracle_hash_forward_bf16(const oracle_hash_shape* s, const double* params, int64_t B,
                             const double* pr, const double* pq, double* out);

/* x -> FP32 (round to nearest) -> BF16 (8 significant bits, round to nearest,
 * ties to even); beyond the FP32 range Inf, NaN stays NaN. */
double oracle_bf16_round(double x);

/* Mean L1 loss and its gradient with respect to every parameter (hand-written
 * backward).  grad has oracle_hash_param_count entries.  Returns 0 or -1. */
int oracle_hash_loss_grad(const oracle_hash_shape* s, const double* params, int64_t B,
                          const double* pr, const double* pq, const double* target,
                          double* loss, double* grad);

#ifdef __cplusplus
}
#endif
#endif

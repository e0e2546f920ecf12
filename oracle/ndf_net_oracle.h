/*
 * CPU FP64 oracle of the neural dependence field (Sec. 4) -- TEST
 * INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline).  Plain loops,
 * no blocking, shares no code with the CUDA library.
 *
 * Network (Sec. 4.1-4.3, in the dense-grid / ReLU form the library trains):
 *   f(p)  = concat over levels l of the trilinear interpolation of a dense
 *           feature grid with res[l] points per axis, corner-aligned on
 *           [-1,1]^3, `feat` features per point                (Sec. 4.2)
 *   x     = [ f(p_ref) * f(p_q) ; f(p_ref) + f(p_q) ]           (multiplicative
 *           merge, symmetric in the two positions, Sec. 4.1)
 *   h1..3 = ReLU(W x + b), 3 hidden layers of width `hidden`
 *   o     = w4 . h3 + b4 ;  y = tanh(o) (Pearson) or softplus(o) (MI)
 *   L     = mean |y - target|                                   (Eq. 3, L1)
 * Adam (Kingma & Ba) for the parameter update (Sec. 4.3).
 *
 * Parameter layout (doubles, in this order): grid levels (level-major, then
 * point (z*R + y)*R + x, then feature), W1 [hidden][2*L*feat] row-major, b1,
 * W2 [hidden][hidden], b2, W3, b3, w4 [hidden], b4 [1].
 */
#ifndef NDF_NET_ORACLE_H
#define NDF_NET_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int levels;
    int res[8];
    int feat;
    int hidden;
    int measure; /* 0: tanh output (Pearson), 1: softplus output (MI) */
} oracle_net_shape;

int64_t oracle_ndf_param_count(const oracle_net_shape* s);

/* features f(p) of one position: out[levels * feat] */
void oracle_ndf_encode(const oracle_net_shape* s, const double* params, const double* p,
                       double* out);

/* y[b] for B position pairs (pr, pq: [B][3]) */
void oracle_ndf_forward(const oracle_net_shape* s, const double* params, int64_t B,
                        const double* pr, const double* pq, double* y);

/* mean L1 loss; grad (may be NULL) receives dL/dparams in the parameter layout */
double oracle_ndf_loss_grad(const oracle_net_shape* s, const double* params, int64_t B,
                            const double* pr, const double* pq, const double* target,
                            double* grad);

/* the same loss and gradient, plus gabs = (1/B) sum_b |gradient of sample b|:
 * the magnitude of the summed terms, which bounds how much rounding in the
 * individual terms can move the (cancelling) sum */
double oracle_ndf_loss_grad_abs(const oracle_net_shape* s, const double* params, int64_t B,
                                const double* pr, const double* pq, const double* target,
                                double* grad, double* gabs);

/* one Adam step (t = step number, starting at 1) on n parameters */
void oracle_adam_step(int64_t n, double* params, const double* grad, double* m, double* v,
                      int64_t t, double lr, double beta1, double beta2, double eps);

#ifdef __cplusplus
}
#endif
#endif

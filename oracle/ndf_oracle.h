/*
 * CPU oracle for the dependence-volume hot path.  TEST INFRASTRUCTURE ONLY:
 * the test suite, the smoke check and the benchmark's CPU-baseline leg are the
 * only callers.  It shares no code with the CUDA library and is never on the
 * product path.
 *
 * Everything here is the plain definition, computed slowly:
 *   - Pearson's r (Sec. 3.1, Eq. 1) in FP64, two-pass;
 *   - the Kraskov-Stoegbauer-Grassberger k-NN mutual-information estimator,
 *     algorithm 1 of the estimator the paper cites in Sec. 3.2 / Sec. 6.2
 *     (max-norm in the joint space, strict counts, self excluded), by brute
 *     force with FP32 distances and long-double digamma sums;
 *   - its algorithm 2 (the second estimator of the same article): the extents
 *     of each member's k-nearest set in each marginal, non-strict counts;
 *   - digamma at positive integers by the recurrence psi(n+1) = psi(n) + 1/n.
 */
#ifndef NDF_ORACLE_H
#define NDF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Pearson r of two length-M samples (Eq. 1); returns 0 if either variance is 0. */
double oracle_pearson(const float* x, const float* y, int64_t M);

/* r between the reference vertex of ref_field and vertices of q_field; fields
 * are float[M][N]; verts (nverts entries) selects query vertices, or NULL for
 * all N in order.  out has nverts (or N) doubles.  Returns 0 or -1. */
int oracle_pearson_volume(const float* ref_field, const float* q_field, int64_t M, int64_t N,
                          int64_t ref_idx, const int64_t* verts, int64_t nverts, double* out,
                          int nthreads);

/* psi(n) for integer n >= 1 (recurrence from psi(1) = -Euler gamma, long double) */
double oracle_digamma_int(int64_t n);

/* KSG algorithm-1 estimate for one pair of samples.  eps/nx/ny (length M, may be
 * NULL) receive the per-member k-th-neighbour distance and marginal counts.
 * Returns MI in nats, or NaN on bad arguments (need 1 <= k < M). */
double oracle_ksg_pair(const float* x, const float* y, int64_t M, int k, float* eps, int32_t* nx,
                       int32_t* ny);

/* KSG MI between the reference vertex and the selected query vertices. */
int oracle_ksg_volume(const float* ref_field, const float* q_field, int64_t M, int64_t N,
                      int64_t ref_idx, int k, const int64_t* verts, int64_t nverts, double* out,
                      int nthreads);
/* oracle_ksg_pair for the reference vertex against each of verts[0..nverts):
 * eps/nx/ny are [nverts][M] (row i for verts[i]), mi is [nverts].  0, or -1 for
 * bad arguments. */
int oracle_ksg_pairs(const float* ref_field, const float* q_field, int64_t M, int64_t N,
                     int64_t ref_idx, int k, const int64_t* verts, int64_t nverts, float* eps,
                     int32_t* nx, int32_t* ny, double* mi, int nthreads);

/* KSG algorithm-2 estimate for one pair of samples.  ex/ey/nx/ny (length M, may
 * be NULL) receive per member the marginal extents of its neighbour set and the
 * non-strict marginal counts.  Returns MI in nats, or NaN (need 1 <= k < M). */
double oracle_ksg2_pair(const float* x, const float* y, int64_t M, int k, float* ex, float* ey,
                        int32_t* nx, int32_t* ny);

/* KSG algorithm-2 MI between the reference vertex and the selected query vertices. */
int oracle_ksg2_volume(const float* ref_field, const float* q_field, int64_t M, int64_t N,
                       int64_t ref_idx, int k, const int64_t* verts, int64_t nverts, double* out,
                       int nthreads);

/* Member column at a continuous position p in [-1,1]^3 (Sec. 4.3: training
 * samples are read from the ensemble by trilinear interpolation).  field is
 * float[M][Z][Y][X], vertex i of an axis of n vertices at -1 + 2 i / (n - 1)
 * (an axis of one vertex is constant).  FP32, in this order per axis:
 *   u  = ((p + 1) * 0.5) * (n - 1), clamped to [0, n - 1]
 *   i0 = min(floor(u), n - 2) (0 when n = 1), w = u - i0, i1 = min(i0 + 1, n - 1)
 *   lerp(a, b, w) = a * (1 - w) + b * w, first along x, then y, then z.
 * out receives M floats.  Returns 0, or -1 on bad arguments. */
int oracle_interp_column(const float* field, int64_t M, int64_t X, int64_t Y, int64_t Z,
                         const float p[3], float* out);

/* number of OpenMP threads a parallel region gets with the given request */
int oracle_threads(int nthreads);

#ifdef __cplusplus
}
#endif
#endif

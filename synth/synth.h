/*
 * Seeded synthetic ensemble generator (input data only; none of the method's
 * arithmetic lives here).  Shared by the CPU oracle's tests and the CUDA
 * library's tests and benchmark, which read the same generated bytes.
 */
#ifndef SYNTH_H
#define SYNTH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { SYNTH_LATENT_NONE = 0, SYNTH_LATENT_SINX = 1, SYNTH_LATENT_THREE_MODES = 2 };
enum { SYNTH_TRANSFORM_NONE = 0, SYNTH_TRANSFORM_QUAD = 1, SYNTH_TRANSFORM_ALTERNATING = 2 };

typedef struct {
    uint64_t seed;
    int stream;            /* noise stream: 0 for field A, 1 for field B, ... */
    double sigma[3];       /* Gaussian smoothing widths in vertices: x, y, z (0 = none) */
    int latent_kind;       /* SYNTH_LATENT_* */
    double latent_period_x;/* period in vertices of the SINX mode */
    int transform;         /* SYNTH_TRANSFORM_* */
    double share;          /* weight of the stream-0 pre-transform field (0 = independent) */
} synth_params;

/* Fill out[M][Z][Y][X]; returns 0, -1 on bad arguments, -2 on allocation failure.
 * nthreads <= 0 keeps the OpenMP default. Deterministic for a given seed. */
int synth_field(float* out, int64_t M, int64_t Z, int64_t Y, int64_t X, const synth_params* p,
                int nthreads);

/* one N(0,1) draw of the counter-based generator (exposed for tests) */
double synth_normal(uint64_t seed, uint64_t domain, uint64_t counter);

#ifdef __cplusplus
}
#endif
#endif

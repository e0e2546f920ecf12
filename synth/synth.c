/*
 * Seeded synthetic ensemble generator.
 *
 * This module produces the input fields that both the CPU oracle and the CUDA
 * library read (the same bytes, in the same process).  It holds none of the
 * method's arithmetic: no correlation, no mutual information, no network.  It
 * stands in for the CSEns weather ensemble of Sec. 6.1 (1000 members on a
 * 250 x 352 x 20 grid), which is not available, with fields of the same shape.
 *
 * Recipe (per member m of field f):
 *   1. white noise w(v) ~ N(0,1) at every vertex, drawn from a counter-based
 *      generator: SplitMix64's output mix applied to key + (c+1)*golden, two
 *      64-bit draws per value turned into one normal by Box-Muller (cos branch);
 *   2. g = separable Gaussian smoothing of w with sigma = (sx, sy, sz) vertices,
 *      kernel truncated at ceil(4 sigma), each 1-D kernel normalised so that
 *      sum(k^2) = 1 (unit variance away from the boundary), boundaries
 *      reflected (d c b a | a b c d | d c b a);
 *   3. u = g + L_m(v), the shared latent mode(s) with N(0,1) amplitudes a_{m,q};
 *   4. for a second field that shares the first one's latent structure:
 *      u_B = share * u_A + sqrt(1 - share^2) * g_B;
 *   5. the per-vertex non-linear transform (none / v + 0.3 v^2 / alternating by
 *      vertical level: even z -> v + 0.3 v^2, odd z -> sign(v) |v|^1.5).
 *
 * Layout of the output: float out[M][Z][Y][X], vertex v = (z*Y + y)*X + x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "synth.h"

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t ctr_u64(uint64_t key, uint64_t ctr) {
    return mix64(key + (ctr + 1ULL) * 0x9e3779b97f4a7c15ULL);
}

static inline uint64_t domain_key(uint64_t seed, uint64_t domain) {
    return mix64(seed ^ (domain * 0xd1b54a32d192ed03ULL + 0x632be59bd9b4e019ULL));
}

/* one N(0,1) value from counter c under key: Box-Muller, cosine branch */
static inline double ctr_normal(uint64_t key, uint64_t c) {
    uint64_t h1 = ctr_u64(key, 2 * c);
    uint64_t h2 = ctr_u64(key, 2 * c + 1);
    double u1 = ((double)(h1 >> 11) + 1.0) * 0x1.0p-53; /* (0, 1] */
    double u2 = (double)(h2 >> 11) * 0x1.0p-53;         /* [0, 1) */
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

double synth_normal(uint64_t seed, uint64_t domain, uint64_t counter) {
    return ctr_normal(domain_key(seed, domain), counter);
}

static int64_t reflect_idx(int64_t i, int64_t n) {
    int64_t p = 2 * n;
    i %= p;
    if (i < 0) i += p;
    return i < n ? i : p - 1 - i;
}

typedef struct {
    int R;
    float* w; /* 2R+1 taps */
} kern1d;

static int make_kernel(double sigma, kern1d* k) {
    if (!(sigma > 0.0)) {
        k->R = 0;
        k->w = (float*)malloc(sizeof(float));
        if (!k->w) return -1;
        k->w[0] = 1.0f;
        return 0;
    }
    int R = (int)ceil(4.0 * sigma);
    k->R = R;
    k->w = (float*)malloc(sizeof(float) * (size_t)(2 * R + 1));
    if (!k->w) return -1;
    double* t = (double*)malloc(sizeof(double) * (size_t)(2 * R + 1));
    if (!t) return -1;
    double s2 = 0.0;
    for (int i = -R; i <= R; ++i) {
        double v = exp(-0.5 * (double)i * (double)i / (sigma * sigma));
        t[i + R] = v;
        s2 += v * v;
    }
    double nrm = 1.0 / sqrt(s2);
    for (int i = 0; i < 2 * R + 1; ++i) k->w[i] = (float)(t[i] * nrm);
    free(t);
    return 0;
}

/* separable smoothing of one member volume in place (a, scratch b, row buffer r) */
static void smooth3(float* a, float* b, float* rowbuf, int64_t Z, int64_t Y, int64_t X,
                    const kern1d* kx, const kern1d* ky, const kern1d* kz) {
    /* x pass: a -> b */
    for (int64_t zy = 0; zy < Z * Y; ++zy) {
        const float* src = a + zy * X;
        float* dst = b + zy * X;
        int R = kx->R;
        for (int64_t i = -R; i < X + R; ++i) rowbuf[i + R] = src[reflect_idx(i, X)];
        for (int64_t x = 0; x < X; ++x) dst[x] = 0.0f;
        for (int t = 0; t <= 2 * R; ++t) {
            float w = kx->w[t];
            const float* s = rowbuf + t;
            for (int64_t x = 0; x < X; ++x) dst[x] += w * s[x];
        }
    }
    /* y pass: b -> a */
    for (int64_t z = 0; z < Z; ++z) {
        for (int64_t y = 0; y < Y; ++y) {
            float* dst = a + (z * Y + y) * X;
            for (int64_t x = 0; x < X; ++x) dst[x] = 0.0f;
            for (int t = -ky->R; t <= ky->R; ++t) {
                float w = ky->w[t + ky->R];
                const float* s = b + (z * Y + reflect_idx(y + t, Y)) * X;
                for (int64_t x = 0; x < X; ++x) dst[x] += w * s[x];
            }
        }
    }
    /* z pass: a -> b, then copy back */
    int64_t P = Y * X;
    for (int64_t z = 0; z < Z; ++z) {
        float* dst = b + z * P;
        for (int64_t i = 0; i < P; ++i) dst[i] = 0.0f;
        for (int t = -kz->R; t <= kz->R; ++t) {
            float w = kz->w[t + kz->R];
            const float* s = a + reflect_idx(z + t, Z) * P;
            for (int64_t i = 0; i < P; ++i) dst[i] += w * s[i];
        }
    }
    memcpy(a, b, sizeof(float) * (size_t)(Z * P));
}

static double latent_value(const synth_params* p, const double* amp, int64_t z, int64_t y,
                           int64_t x, int64_t Z, int64_t Y, int64_t X) {
    const double two_pi = 6.283185307179586;
    if (p->latent_kind == SYNTH_LATENT_SINX) {
        return amp[0] * sin(two_pi * (double)x / p->latent_period_x);
    }
    if (p->latent_kind == SYNTH_LATENT_THREE_MODES) {
        /* wavelengths = extent / q for q = 1, 2, 3 */
        double s = 0.0;
        for (int q = 1; q <= 3; ++q) {
            double fx = sin(two_pi * q * ((double)x + 0.5) / (double)X + 0.7 * q);
            double fy = sin(two_pi * q * ((double)y + 0.5) / (double)Y + 1.3 * q);
            double fz = 1.0 + 0.5 * cos(3.141592653589793 * q * ((double)z + 0.5) / (double)Z);
            s += amp[q - 1] * 1.4 * fx * fy * fz;
        }
        return s;
    }
    return 0.0;
}

static double transform_value(int kind, double u, int64_t z) {
    if (kind == SYNTH_TRANSFORM_QUAD) return u + 0.3 * u * u;
    if (kind == SYNTH_TRANSFORM_ALTERNATING) {
        if ((z & 1) == 0) return u + 0.3 * u * u;
        double a = fabs(u);
        double r = a * sqrt(a);
        return u < 0.0 ? -r : r;
    }
    return u;
}

/* pre-transform value u (GRF + latent) of member m of a given stream */
static void member_pre(float* out, float* scratch, float* rowbuf, int64_t m, int64_t Z, int64_t Y,
                       int64_t X, const synth_params* p, int stream, int with_latent,
                       const kern1d* k3) {
    int64_t N = Z * Y * X;
    uint64_t key_noise = domain_key(p->seed, 0x100ULL + (uint64_t)stream);
    uint64_t key_lat = domain_key(p->seed, 0x200ULL);
    for (int64_t v = 0; v < N; ++v) out[v] = (float)ctr_normal(key_noise, (uint64_t)(m * N + v));
    smooth3(out, scratch, rowbuf, Z, Y, X, &k3[0], &k3[1], &k3[2]);
    if (with_latent && p->latent_kind != SYNTH_LATENT_NONE) {
        double amp[3];
        for (int q = 0; q < 3; ++q) amp[q] = ctr_normal(key_lat, (uint64_t)(m * 3 + q));
        for (int64_t z = 0; z < Z; ++z)
            for (int64_t y = 0; y < Y; ++y)
                for (int64_t x = 0; x < X; ++x) {
                    int64_t v = (z * Y + y) * X + x;
                    out[v] = (float)((double)out[v] + latent_value(p, amp, z, y, x, Z, Y, X));
                }
    }
}

int synth_field(float* out, int64_t M, int64_t Z, int64_t Y, int64_t X, const synth_params* p,
                int nthreads) {
    if (!out || !p || M <= 0 || Z <= 0 || Y <= 0 || X <= 0) return -1;
    if (p->share < 0.0 || p->share > 1.0) return -1;
    int64_t N = Z * Y * X;
    kern1d k3[3];
    if (make_kernel(p->sigma[0], &k3[0]) || make_kernel(p->sigma[1], &k3[1]) ||
        make_kernel(p->sigma[2], &k3[2]))
        return -2;
    int64_t maxpad = X + 2 * (int64_t)k3[0].R;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        float* scratch = (float*)malloc(sizeof(float) * (size_t)N);
        float* other = (float*)malloc(sizeof(float) * (size_t)N);
        float* rowbuf = (float*)malloc(sizeof(float) * (size_t)maxpad);
        if (!scratch || !other || !rowbuf) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t m = 0; m < M; ++m) {
                float* dst = out + m * N;
                int shared = p->share > 0.0;
                /* a field with shared structure takes its latent modes through the shared part */
                member_pre(dst, scratch, rowbuf, m, Z, Y, X, p, p->stream, !shared, k3);
                if (shared) {
                    member_pre(other, scratch, rowbuf, m, Z, Y, X, p, 0, 1, k3);
                    double c = sqrt(1.0 - p->share * p->share);
                    for (int64_t v = 0; v < N; ++v)
                        dst[v] = (float)(p->share * (double)other[v] + c * (double)dst[v]);
                }
                if (p->transform != SYNTH_TRANSFORM_NONE) {
                    for (int64_t z = 0; z < Z; ++z) {
                        float* pl = dst + z * Y * X;
                        for (int64_t i = 0; i < Y * X; ++i)
                            pl[i] = (float)transform_value(p->transform, (double)pl[i], z);
                    }
                }
            }
        }
        free(scratch);
        free(other);
        free(rowbuf);
    }
    for (int i = 0; i < 3; ++i) free(k3[i].w);
    return failed ? -2 : 0;
}

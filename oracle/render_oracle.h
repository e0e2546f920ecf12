/*
 * CPU oracle for the headless volume ray-march of decoded dependence volumes
 * (Sec. 5: a dependence field displayed by direct volume rendering with a
 * transfer function, or as an iso-surface; Sec. 6.5: the difference of two
 * reference fields).  TEST INFRASTRUCTURE ONLY, FP64, one pixel at a time.
 *
 * Definitions (the CUDA renderer follows the same ones in FP32):
 *   volume      phi[z][y][x], X, Y, Z >= 2, vertex-aligned on [-1,1]^3:
 *               vertex i of an axis of n vertices sits at -1 + 2 i / (n - 1)
 *   sample      trilinear interpolation at p, the cell coordinate
 *               u = (p + 1) / 2 * (n - 1) clamped to [0, n - 1]; with a second
 *               volume the sample is phi_a(p) - phi_b(p)
 *   camera      pinhole: f = normalize(target - eye), r = normalize(f x up),
 *               u = r x f; pixel (i, j) (j = 0 at the top) looks along
 *               normalize(f + sx r + sy u), sx = (2 (i + 0.5) / W - 1) t a,
 *               sy = (1 - 2 (j + 0.5) / H) t, t = tan(fov_y / 2), a = W / H
 *   ray         slab intersection with [-1,1]^3 -> [t0, t1] (t0 >= 0); samples
 *               at t_k = t0 + (k + 0.5) step while t_k < t1
 *   tf          n_tf RGBA entries over [vmin, vmax]: s = clamp((v - vmin) /
 *               (vmax - vmin), 0, 1) * (n_tf - 1), linear between entries;
 *               A is an opacity per unit length
 *   DVR         alpha_k = 1 - exp(-A_k step); front to back:
 *               C += (1 - T) alpha_k rgb_k, T += (1 - T) alpha_k; pixel =
 *               (C + (1 - T) bg.rgb, T + (1 - T) bg.a)
 *   ISO         first k >= 1 with (v_{k-1} - iso) and (v_k - iso) of opposite
 *               sign or v_k == iso; hit t = t_{k-1} + (iso - v_{k-1}) /
 *               (v_k - v_{k-1}) step (t_k when the two are equal); normal =
 *               central differences of the sample at the hit with h = step,
 *               turned toward the viewer; pixel = tf(iso).rgb * (ambient +
 *               (1 - ambient) max(0, n . -dir)), alpha 1; no hit -> bg
 */
#ifndef NDF_RENDER_ORACLE_H
#define NDF_RENDER_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double eye[3], target[3], up[3];
    double fov_y_deg;
    int32_t width, height;
    double step;
    int32_t mode;  // 0 = DVR, 1 = ISO
    double iso;
    double vmin, vmax;
    double background[4];
    double ambient;
    int32_t n_tf;
    const double* tf;  // [n_tf][4]
} oracle_render_cfg;

/* Renders into out[H][W][4] (RGBA, FP64).  vol_b may be NULL.  Returns 0, or -1
 * on bad arguments. */
int oracle_render(const float* vol_a, const float* vol_b, int64_t X, int64_t Y, int64_t Z,
                  const oracle_render_cfg* cfg, double* out, int nthreads);

#ifdef __cplusplus
}
#endif
#endif

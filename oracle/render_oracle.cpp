// CPU oracle of the headless volume ray-march (see render_oracle.h for the
// definitions).  Test infrastructure only.
#include "render_oracle.h"

#include <algorithm>
#include <cmath>

#include <omp.h>

namespace {

struct V3 {
    double x, y, z;
};
V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 mul(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
V3 normalize(V3 a) {
    double n = std::sqrt(dot(a, a));
    return n > 0.0 ? mul(a, 1.0 / n) : a;
}

struct Vol {
    const float* a;
    const float* b;
    int64_t X, Y, Z;
    double at(const float* v, int64_t x, int64_t y, int64_t z) const {
        return (double)v[(z * Y + y) * X + x];
    }
    double tri(const float* v, V3 p) const {
        auto cell = [](double c, int64_t n, int64_t& i0, double& w) {
            double u = (c + 1.0) * 0.5 * (double)(n - 1);
            u = std::min(std::max(u, 0.0), (double)(n - 1));
            i0 = std::min((int64_t)std::floor(u), n - 2);
            w = u - (double)i0;
        };
        int64_t x0, y0, z0;
        double wx, wy, wz;
        cell(p.x, X, x0, wx);
        cell(p.y, Y, y0, wy);
        cell(p.z, Z, z0, wz);
        double c = 0.0;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    double w = (dx ? wx : 1.0 - wx) * (dy ? wy : 1.0 - wy) * (dz ? wz : 1.0 - wz);
                    c += w * at(v, x0 + dx, y0 + dy, z0 + dz);
                }
        return c;
    }
    double sample(V3 p) const { return b ? tri(a, p) - tri(b, p) : tri(a, p); }
};

void tf_lookup(const oracle_render_cfg& c, double v, double rgba[4]) {
    double s = (v - c.vmin) / (c.vmax - c.vmin);
    s = std::min(std::max(s, 0.0), 1.0) * (double)(c.n_tf - 1);
    int i0 = std::min((int)std::floor(s), c.n_tf - 2);
    if (c.n_tf == 1) i0 = 0;
    double w = c.n_tf == 1 ? 0.0 : s - (double)i0;
    for (int q = 0; q < 4; ++q) {
        double lo = c.tf[4 * i0 + q];
        double hi = c.n_tf == 1 ? lo : c.tf[4 * (i0 + 1) + q];
        rgba[q] = lo + w * (hi - lo);
    }
}

}  // namespace

extern "C" int oracle_render(const float* vol_a, const float* vol_b, int64_t X, int64_t Y,
                             int64_t Z, const oracle_render_cfg* cfg, double* out, int nthreads) {
    if (!vol_a || !cfg || !out || X < 2 || Y < 2 || Z < 2 || cfg->width < 1 || cfg->height < 1 ||
        !(cfg->step > 0.0) || cfg->n_tf < 1 || !cfg->tf || !(cfg->vmax > cfg->vmin))
        return -1;
    const oracle_render_cfg c = *cfg;
    const Vol vol{vol_a, vol_b, X, Y, Z};
    const V3 eye{c.eye[0], c.eye[1], c.eye[2]};
    const V3 f = normalize(sub(V3{c.target[0], c.target[1], c.target[2]}, eye));
    const V3 r = normalize(cross(f, V3{c.up[0], c.up[1], c.up[2]}));
    const V3 u = cross(r, f);
    const double t = std::tan(c.fov_y_deg * 3.14159265358979323846 / 360.0);
    const double aspect = (double)c.width / (double)c.height;
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < c.height; ++j) {
        for (int64_t i = 0; i < c.width; ++i) {
            double* px = out + (j * c.width + i) * 4;
            const double sx = (2.0 * ((double)i + 0.5) / c.width - 1.0) * t * aspect;
            const double sy = (1.0 - 2.0 * ((double)j + 0.5) / c.height) * t;
            const V3 d = normalize(add(f, add(mul(r, sx), mul(u, sy))));
            // slab intersection with [-1,1]^3
            double t0 = 0.0, t1 = 1e300;
            const double o[3] = {eye.x, eye.y, eye.z}, dd[3] = {d.x, d.y, d.z};
            bool hit_box = true;
            for (int a = 0; a < 3; ++a) {
                if (dd[a] == 0.0) {
                    if (o[a] < -1.0 || o[a] > 1.0) hit_box = false;
                    continue;
                }
                double ta = (-1.0 - o[a]) / dd[a], tb = (1.0 - o[a]) / dd[a];
                if (ta > tb) std::swap(ta, tb);
                t0 = std::max(t0, ta);
                t1 = std::min(t1, tb);
            }
            for (int q = 0; q < 4; ++q) px[q] = c.background[q];
            if (!hit_box || !(t0 < t1)) continue;
            if (c.mode == 0) {
                double C[3] = {0.0, 0.0, 0.0}, T = 0.0;
                for (int64_t k = 0;; ++k) {
                    const double tk = t0 + ((double)k + 0.5) * c.step;
                    if (!(tk < t1)) break;
                    double rgba[4];
                    tf_lookup(c, vol.sample(add(eye, mul(d, tk))), rgba);
                    const double al = 1.0 - std::exp(-rgba[3] * c.step);
                    for (int q = 0; q < 3; ++q) C[q] += (1.0 - T) * al * rgba[q];
                    T += (1.0 - T) * al;
                }
                for (int q = 0; q < 3; ++q) px[q] = C[q] + (1.0 - T) * c.background[q];
                px[3] = T + (1.0 - T) * c.background[3];
            } else {
                double vprev = 0.0, tprev = 0.0;
                for (int64_t k = 0;; ++k) {
                    const double tk = t0 + ((double)k + 0.5) * c.step;
                    if (!(tk < t1)) break;
                    const double v = vol.sample(add(eye, mul(d, tk)));
                    if (k > 0 && ((vprev - c.iso) * (v - c.iso) < 0.0 || v == c.iso)) {
                        const double th = v == vprev ? tk : tprev + (c.iso - vprev) / (v - vprev) * c.step;
                        const V3 p = add(eye, mul(d, th));
                        const double h = c.step;
                        V3 g{vol.sample(add(p, V3{h, 0, 0})) - vol.sample(sub(p, V3{h, 0, 0})),
                             vol.sample(add(p, V3{0, h, 0})) - vol.sample(sub(p, V3{0, h, 0})),
                             vol.sample(add(p, V3{0, 0, h})) - vol.sample(sub(p, V3{0, 0, h}))};
                        V3 n = normalize(g);
                        const V3 l = mul(d, -1.0);
                        if (dot(n, l) < 0.0) n = mul(n, -1.0);
                        const double lam = c.ambient + (1.0 - c.ambient) * std::max(0.0, dot(n, l));
                        double rgba[4];
                        tf_lookup(c, c.iso, rgba);
                        for (int q = 0; q < 3; ++q) px[q] = rgba[q] * lam;
                        px[3] = 1.0;
                        break;
                    }
                    vprev = v;
                    tprev = tk;
                }
            }
        }
    }
    return 0;
}

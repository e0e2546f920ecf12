// Headless volume ray-march of a dependence volume (Sec. 5: the decoded field is
// shown by direct volume rendering with a transfer function or as an
// iso-surface; Sec. 6.5: the difference of two reference fields) into an RGBA
// buffer.  One thread per pixel; the volume (and the optional second one) is
// read through L1 with trilinear interpolation in FP32.
//
// Definitions (shared with the FP64 CPU oracle):
//   volume   phi[z][y][x], vertex-aligned on [-1,1]^3 (vertex i of n at -1 + 2i/(n-1));
//            sample = trilinear at the clamped cell coordinate, minus the second
//            volume's sample when one is given
//   camera   pinhole from eye / target / up / vertical field of view
//   ray      slab intersection with [-1,1]^3, samples at t0 + (k + 1/2) step < t1
//   DVR      transfer function (RGBA table over [vmin, vmax], linear between
//            entries, A = opacity per unit length), alpha = 1 - exp(-A step),
//            front-to-back compositing over the background
//   ISO      first sign change of (v - iso) between consecutive samples, linear
//            refinement, central-difference normal (h = step) turned to the
//            viewer, Lambert headlight with an ambient term
#include <math.h>

#include "ndf_internal.h"

namespace ndf {

struct RenderParams {
    const float* a;
    const float* b;
    int X, Y, Z;
    float3 eye, f, r, u;
    float tan_half, aspect;
    int W, H;
    float step;
    int mode;
    float iso, vmin, vmax, ambient;
    float4 bg;
    const float4* tf;
    int n_tf;
};

__device__ __forceinline__ float tri(const float* __restrict__ v, int X, int Y, int Z, float3 p) {
    auto cell = [](float c, int n, int& i0, float& w) {
        float q = (c + 1.0f) * 0.5f * (float)(n - 1);
        q = fminf(fmaxf(q, 0.0f), (float)(n - 1));
        i0 = min((int)floorf(q), n - 2);
        w = q - (float)i0;
    };
    int x0, y0, z0;
    float wx, wy, wz;
    cell(p.x, X, x0, wx);
    cell(p.y, Y, y0, wy);
    cell(p.z, Z, z0, wz);
    const int64_t sx = 1, sy = X, sz = (int64_t)X * Y;
    const float* q = v + z0 * sz + y0 * sy + x0;
    const float c00 = __ldg(q) * (1.0f - wx) + __ldg(q + sx) * wx;
    const float c01 = __ldg(q + sy) * (1.0f - wx) + __ldg(q + sy + sx) * wx;
    const float c10 = __ldg(q + sz) * (1.0f - wx) + __ldg(q + sz + sx) * wx;
    const float c11 = __ldg(q + sz + sy) * (1.0f - wx) + __ldg(q + sz + sy + sx) * wx;
    const float c0 = c00 * (1.0f - wy) + c01 * wy;
    const float c1 = c10 * (1.0f - wy) + c11 * wy;
    return c0 * (1.0f - wz) + c1 * wz;
}

__device__ __forceinline__ float sample(const RenderParams& P, float3 p) {
    const float s = tri(P.a, P.X, P.Y, P.Z, p);
    return P.b ? s - tri(P.b, P.X, P.Y, P.Z, p) : s;
}

__device__ __forceinline__ float4 tf_lookup(const RenderParams& P, float v) {
    float s = (v - P.vmin) / (P.vmax - P.vmin);
    s = fminf(fmaxf(s, 0.0f), 1.0f) * (float)(P.n_tf - 1);
    if (P.n_tf == 1) return P.tf[0];
    const int i0 = min((int)floorf(s), P.n_tf - 2);
    const float w = s - (float)i0;
    const float4 lo = P.tf[i0], hi = P.tf[i0 + 1];
    return make_float4(lo.x + w * (hi.x - lo.x), lo.y + w * (hi.y - lo.y), lo.z + w * (hi.z - lo.z),
                       lo.w + w * (hi.w - lo.w));
}

__device__ __forceinline__ float3 axpy(float3 o, float t, float3 d) {
    return make_float3(o.x + t * d.x, o.y + t * d.y, o.z + t * d.z);
}

__global__ void __launch_bounds__(128) render_kernel(RenderParams P, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= P.W || j >= P.H) return;
    const float sx = (2.0f * ((float)i + 0.5f) / (float)P.W - 1.0f) * P.tan_half * P.aspect;
    const float sy = (1.0f - 2.0f * ((float)j + 0.5f) / (float)P.H) * P.tan_half;
    float3 d = make_float3(P.f.x + sx * P.r.x + sy * P.u.x, P.f.y + sx * P.r.y + sy * P.u.y,
                           P.f.z + sx * P.r.z + sy * P.u.z);
    const float inv = 1.0f / sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
    d = make_float3(d.x * inv, d.y * inv, d.z * inv);
    float t0 = 0.0f, t1 = 3.0e38f;
    bool hit_box = true;
    const float o[3] = {P.eye.x, P.eye.y, P.eye.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == 0.0f) {
            if (o[a] < -1.0f || o[a] > 1.0f) hit_box = false;
            continue;
        }
        float ta = (-1.0f - o[a]) / dd[a], tb = (1.0f - o[a]) / dd[a];
        if (ta > tb) {
            const float s = ta;
            ta = tb;
            tb = s;
        }
        t0 = fmaxf(t0, ta);
        t1 = fminf(t1, tb);
    }
    float4 px = P.bg;
    if (hit_box && t0 < t1) {
        if (P.mode == NDF_RENDER_DVR) {
            float cr = 0.0f, cg = 0.0f, cb = 0.0f, T = 0.0f;
            for (int k = 0;; ++k) {
                const float tk = t0 + ((float)k + 0.5f) * P.step;
                if (!(tk < t1)) break;
                const float4 c = tf_lookup(P, sample(P, axpy(P.eye, tk, d)));
                const float al = 1.0f - expf(-c.w * P.step);
                const float wgt = (1.0f - T) * al;
                cr += wgt * c.x;
                cg += wgt * c.y;
                cb += wgt * c.z;
                T += wgt;
            }
            px = make_float4(cr + (1.0f - T) * P.bg.x, cg + (1.0f - T) * P.bg.y,
                             cb + (1.0f - T) * P.bg.z, T + (1.0f - T) * P.bg.w);
        } else {
            float vprev = 0.0f, tprev = 0.0f;
            for (int k = 0;; ++k) {
                const float tk = t0 + ((float)k + 0.5f) * P.step;
                if (!(tk < t1)) break;
                const float v = sample(P, axpy(P.eye, tk, d));
                if (k > 0 && ((vprev - P.iso) * (v - P.iso) < 0.0f || v == P.iso)) {
                    const float th = v == vprev ? tk : tprev + (P.iso - vprev) / (v - vprev) * P.step;
                    const float3 p = axpy(P.eye, th, d);
                    const float h = P.step;
                    float3 g = make_float3(
                        sample(P, make_float3(p.x + h, p.y, p.z)) - sample(P, make_float3(p.x - h, p.y, p.z)),
                        sample(P, make_float3(p.x, p.y + h, p.z)) - sample(P, make_float3(p.x, p.y - h, p.z)),
                        sample(P, make_float3(p.x, p.y, p.z + h)) - sample(P, make_float3(p.x, p.y, p.z - h)));
                    const float gn = sqrtf(g.x * g.x + g.y * g.y + g.z * g.z);
                    if (gn > 0.0f) g = make_float3(g.x / gn, g.y / gn, g.z / gn);
                    float nl = -(g.x * d.x + g.y * d.y + g.z * d.z);
                    if (nl < 0.0f) nl = -nl;  // normal turned toward the viewer
                    const float lam = P.ambient + (1.0f - P.ambient) * fmaxf(0.0f, nl);
                    const float4 c = tf_lookup(P, P.iso);
                    px = make_float4(c.x * lam, c.y * lam, c.z * lam, 1.0f);
                    break;
                }
                vprev = v;
                tprev = tk;
            }
        }
    }
    out[(int64_t)j * P.W + i] = px;
}

}  // namespace ndf

using namespace ndf;

extern "C" ndf_status ndf_render_volume(ndf_ctx* ctx, const float* vol_a, const float* vol_b,
                                        int64_t X, int64_t Y, int64_t Z, const ndf_render_cfg* cfg,
                                        float* out_rgba) {
    if (!ctx) return NDF_ERR_ARG;
    if (!vol_a || !cfg || !out_rgba) return fail(ctx, NDF_ERR_ARG, "null pointer");
    if (X < 2 || Y < 2 || Z < 2 || X * Y * Z > ((int64_t)1 << 31))
        return fail(ctx, NDF_ERR_ARG, "volume needs 2 <= X, Y, Z and at most 2^31 vertices");
    if (cfg->width < 1 || cfg->height < 1 || (int64_t)cfg->width * cfg->height > (1 << 28))
        return fail(ctx, NDF_ERR_ARG, "bad image size");
    if (!(cfg->step > 0.0f) || cfg->n_tf < 1 || !cfg->tf || !(cfg->vmax > cfg->vmin) ||
        (cfg->mode != NDF_RENDER_DVR && cfg->mode != NDF_RENDER_ISO) ||
        !(cfg->fov_y_deg > 0.0f && cfg->fov_y_deg < 180.0f))
        return fail(ctx, NDF_ERR_ARG, "bad render configuration");
    // camera basis in FP64 on the host
    double e[3] = {cfg->eye[0], cfg->eye[1], cfg->eye[2]};
    double f[3] = {cfg->target[0] - e[0], cfg->target[1] - e[1], cfg->target[2] - e[2]};
    double up[3] = {cfg->up[0], cfg->up[1], cfg->up[2]};
    auto norm = [](double* v) {
        const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (n > 0.0)
            for (int q = 0; q < 3; ++q) v[q] /= n;
        return n;
    };
    if (norm(f) == 0.0) return fail(ctx, NDF_ERR_ARG, "eye and target coincide");
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    if (norm(r) == 0.0) return fail(ctx, NDF_ERR_ARG, "up is parallel to the view direction");
    double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    cudaSetDevice(ctx->device);
    const size_t vbytes = sizeof(float) * (size_t)(X * Y * Z);
    const size_t tbytes = sizeof(float4) * (size_t)cfg->n_tf;
    const bool a_dev = pointer_kind(vol_a) == PTR_DEVICE;
    const bool b_dev = !vol_b || pointer_kind(vol_b) == PTR_DEVICE;
    // scratch: transfer function, then host volumes
    size_t need = (tbytes + 255) / 256 * 256 + (a_dev ? 0 : vbytes) + (b_dev ? 0 : vbytes);
    cudaError_t err = ctx->render_buf.reserve(need);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "render scratch");
    char* base = ctx->render_buf.as<char>();
    float4* d_tf = reinterpret_cast<float4*>(base);
    char* cur = base + (tbytes + 255) / 256 * 256;
    const float* da = vol_a;
    const float* db = vol_b;
    err = cudaMemcpyAsync(d_tf, cfg->tf, tbytes, cudaMemcpyHostToDevice, ctx->stream);
    if (err == cudaSuccess && !a_dev) {
        err = cudaMemcpyAsync(cur, vol_a, vbytes, cudaMemcpyHostToDevice, ctx->stream);
        da = reinterpret_cast<const float*>(cur);
        cur += vbytes;
    }
    if (err == cudaSuccess && !b_dev) {
        err = cudaMemcpyAsync(cur, vol_b, vbytes, cudaMemcpyHostToDevice, ctx->stream);
        db = reinterpret_cast<const float*>(cur);
    }
    if (err != cudaSuccess) return cuda_fail(ctx, err, "render upload");
    const size_t obytes = sizeof(float4) * (size_t)cfg->width * (size_t)cfg->height;
    void* dev_out;
    bool is_host;
    ndf_status st = resolve_out(ctx, out_rgba, obytes, &dev_out, &is_host);
    if (st != NDF_OK) return st;
    RenderParams P;
    P.a = da;
    P.b = db;
    P.X = (int)X;
    P.Y = (int)Y;
    P.Z = (int)Z;
    P.eye = make_float3((float)e[0], (float)e[1], (float)e[2]);
    P.f = make_float3((float)f[0], (float)f[1], (float)f[2]);
    P.r = make_float3((float)r[0], (float)r[1], (float)r[2]);
    P.u = make_float3((float)u[0], (float)u[1], (float)u[2]);
    P.tan_half = (float)tan((double)cfg->fov_y_deg * 3.14159265358979323846 / 360.0);
    P.aspect = (float)((double)cfg->width / (double)cfg->height);
    P.W = cfg->width;
    P.H = cfg->height;
    P.step = cfg->step;
    P.mode = cfg->mode;
    P.iso = cfg->iso;
    P.vmin = cfg->vmin;
    P.vmax = cfg->vmax;
    P.ambient = cfg->ambient;
    P.bg = make_float4(cfg->background[0], cfg->background[1], cfg->background[2], cfg->background[3]);
    P.tf = d_tf;
    P.n_tf = cfg->n_tf;
    const dim3 block(16, 8), grid((cfg->width + 15) / 16, (cfg->height + 7) / 8);
    render_kernel<<<grid, block, 0, ctx->stream>>>(P, static_cast<float4*>(dev_out));
    ctx->launches++;
    if ((err = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, err, "render launch");
    return finish_out(ctx, out_rgba, dev_out, obytes, is_host);
}

// CPU FP64 oracle of the neural dependence field -- TEST INFRASTRUCTURE ONLY
// (see ndf_net_oracle.h).  Forward and backward written out layer by layer.
#include "ndf_net_oracle.h"

#include <cmath>
#include <vector>

namespace {

struct Offsets {
    int64_t grid[8];
    int64_t W1, b1, W2, b2, W3, b3, w4, b4, total;
    int in;
};

Offsets offsets(const oracle_net_shape* s) {
    Offsets o{};
    int64_t p = 0;
    for (int l = 0; l < s->levels; ++l) {
        o.grid[l] = p;
        int64_t r = s->res[l];
        p += r * r * r * s->feat;
    }
    const int H = s->hidden;
    o.in = 2 * s->levels * s->feat;
    o.W1 = p; p += (int64_t)H * o.in;
    o.b1 = p; p += H;
    o.W2 = p; p += (int64_t)H * H;
    o.b2 = p; p += H;
    o.W3 = p; p += (int64_t)H * H;
    o.b3 = p; p += H;
    o.w4 = p; p += H;
    o.b4 = p; p += 1;
    o.total = p;
    return o;
}

// one axis of one level: lower corner index and fractional weight
void axis(double p, int R, int* i0, double* w) {
    double u = (p + 1.0) * 0.5 * (double)(R - 1);
    double fl = std::floor(u);
    int i = (int)fl;
    if (i < 0) i = 0;
    if (i > R - 2) i = R - 2;
    *i0 = i;
    *w = u - (double)i;
}

// trilinear corners of position p at level l: point indices and weights
void corners(const oracle_net_shape* s, int l, const double* p, int64_t idx[8], double wt[8]) {
    const int R = s->res[l];
    int ix, iy, iz;
    double wx, wy, wz;
    axis(p[0], R, &ix, &wx);
    axis(p[1], R, &iy, &wy);
    axis(p[2], R, &iz, &wz);
    for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        idx[c] = ((int64_t)(iz + dz) * R + (iy + dy)) * R + (ix + dx);
        wt[c] = (dx ? wx : 1.0 - wx) * (dy ? wy : 1.0 - wy) * (dz ? wz : 1.0 - wz);
    }
}

double act(int measure, double o) {
    if (measure == 0) return std::tanh(o);
    return o > 30.0 ? o : std::log1p(std::exp(o));  // softplus
}

double dact(int measure, double o) {
    if (measure == 0) {
        double t = std::tanh(o);
        return 1.0 - t * t;
    }
    return 1.0 / (1.0 + std::exp(-o));  // sigmoid
}

// dense layer y = W x + b (W: [out][in])
void dense(const double* W, const double* b, const double* x, int in, int out, double* y) {
    for (int i = 0; i < out; ++i) {
        double a = b[i];
        for (int j = 0; j < in; ++j) a += W[(int64_t)i * in + j] * x[j];
        y[i] = a;
    }
}

}  // namespace

extern "C" {

int64_t oracle_ndf_param_count(const oracle_net_shape* s) { return offsets(s).total; }

void oracle_ndf_encode(const oracle_net_shape* s, const double* params, const double* p,
                       double* out) {
    Offsets o = offsets(s);
    const int F = s->feat;
    for (int l = 0; l < s->levels; ++l) {
        int64_t idx[8];
        double wt[8];
        corners(s, l, p, idx, wt);
        for (int f = 0; f < F; ++f) {
            double a = 0.0;
            for (int c = 0; c < 8; ++c) a += wt[c] * params[o.grid[l] + idx[c] * F + f];
            out[l * F + f] = a;
        }
    }
}

// Shared by forward and backward: all intermediate values of one sample.
struct Sample {
    std::vector<double> fr, fq, x, z1, h1, z2, h2, z3, h3;
    double o = 0.0, y = 0.0;
};

static void forward_one(const oracle_net_shape* s, const Offsets& o, const double* params,
                        const double* pr, const double* pq, Sample& S) {
    const int LF = s->levels * s->feat, H = s->hidden;
    S.fr.assign(LF, 0.0);
    S.fq.assign(LF, 0.0);
    oracle_ndf_encode(s, params, pr, S.fr.data());
    oracle_ndf_encode(s, params, pq, S.fq.data());
    S.x.assign(2 * LF, 0.0);
    for (int i = 0; i < LF; ++i) {
        S.x[i] = S.fr[i] * S.fq[i];
        S.x[LF + i] = S.fr[i] + S.fq[i];
    }
    S.z1.assign(H, 0.0); S.h1.assign(H, 0.0);
    S.z2.assign(H, 0.0); S.h2.assign(H, 0.0);
    S.z3.assign(H, 0.0); S.h3.assign(H, 0.0);
    dense(params + o.W1, params + o.b1, S.x.data(), 2 * LF, H, S.z1.data());
    for (int i = 0; i < H; ++i) S.h1[i] = S.z1[i] > 0.0 ? S.z1[i] : 0.0;
    dense(params + o.W2, params + o.b2, S.h1.data(), H, H, S.z2.data());
    for (int i = 0; i < H; ++i) S.h2[i] = S.z2[i] > 0.0 ? S.z2[i] : 0.0;
    dense(params + o.W3, params + o.b3, S.h2.data(), H, H, S.z3.data());
    for (int i = 0; i < H; ++i) S.h3[i] = S.z3[i] > 0.0 ? S.z3[i] : 0.0;
    double a = params[o.b4];
    for (int i = 0; i < H; ++i) a += params[o.w4 + i] * S.h3[i];
    S.o = a;
    S.y = act(s->measure, a);
}

void oracle_ndf_forward(const oracle_net_shape* s, const double* params, int64_t B,
                        const double* pr, const double* pq, double* y) {
    Offsets o = offsets(s);
    Sample S;
    for (int64_t b = 0; b < B; ++b) {
        forward_one(s, o, params, pr + 3 * b, pq + 3 * b, S);
        y[b] = S.y;
    }
}

double oracle_ndf_loss_grad(const oracle_net_shape* s, const double* params, int64_t B,
                            const double* pr, const double* pq, const double* target,
                            double* grad) {
    Offsets o = offsets(s);
    const int LF = s->levels * s->feat, H = s->hidden, IN = 2 * LF, F = s->feat;
    if (grad)
        for (int64_t i = 0; i < o.total; ++i) grad[i] = 0.0;
    Sample S;
    std::vector<double> dz1(H), dz2(H), dz3(H), dh(H), dx(IN), dfr(LF), dfq(LF);
    double loss = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        forward_one(s, o, params, pr + 3 * b, pq + 3 * b, S);
        const double e = S.y - target[b];
        loss += std::fabs(e);
        if (!grad) continue;
        // dL/dy of the mean L1 loss (sign, 0 at a tie), then through the output activation
        const double dy = (e > 0.0 ? 1.0 : (e < 0.0 ? -1.0 : 0.0)) / (double)B;
        const double dout = dy * dact(s->measure, S.o);
        grad[o.b4] += dout;
        for (int i = 0; i < H; ++i) {
            grad[o.w4 + i] += dout * S.h3[i];
            dz3[i] = S.z3[i] > 0.0 ? dout * params[o.w4 + i] : 0.0;
        }
        // layer 3: z3 = W3 h2 + b3
        for (int i = 0; i < H; ++i) {
            grad[o.b3 + i] += dz3[i];
            for (int j = 0; j < H; ++j) grad[o.W3 + (int64_t)i * H + j] += dz3[i] * S.h2[j];
        }
        for (int j = 0; j < H; ++j) {
            double a = 0.0;
            for (int i = 0; i < H; ++i) a += params[o.W3 + (int64_t)i * H + j] * dz3[i];
            dz2[j] = S.z2[j] > 0.0 ? a : 0.0;
        }
        // layer 2
        for (int i = 0; i < H; ++i) {
            grad[o.b2 + i] += dz2[i];
            for (int j = 0; j < H; ++j) grad[o.W2 + (int64_t)i * H + j] += dz2[i] * S.h1[j];
        }
        for (int j = 0; j < H; ++j) {
            double a = 0.0;
            for (int i = 0; i < H; ++i) a += params[o.W2 + (int64_t)i * H + j] * dz2[i];
            dz1[j] = S.z1[j] > 0.0 ? a : 0.0;
        }
        // layer 1: z1 = W1 x + b1
        for (int i = 0; i < H; ++i) {
            grad[o.b1 + i] += dz1[i];
            for (int j = 0; j < IN; ++j) grad[o.W1 + (int64_t)i * IN + j] += dz1[i] * S.x[j];
        }
        for (int j = 0; j < IN; ++j) {
            double a = 0.0;
            for (int i = 0; i < H; ++i) a += params[o.W1 + (int64_t)i * IN + j] * dz1[i];
            dx[j] = a;
        }
        // merge: x = [fr * fq ; fr + fq]
        for (int i = 0; i < LF; ++i) {
            dfr[i] = dx[i] * S.fq[i] + dx[LF + i];
            dfq[i] = dx[i] * S.fr[i] + dx[LF + i];
        }
        // encoding: scatter through the trilinear weights of both positions
        const double* pos[2] = {pr + 3 * b, pq + 3 * b};
        const double* dfs[2] = {dfr.data(), dfq.data()};
        for (int side = 0; side < 2; ++side) {
            for (int l = 0; l < s->levels; ++l) {
                int64_t idx[8];
                double wt[8];
                corners(s, l, pos[side], idx, wt);
                for (int c = 0; c < 8; ++c)
                    for (int f = 0; f < F; ++f)
                        grad[o.grid[l] + idx[c] * F + f] += wt[c] * dfs[side][l * F + f];
            }
        }
    }
    return loss / (double)B;
}

double oracle_ndf_loss_grad_abs(const oracle_net_shape* s, const double* params, int64_t B,
                                const double* pr, const double* pq, const double* target,
                                double* grad, double* gabs) {
    // same gradient, one sample at a time, also summing |per-sample gradient|
    Offsets o = offsets(s);
    std::vector<double> one((size_t)o.total);
    for (int64_t i = 0; i < o.total; ++i) grad[i] = gabs[i] = 0.0;
    double loss = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        loss += oracle_ndf_loss_grad(s, params, 1, pr + 3 * b, pq + 3 * b, target + b, one.data());
        for (int64_t i = 0; i < o.total; ++i) {
            grad[i] += one[(size_t)i] / (double)B;
            gabs[i] += std::fabs(one[(size_t)i]) / (double)B;
        }
    }
    return loss / (double)B;
}

void oracle_adam_step(int64_t n, double* params, const double* grad, double* m, double* v,
                      int64_t t, double lr, double beta1, double beta2, double eps) {
    const double c1 = 1.0 - std::pow(beta1, (double)t);
    const double c2 = 1.0 - std::pow(beta2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        const double mh = m[i] / c1;
        const double vh = v[i] / c2;
        params[i] -= lr * mh / (std::sqrt(vh) + eps);
    }
}

}  // extern "C"

// CPU oracle of the paper's NDF architecture (see hash_net_oracle.h).  Test
// infrastructure only; plain loops in FP64, one sample at a time.
#include "hash_net_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;

struct Layout {
    int levels, F, L, c, le, ld, n_enc, din, merge, dlat, ddec;
    std::vector<int64_t> res, entries;
    int64_t enc_size = 0, total = 0;
    std::vector<int64_t> table_off;      // within an encoder
    std::vector<int64_t> enc_w, enc_b;   // within an encoder
    std::vector<int64_t> dec_w, dec_b;   // absolute
    bool ok = false;
    explicit Layout(const oracle_hash_shape& s) {
        if (s.levels < 1 || s.base_res < 2 || s.log2_table < 1 || s.log2_table > 30 || s.feat < 1 ||
            s.n_freq < 0 || s.width < 1 || s.enc_layers < 0 || s.dec_layers < 1 ||
            (s.n_enc != 1 && s.n_enc != 2) || s.act < 0 || s.act > 2 || s.merge < 0 || s.merge > 3)
            return;
        levels = s.levels;
        F = s.feat;
        L = s.n_freq;
        c = s.width;
        le = s.enc_layers;
        ld = s.dec_layers;
        n_enc = s.n_enc;
        merge = s.merge;
        din = 3 + 6 * L + levels * F;
        dlat = le > 0 ? c : din;
        ddec = merge == 3 ? 2 * dlat : dlat;
        int64_t o = 0;
        for (int l = 0; l < levels; ++l) {
            const int64_t R = (int64_t)s.base_res << l;
            res.push_back(R);
            const int64_t dense = R * R * R;
            const int64_t cap = int64_t(1) << s.log2_table;
            entries.push_back(std::min(dense, cap));
            table_off.push_back(o);
            o += entries.back() * F;
        }
        for (int k = 0; k < le; ++k) {
            const int64_t in = k == 0 ? din : c;
            enc_w.push_back(o);
            o += in * c;
            enc_b.push_back(o);
            o += c;
        }
        enc_size = o;
        o = enc_size * n_enc;
        for (int k = 0; k < ld; ++k) {
            const int64_t out = k == ld - 1 ? 1 : c, in = k == 0 ? ddec : c;
            dec_w.push_back(o);
            o += out * in;
            dec_b.push_back(o);
            o += out;
        }
        total = o;
        ok = true;
    }
};

// x rounded to BF16 (8 significant bits) by round-to-nearest-even, after a
// round-to-nearest conversion to FP32 (the values a BF16 tensor-core operand is
// made from are FP32)
double bf16_round(double x) {
    const float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (double)f;  // Inf (also from overflow) / NaN
    const uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7FFFu + lsb) & 0xFFFF0000u;
    float r;
    std::memcpy(&r, &u, 4);
    return (double)r;
}

inline double opnd(bool rb, double x) { return rb ? bf16_round(x) : x; }

double act(int a, double x) {
    if (a == 0) return x > 0.0 ? x : 0.0;
    const double s = std::sin(x);
    return (a == 1 ? x : 0.5 * x) + s * s;
}
double dact(int a, double x) {
    if (a == 0) return x > 0.0 ? 1.0 : 0.0;
    return (a == 1 ? 1.0 : 0.5) + std::sin(2.0 * x);
}

// corner entry index and trilinear weight of corner q (bit 0: x, 1: y, 2: z)
struct Corners {
    int64_t idx[8];
    double w[8];
};

Corners corners(const double p[3], int64_t R, int64_t E, bool dense) {
    int64_t i0[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        double u = (p[a] + 1.0) * 0.5 * (double)(R - 1);
        u = std::min(std::max(u, 0.0), (double)(R - 1));
        i0[a] = std::min((int64_t)std::floor(u), R - 2);
        t[a] = u - (double)i0[a];
    }
    Corners c;
    for (int q = 0; q < 8; ++q) {
        const int64_t x = i0[0] + (q & 1), y = i0[1] + ((q >> 1) & 1), z = i0[2] + ((q >> 2) & 1);
        if (dense) {
            c.idx[q] = x + R * y + R * R * z;
        } else {
            const uint32_t h = (uint32_t)x * 1u ^ (uint32_t)y * 2654435761u ^ (uint32_t)z * 805459861u;
            c.idx[q] = (int64_t)(h % (uint32_t)E);
        }
        c.w[q] = ((q & 1) ? t[0] : 1.0 - t[0]) * (((q >> 1) & 1) ? t[1] : 1.0 - t[1]) *
                 (((q >> 2) & 1) ? t[2] : 1.0 - t[2]);
    }
    return c;
}

struct EncCache {
    std::vector<double> x0;                 // embedding
    std::vector<std::vector<double>> pre;   // pre-activations per layer
    std::vector<std::vector<double>> post;  // layer outputs (after activation when any)
    std::vector<Corners> cs;                // per level
    std::vector<double> lat;                // the latent (last layer output or x0)
};

// rb: every layer's product takes its operands rounded to BF16 (bf16_round)
void encode(const Layout& Ly, const oracle_hash_shape& s, const double* P, int e, const double p[3],
            EncCache& C, bool rb = false) {
    const double* enc = P + Ly.enc_size * e;
    C.x0.assign(Ly.din, 0.0);
    C.x0[0] = p[0];
    C.x0[1] = p[1];
    C.x0[2] = p[2];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < Ly.L; ++i) {
            const double a = std::ldexp(kPi, i) * p[j];
            C.x0[3 + (j * Ly.L + i) * 2] = std::sin(a);
            C.x0[3 + (j * Ly.L + i) * 2 + 1] = std::cos(a);
        }
    C.cs.clear();
    for (int l = 0; l < Ly.levels; ++l) {
        const int64_t R = Ly.res[l], E = Ly.entries[l];
        const bool dense = R * R * R <= (int64_t(1) << s.log2_table);
        Corners cc = corners(p, R, E, dense);
        C.cs.push_back(cc);
        for (int f = 0; f < Ly.F; ++f) {
            double v = 0.0;
            for (int q = 0; q < 8; ++q) v += cc.w[q] * enc[Ly.table_off[l] + cc.idx[q] * Ly.F + f];
            C.x0[3 + 6 * Ly.L + l * Ly.F + f] = v;
        }
    }
    C.pre.assign(Ly.le, {});
    C.post.assign(Ly.le, {});
    C.lat = C.x0;
    const std::vector<double>* in = &C.x0;
    for (int k = 0; k < Ly.le; ++k) {
        const int64_t nin = k == 0 ? Ly.din : Ly.c;
        const double* W = enc + Ly.enc_w[k];
        const double* b = enc + Ly.enc_b[k];
        C.pre[k].assign(Ly.c, 0.0);
        C.post[k].assign(Ly.c, 0.0);
        for (int o = 0; o < Ly.c; ++o) {
            double a = b[o];
            for (int64_t i = 0; i < nin; ++i) a += opnd(rb, W[o * nin + i]) * opnd(rb, (*in)[i]);
            C.pre[k][o] = a;
            C.post[k][o] = k < Ly.le - 1 ? act(s.act, a) : a;
        }
        in = &C.post[k];
        C.lat = C.post[k];
    }
}

// grad with respect to the encoder's parameters, given dL/d(latent)
void encode_backward(const Layout& Ly, const oracle_hash_shape& s, const double* P, int e,
                     const EncCache& C, std::vector<double> g, double* G) {
    const double* enc = P + Ly.enc_size * e;
    double* genc = G + Ly.enc_size * e;
    for (int k = Ly.le - 1; k >= 0; --k) {
        const int64_t nin = k == 0 ? Ly.din : Ly.c;
        if (k < Ly.le - 1)
            for (int o = 0; o < Ly.c; ++o) g[o] *= dact(s.act, C.pre[k][o]);
        const std::vector<double>& in = k == 0 ? C.x0 : C.post[k - 1];
        std::vector<double> gin(nin, 0.0);
        for (int o = 0; o < Ly.c; ++o) {
            genc[Ly.enc_b[k] + o] += g[o];
            for (int64_t i = 0; i < nin; ++i) {
                genc[Ly.enc_w[k] + o * nin + i] += g[o] * in[i];
                gin[i] += enc[Ly.enc_w[k] + o * nin + i] * g[o];
            }
        }
        g = gin;
    }
    // g is dL/d(embedding); only the hash features carry parameters
    for (int l = 0; l < Ly.levels; ++l)
        for (int f = 0; f < Ly.F; ++f) {
            const double gv = g[3 + 6 * Ly.L + l * Ly.F + f];
            for (int q = 0; q < 8; ++q)
                genc[Ly.table_off[l] + C.cs[l].idx[q] * Ly.F + f] += C.cs[l].w[q] * gv;
        }
}

double out_act(int measure, double x) { return measure == 0 ? std::tanh(x) : std::log1p(std::exp(-std::fabs(x))) + std::max(x, 0.0); }
double dout_act(int measure, double x) {
    if (measure == 0) {
        const double t = std::tanh(x);
        return 1.0 - t * t;
    }
    return 1.0 / (1.0 + std::exp(-x));
}

// decoder forward; keeps pre-activations and inputs for the backward
// rb: the hidden layers' products take BF16-rounded operands (the output layer's do not)
double decode(const Layout& Ly, const oracle_hash_shape& s, const double* P, const std::vector<double>& z,
              std::vector<std::vector<double>>& ins, std::vector<std::vector<double>>& pres,
              bool rb = false) {
    ins.assign(Ly.ld, {});
    pres.assign(Ly.ld, {});
    std::vector<double> h = z;
    for (int k = 0; k < Ly.ld; ++k) {
        const int nout = k == Ly.ld - 1 ? 1 : Ly.c, nin = k == 0 ? Ly.ddec : Ly.c;
        ins[k] = h;
        pres[k].assign(nout, 0.0);
        std::vector<double> nh(nout);
        for (int o = 0; o < nout; ++o) {
            double a = P[Ly.dec_b[k] + o];
            const bool r = rb && k < Ly.ld - 1;
            for (int i = 0; i < nin; ++i) a += opnd(r, P[Ly.dec_w[k] + (int64_t)o * nin + i]) * opnd(r, h[i]);
            pres[k][o] = a;
            nh[o] = k < Ly.ld - 1 ? act(s.act, a) : a;
        }
        h = nh;
    }
    return h[0];
}

std::vector<double> merge_fwd(const Layout& Ly, const std::vector<double>& a, const std::vector<double>& b) {
    std::vector<double> z(Ly.ddec);
    for (int i = 0; i < Ly.dlat; ++i) {
        if (Ly.merge == 0) z[i] = a[i] * b[i];
        else if (Ly.merge == 1) z[i] = a[i] + b[i];
        else if (Ly.merge == 2) z[i] = std::fabs(a[i] - b[i]);
        else {
            z[i] = a[i];
            z[Ly.dlat + i] = b[i];
        }
    }
    return z;
}

void merge_bwd(const Layout& Ly, const std::vector<double>& g, const std::vector<double>& a,
               const std::vector<double>& b, std::vector<double>& ga, std::vector<double>& gb) {
    ga.assign(Ly.dlat, 0.0);
    gb.assign(Ly.dlat, 0.0);
    for (int i = 0; i < Ly.dlat; ++i) {
        if (Ly.merge == 0) {
            ga[i] = g[i] * b[i];
            gb[i] = g[i] * a[i];
        } else if (Ly.merge == 1) {
            ga[i] = gb[i] = g[i];
        } else if (Ly.merge == 2) {
            const double sg = a[i] > b[i] ? 1.0 : (a[i] < b[i] ? -1.0 : 0.0);
            ga[i] = g[i] * sg;
            gb[i] = -g[i] * sg;
        } else {
            ga[i] = g[i];
            gb[i] = g[Ly.dlat + i];
        }
    }
}

}  // namespace

extern "C" {

int64_t oracle_hash_param_count(const oracle_hash_shape* s) {
    if (!s) return -1;
    Layout Ly(*s);
    return Ly.ok ? Ly.total : -1;
}

static int forward_impl(const oracle_hash_shape* s, const double* params, int64_t B, const double* pr,
                        const double* pq, double* out, bool rb) {
    if (!s || !params || !pr || !pq || !out || B < 0) return -1;
    Layout Ly(*s);
    if (!Ly.ok) return -1;
    for (int64_t b = 0; b < B; ++b) {
        EncCache cr, cq;
        encode(Ly, *s, params, 0, pr + 3 * b, cr, rb);
        encode(Ly, *s, params, Ly.n_enc - 1, pq + 3 * b, cq, rb);
        const std::vector<double> z = merge_fwd(Ly, cr.lat, cq.lat);
        std::vector<std::vector<double>> ins, pres;
        out[b] = out_act(s->measure, decode(Ly, *s, params, z, ins, pres, rb));
    }
    return 0;
}

int oracle_hash_forward(const oracle_hash_shape* s, const double* params, int64_t B,
                        const double* pr, const double* pq, double* out) {
    return forward_impl(s, params, B, pr, pq, out, false);
}

int oracle_hash_forward_bf16(const oracle_hash_shape* s, const double* params, int64_t B,
                             const double* pr, const double* pq, double* out) {
    return forward_impl(s, params, B, pr, pq, out, true);
}

double oracle_bf16_round(double x) { return bf16_round(x); }

int oracle_hash_loss_grad(const oracle_hash_shape* s, const double* params, int64_t B,
                          const double* pr, const double* pq, const double* target, double* loss,
                          double* grad) {
    if (!s || !params || !pr || !pq || !target || !loss || !grad || B < 1) return -1;
    Layout Ly(*s);
    if (!Ly.ok) return -1;
    std::memset(grad, 0, sizeof(double) * (size_t)Ly.total);
    double lsum = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        EncCache cr, cq;
        encode(Ly, *s, params, 0, pr + 3 * b, cr);
        encode(Ly, *s, params, Ly.n_enc - 1, pq + 3 * b, cq);
        const std::vector<double> z = merge_fwd(Ly, cr.lat, cq.lat);
        std::vector<std::vector<double>> ins, pres;
        const double raw = decode(Ly, *s, params, z, ins, pres);
        const double y = out_act(s->measure, raw);
        const double d = y - target[b];
        lsum += std::fabs(d);
        const double sg = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
        std::vector<double> g{sg / (double)B * dout_act(s->measure, raw)};
        for (int k = Ly.ld - 1; k >= 0; --k) {
            const int nout = k == Ly.ld - 1 ? 1 : Ly.c, nin = k == 0 ? Ly.ddec : Ly.c;
            if (k < Ly.ld - 1)
                for (int o = 0; o < nout; ++o) g[o] *= dact(s->act, pres[k][o]);
            std::vector<double> gin(nin, 0.0);
            for (int o = 0; o < nout; ++o) {
                grad[Ly.dec_b[k] + o] += g[o];
                for (int i = 0; i < nin; ++i) {
                    grad[Ly.dec_w[k] + (int64_t)o * nin + i] += g[o] * ins[k][i];
                    gin[i] += params[Ly.dec_w[k] + (int64_t)o * nin + i] * g[o];
                }
            }
            g = gin;
        }
        std::vector<double> gr, gq;
        merge_bwd(Ly, g, cr.lat, cq.lat, gr, gq);
        encode_backward(Ly, *s, params, 0, cr, gr, grad);
        encode_backward(Ly, *s, params, Ly.n_enc - 1, cq, gq, grad);
    }
    *loss = lsum / (double)B;
    return 0;
}

}  // extern "C"

// CPU oracle for the dependence-volume hot path.  TEST INFRASTRUCTURE ONLY (see
// ndf_oracle.h).  Plain, slow, obviously correct; no blocking, fusion or
// reordering beyond what the definitions state.
#include "ndf_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

void gather_column(const float* field, int64_t M, int64_t N, int64_t v, float* col) {
    for (int64_t m = 0; m < M; ++m) col[m] = field[m * N + v];
}

// psi(n), n = 1..nmax, by psi(1) = -gamma and psi(n+1) = psi(n) + 1/n.
std::vector<long double> digamma_table(int64_t nmax) {
    std::vector<long double> t(static_cast<size_t>(nmax + 1), 0.0L);
    const long double euler_gamma = 0.577215664901532860606512090082402431L;
    if (nmax >= 1) t[1] = -euler_gamma;
    for (int64_t n = 1; n < nmax; ++n) t[n + 1] = t[n] + 1.0L / static_cast<long double>(n);
    return t;
}

}  // namespace

extern "C" {

int oracle_threads(int nthreads) {
    set_threads(nthreads);
    int n = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
#endif
    return n;
}

// Sec. 3.1, Eq. 1: r = cov(e1, e2) / sqrt(var(e1) var(e2)).  The 1/(M-1) of
// the sample (co)variances cancels, so r = Sxy / sqrt(Sxx Syy) with centred
// sums taken around the FP64 means (two passes).
double oracle_pearson(const float* x, const float* y, int64_t M) {
    double mx = 0.0, my = 0.0;
    for (int64_t m = 0; m < M; ++m) {
        mx += static_cast<double>(x[m]);
        my += static_cast<double>(y[m]);
    }
    mx /= static_cast<double>(M);
    my /= static_cast<double>(M);
    double sxy = 0.0, sxx = 0.0, syy = 0.0;
    for (int64_t m = 0; m < M; ++m) {
        double dx = static_cast<double>(x[m]) - mx;
        double dy = static_cast<double>(y[m]) - my;
        sxy += dx * dy;
        sxx += dx * dx;
        syy += dy * dy;
    }
    if (sxx == 0.0 || syy == 0.0) return 0.0;
    return sxy / std::sqrt(sxx * syy);
}

int oracle_pearson_volume(const float* ref_field, const float* q_field, int64_t M, int64_t N,
                          int64_t ref_idx, const int64_t* verts, int64_t nverts, double* out,
                          int nthreads) {
    if (!ref_field || !q_field || !out || M < 2 || N < 1 || ref_idx < 0 || ref_idx >= N) return -1;
    int64_t count = verts ? nverts : N;
    std::vector<float> x(static_cast<size_t>(M));
    gather_column(ref_field, M, N, ref_idx, x.data());
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel
    {
        std::vector<float> y(static_cast<size_t>(M));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < count; ++i) {
            int64_t v = verts ? verts[i] : i;
            if (v < 0 || v >= N) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            gather_column(q_field, M, N, v, y.data());
            out[i] = oracle_pearson(x.data(), y.data(), M);
        }
    }
    return bad ? -1 : 0;
}

double oracle_digamma_int(int64_t n) {
    if (n < 1) return std::numeric_limits<double>::quiet_NaN();
    return static_cast<double>(digamma_table(n)[static_cast<size_t>(n)]);
}

// KSG algorithm 1 (the estimator cited in Sec. 3.2, used in Sec. 6.2), one pair:
//   d_ij  = max(|x_i - x_j|, |y_i - y_j|), FP32, j != i     (joint max-norm)
//   eps_i = k-th smallest of {d_ij : j != i}                  (a multiset)
//   nx_i  = #{j != i : |x_i - x_j| < eps_i}, ny_i likewise    (strict)
//   I     = psi(k) + psi(M) - (1/M) sum_i [psi(nx_i + 1) + psi(ny_i + 1)]
double oracle_ksg_pair(const float* x, const float* y, int64_t M, int k, float* eps, int32_t* nx,
                       int32_t* ny) {
    if (!x || !y || M < 2 || k < 1 || k >= M) return std::numeric_limits<double>::quiet_NaN();
    std::vector<long double> psi = digamma_table(M + 1);
    std::vector<float> d(static_cast<size_t>(M - 1));
    long double acc = 0.0L;
    for (int64_t i = 0; i < M; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < M; ++j) {
            if (j == i) continue;
            float dx = std::fabs(x[i] - x[j]);
            float dy = std::fabs(y[i] - y[j]);
            d[static_cast<size_t>(c++)] = std::max(dx, dy);
        }
        std::nth_element(d.begin(), d.begin() + (k - 1), d.end());
        float e = d[static_cast<size_t>(k - 1)];
        int32_t cx = 0, cy = 0;
        for (int64_t j = 0; j < M; ++j) {
            if (j == i) continue;
            if (std::fabs(x[i] - x[j]) < e) ++cx;
            if (std::fabs(y[i] - y[j]) < e) ++cy;
        }
        if (eps) eps[i] = e;
        if (nx) nx[i] = cx;
        if (ny) ny[i] = cy;
        acc += psi[static_cast<size_t>(cx + 1)] + psi[static_cast<size_t>(cy + 1)];
    }
    long double mi = psi[static_cast<size_t>(k)] + psi[static_cast<size_t>(M)] -
                     acc / static_cast<long double>(M);
    return static_cast<double>(mi);
}

int oracle_ksg_volume(const float* ref_field, const float* q_field, int64_t M, int64_t N,
                      int64_t ref_idx, int k, const int64_t* verts, int64_t nverts, double* out,
                      int nthreads) {
    if (!ref_field || !q_field || !out || M < 2 || N < 1 || ref_idx < 0 || ref_idx >= N || k < 1 ||
        k >= M)
        return -1;
    int64_t count = verts ? nverts : N;
    std::vector<float> x(static_cast<size_t>(M));
    gather_column(ref_field, M, N, ref_idx, x.data());
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel
    {
        std::vector<float> y(static_cast<size_t>(M));
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < count; ++i) {
            int64_t v = verts ? verts[i] : i;
            if (v < 0 || v >= N) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            gather_column(q_field, M, N, v, y.data());
            out[i] = oracle_ksg_pair(x.data(), y.data(), M, k, nullptr, nullptr, nullptr);
        }
    }
    return bad ? -1 : 0;
}

// oracle_ksg_pair for the reference vertex and each listed query vertex, with
// the per-member eps / nx / ny of every pair (row i of the [nverts][M] outputs
// belongs to verts[i]); the pairs are independent and run in parallel.
int oracle_ksg_pairs(const float* ref_field, const float* q_field, int64_t M, int64_t N,
                     int64_t ref_idx, int k, const int64_t* verts, int64_t nverts, float* eps,
                     int32_t* nx, int32_t* ny, double* mi, int nthreads) {
    if (!ref_field || !q_field || !verts || !eps || !nx || !ny || !mi || M < 2 || N < 1 ||
        ref_idx < 0 || ref_idx >= N || k < 1 || k >= M || nverts < 0)
        return -1;
    std::vector<float> x(static_cast<size_t>(M));
    gather_column(ref_field, M, N, ref_idx, x.data());
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel
    {
        std::vector<float> y(static_cast<size_t>(M));
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < nverts; ++i) {
            int64_t v = verts[i];
            if (v < 0 || v >= N) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            gather_column(q_field, M, N, v, y.data());
            mi[i] = oracle_ksg_pair(x.data(), y.data(), M, k, eps + i * M, nx + i * M, ny + i * M);
        }
    }
    return bad ? -1 : 0;
}

// KSG algorithm 2 (the second estimator of the article cited in Sec. 3.2), one pair:
//   d_ij, eps_i      as in algorithm 1 (k-th smallest joint max-norm distance, j != i)
//   neighbour set    S_i = {j != i : d_ij <= eps_i}: the k nearest; with ties at the
//                    k-th distance every tied member belongs to it (reading)
//   ex_i, ey_i       max over S_i of |x_i - x_j| and of |y_i - y_j| (FP32)
//   nx_i             #{j != i : |x_i - x_j| <= ex_i}, ny_i likewise   (non-strict)
//   I2               psi(k) - 1/k + psi(M) - (1/M) sum_i [psi(nx_i) + psi(ny_i)]
double oracle_ksg2_pair(const float* x, const float* y, int64_t M, int k, float* ex, float* ey,
                        int32_t* nx, int32_t* ny) {
    if (!x || !y || M < 2 || k < 1 || k >= M) return std::numeric_limits<double>::quiet_NaN();
    std::vector<long double> psi = digamma_table(M + 1);
    std::vector<float> d(static_cast<size_t>(M - 1));
    long double acc = 0.0L;
    for (int64_t i = 0; i < M; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < M; ++j) {
            if (j == i) continue;
            d[static_cast<size_t>(c++)] = std::max(std::fabs(x[i] - x[j]), std::fabs(y[i] - y[j]));
        }
        std::nth_element(d.begin(), d.begin() + (k - 1), d.end());
        const float e = d[static_cast<size_t>(k - 1)];
        float wx = 0.0f, wy = 0.0f;
        for (int64_t j = 0; j < M; ++j) {
            if (j == i) continue;
            const float dx = std::fabs(x[i] - x[j]), dy = std::fabs(y[i] - y[j]);
            if (std::max(dx, dy) <= e) {
                wx = std::max(wx, dx);
                wy = std::max(wy, dy);
            }
        }
        int32_t cx = 0, cy = 0;
        for (int64_t j = 0; j < M; ++j) {
            if (j == i) continue;
            if (std::fabs(x[i] - x[j]) <= wx) ++cx;
            if (std::fabs(y[i] - y[j]) <= wy) ++cy;
        }
        if (ex) ex[i] = wx;
        if (ey) ey[i] = wy;
        if (nx) nx[i] = cx;
        if (ny) ny[i] = cy;
        acc += psi[static_cast<size_t>(cx)] + psi[static_cast<size_t>(cy)];
    }
    long double mi = psi[static_cast<size_t>(k)] - 1.0L / static_cast<long double>(k) +
                     psi[static_cast<size_t>(M)] - acc / static_cast<long double>(M);
    return static_cast<double>(mi);
}

int oracle_ksg2_volume(const float* ref_field, const float* q_field, int64_t M, int64_t N,
                       int64_t ref_idx, int k, const int64_t* verts, int64_t nverts, double* out,
                       int nthreads) {
    if (!ref_field || !q_field || !out || M < 2 || N < 1 || ref_idx < 0 || ref_idx >= N || k < 1 ||
        k >= M)
        return -1;
    int64_t count = verts ? nverts : N;
    std::vector<float> x(static_cast<size_t>(M));
    gather_column(ref_field, M, N, ref_idx, x.data());
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel
    {
        std::vector<float> y(static_cast<size_t>(M));
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < count; ++i) {
            int64_t v = verts ? verts[i] : i;
            if (v < 0 || v >= N) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            gather_column(q_field, M, N, v, y.data());
            out[i] = oracle_ksg2_pair(x.data(), y.data(), M, k, nullptr, nullptr, nullptr, nullptr);
        }
    }
    return bad ? -1 : 0;
}

int oracle_interp_column(const float* field, int64_t M, int64_t X, int64_t Y, int64_t Z,
                         const float p[3], float* out) {
    if (!field || !p || !out || M < 1 || X < 1 || Y < 1 || Z < 1) return -1;
    const int64_t n[3] = {X, Y, Z};
    int64_t i0[3], i1[3];
    float w[3];
    for (int a = 0; a < 3; ++a) {
        float u = ((p[a] + 1.0f) * 0.5f) * (float)(n[a] - 1);
        u = std::min(std::max(u, 0.0f), (float)(n[a] - 1));
        int64_t f = (int64_t)std::floor(u);
        i0[a] = n[a] > 1 ? std::min(f, n[a] - 2) : 0;
        w[a] = u - (float)i0[a];
        i1[a] = std::min(i0[a] + 1, n[a] - 1);
    }
    const int64_t N = X * Y * Z;
    auto at = [&](int64_t m, int64_t x, int64_t y, int64_t z) { return field[m * N + (z * Y + y) * X + x]; };
    auto lerp = [](float a, float b, float t) { return a * (1.0f - t) + b * t; };
    for (int64_t m = 0; m < M; ++m) {
        const float c00 = lerp(at(m, i0[0], i0[1], i0[2]), at(m, i1[0], i0[1], i0[2]), w[0]);
        const float c10 = lerp(at(m, i0[0], i1[1], i0[2]), at(m, i1[0], i1[1], i0[2]), w[0]);
        const float c01 = lerp(at(m, i0[0], i0[1], i1[2]), at(m, i1[0], i0[1], i1[2]), w[0]);
        const float c11 = lerp(at(m, i0[0], i1[1], i1[2]), at(m, i1[0], i1[1], i1[2]), w[0]);
        const float c0 = lerp(c00, c10, w[1]);
        const float c1 = lerp(c01, c11, w[1]);
        out[m] = lerp(c0, c1, w[2]);
    }
    return 0;
}

}  // extern "C"

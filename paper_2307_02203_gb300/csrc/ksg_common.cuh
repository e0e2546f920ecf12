// Device helpers shared by the KSG kernels (brute-force and pruned).
#pragma once

#include <cuda_runtime.h>

namespace ndf {

// sorted ascending a[0..K1): insert d, dropping the largest; identity if d >= a[K1-1]
template <int K1>
__device__ __forceinline__ void topk_insert(float (&a)[K1], float d) {
#pragma unroll
    for (int p = K1 - 1; p > 0; --p) a[p] = fmaxf(a[p - 1], fminf(a[p], d));
    a[0] = fminf(a[0], d);
}

// #{p : |fl(a[p] - c)| < e} in the ascending array a[0..n) by two binary
// searches on predicates that are monotone in p.
__device__ __forceinline__ int count_within(const float* a, int n, float c, float e) {
    int lo = 0, len = n;
    while (len > 0) {  // first p with fl(c - a[p]) < e
        int h = len >> 1;
        if (!((c - a[lo + h]) < e)) {
            lo += h + 1;
            len -= h + 1;
        } else {
            len = h;
        }
    }
    int hi = 0;
    len = n;
    while (len > 0) {  // first p with fl(a[p] - c) >= e
        int h = len >> 1;
        if (!((a[hi + h] - c) >= e)) {
            hi += h + 1;
            len -= h + 1;
        } else {
            len = h;
        }
    }
    return hi > lo ? hi - lo : 0;
}

// count_within for two arrays at once: na = #{p : |fl(a[p] - c)| < e} in the
// ascending a[0..n), nb = the same for (b, d).  The four bounds are found by
// interleaved branchless binary searches over powers of two (top = the largest power
// of two <= n): each step moves a bound by `step` while the predicate is still false
// there, so the four dependent load chains overlap.  The predicates are those of
// count_within and monotone in p, so the counts are identical.
__device__ __forceinline__ void count_within_pair(const float* __restrict__ a, const float* __restrict__ b,
                                                  int n, int top, float c, float d, float e, int& na,
                                                  int& nb) {
    int la = 0, ha = 0, lb = 0, hb = 0;
    for (int step = top; step > 0; step >>= 1) {
        const int i1 = la + step, i2 = ha + step, i3 = lb + step, i4 = hb + step;
        if (i1 <= n && !((c - a[i1 - 1]) < e)) la = i1;   // first p with fl(c - a[p]) < e
        if (i2 <= n && !((a[i2 - 1] - c) >= e)) ha = i2;  // first p with fl(a[p] - c) >= e
        if (i3 <= n && !((d - b[i3 - 1]) < e)) lb = i3;
        if (i4 <= n && !((b[i4 - 1] - d) >= e)) hb = i4;
    }
    na = ha > la ? ha - la : 0;
    nb = hb > lb ? hb - lb : 0;
}

// The non-strict counts of KSG algorithm 2 for two arrays at once, by the same
// interleaved searches: na = #{p : |fl(a[p] - c)| <= ea}, nb = #{p : |fl(b[p] - d)| <= eb}
// (the predicates of count_le).
__device__ __forceinline__ void count_le_pair(const float* __restrict__ a, const float* __restrict__ b, int n,
                                              int top, float c, float ea, float d, float eb, int& na,
                                              int& nb) {
    int la = 0, ha = 0, lb = 0, hb = 0;
    for (int step = top; step > 0; step >>= 1) {
        const int i1 = la + step, i2 = ha + step, i3 = lb + step, i4 = hb + step;
        if (i1 <= n && !((c - a[i1 - 1]) <= ea)) la = i1;  // first p with fl(c - a[p]) <= ea
        if (i2 <= n && !((a[i2 - 1] - c) > ea)) ha = i2;   // first p with fl(a[p] - c) > ea
        if (i3 <= n && !((d - b[i3 - 1]) <= eb)) lb = i3;
        if (i4 <= n && !((b[i4 - 1] - d) > eb)) hb = i4;
    }
    na = ha > la ? ha - la : 0;
    nb = hb > lb ? hb - lb : 0;
}

// the largest power of two <= n (n >= 1)
__device__ __forceinline__ int pow2_floor(int n) { return 1 << (31 - __clz(n)); }

// #{p : |fl(a[p] - c)| <= e} in the ascending sequence at(0..n) (non-strict, as
// KSG algorithm 2 counts), by two binary searches on monotone predicates.
template <class Get>
__device__ __forceinline__ int count_le(Get at, int n, float c, float e) {
    int lo = 0, len = n;
    while (len > 0) {  // first p with fl(c - a[p]) <= e
        const int h = len >> 1;
        if (!((c - at(lo + h)) <= e)) { lo += h + 1; len -= h + 1; }
        else len = h;
    }
    int hi = 0;
    len = n;
    while (len > 0) {  // first p with fl(a[p] - c) > e
        const int h = len >> 1;
        if (!((at(hi + h) - c) > e)) { hi += h + 1; len -= h + 1; }
        else len = h;
    }
    return hi > lo ? hi - lo : 0;
}

// KSG algorithm 2: the largest |dx| and |dy| over the members j != s whose joint
// max-norm distance to the x-sorted point s is <= e (they lie in the x-window
// |dx| <= e around position s, scanned outward).  pt(j) returns the x-sorted point.
template <class Get>
__device__ __forceinline__ void alg2_extents(Get pt, int M, int s, float2 ps, float e, float& ex,
                                             float& ey) {
    ex = 0.0f;
    ey = 0.0f;
    for (int j = s + 1; j < M; ++j) {
        const float2 c = pt(j);
        const float dx = c.x - ps.x;
        if (dx > e) break;
        const float dy = fabsf(ps.y - c.y);
        if (fmaxf(dx, dy) <= e) {
            ex = fmaxf(ex, dx);
            ey = fmaxf(ey, dy);
        }
    }
    for (int j = s - 1; j >= 0; --j) {
        const float2 c = pt(j);
        const float dx = ps.x - c.x;
        if (dx > e) break;
        const float dy = fabsf(ps.y - c.y);
        if (fmaxf(dx, dy) <= e) {
            ex = fmaxf(ex, dx);
            ey = fmaxf(ey, dy);
        }
    }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        int nw = (blockDim.x + 31) >> 5;
        t = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

}  // namespace ndf

"""The per-vertex statistics scheme of the column-sort kernel (Eq. 1's mean and
1/sqrt(S)), restated in float32 numpy and held against FP64: FP32 sums over each
lane's consecutive sorted members centred on the column's median member, the 32
lanes' sums added by an xor butterfly of Knuth two-sums (double-float), then
mu = c + s1 / M and S = s2 - s1^2 / M in FP64.  The GPU tests check the kernel's
own mu, 1/sqrt(S) and Pearson volumes against the FP64 oracle; this pins the
scheme's accuracy on columns far harder than the benchmark's (large offsets,
tiny spreads, skew)."""
import numpy as np

F32 = np.float32


def two_sum(a, b):
    s = F32(a + b)
    bb = F32(s - a)
    return s, F32(F32(a - F32(s - bb)) + F32(b - bb))


def warp_sum_df(x):
    hi = np.asarray(x, dtype=np.float32).copy()
    lo = np.zeros(32, dtype=np.float32)
    for o in (16, 8, 4, 2, 1):
        h2, l2 = hi[np.arange(32) ^ o].copy(), lo[np.arange(32) ^ o].copy()
        for i in range(32):
            s, e = two_sum(hi[i], h2[i])
            hi[i], lo[i] = two_sum(s, F32(e + F32(lo[i] + l2[i])))
    assert (hi == hi[0]).all() and (lo == lo[0]).all()  # every lane ends with the same pair
    return float(hi[0]) + float(lo[0])


def scheme(col):
    M = len(col)
    R = 1
    while 32 * R < M:
        R *= 2
    srt = np.sort(col).astype(np.float32)
    c = srt[M >> 1]
    c1 = np.zeros(32, dtype=np.float32)
    c2 = np.zeros(32, dtype=np.float32)
    for lane in range(32):
        a, b = F32(0), F32(0)
        for r in range(R):
            e = lane * R + r
            if e < M:
                d = F32(srt[e] - c)
                a = F32(a + d)
                b = F32(float(d) * float(d) + float(b))  # fmaf: one rounding
        c1[lane], c2[lane] = a, b
    s1, s2 = warp_sum_df(c1), warp_sum_df(c2)
    return float(c) + s1 / M, 1.0 / np.sqrt(s2 - s1 * s1 / M)


def test_two_sum_is_exact():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a, b = (F32(v) for v in rng.normal(size=2) * 10.0 ** rng.integers(-20, 20, size=2))
        s, e = two_sum(a, b)
        assert float(s) + float(e) == float(a) + float(b)  # float32 sums are exact in FP64


def test_scheme_against_fp64():
    rng = np.random.default_rng(11)
    cases = [(1000, 0.0, 1.0), (1000, 1000.0, 1.0), (37, -3e4, 50.0), (513, 1e-3, 1e-3),
             (1024, 5.0, 1e-3), (64, 0.0, 50.0)]
    for M, off, sd in cases:
        x = (rng.normal(size=M) * sd + off).astype(np.float32)
        for col in (x, (rng.exponential(size=M) * 3.0).astype(np.float32)):
            mu, inv = scheme(col)
            y = col.astype(np.float64)
            mu64 = y.mean()
            S = ((y - mu64) ** 2).sum()
            assert abs(mu - mu64) <= 1e-6 * np.sqrt(S / M)
            assert abs(inv * np.sqrt(S) - 1.0) <= 1e-6

"""The FP32 orientation filter's error bound, checked on the CPU.

The filter computes d = dx1*dy1 - dy2*dx2 from exact int32 differences as
t1 = fl(fl(dx1) * fl(dy1)), t2 = fl(fl(dy2) * fl(dx2)), d_f = fl(t1 - t2) with
round-to-nearest and no fused multiply-add, and trusts sign(d_f) only when
|d_f| > E = 2^-21 * (|t1| + |t2|).  Forward error analysis (4 conversions,
2 products and 1 difference, each with relative error <= u = 2^-24) gives
|d_f - d| <= (gamma_3 + u (1 + gamma_3)) (|t1| + |t2|) < 4.01 u (|t1| + |t2|),
so E = 8u (|t1| + |t2|) leaves a factor-2 margin, also covering the rounding
in computing E.  numpy float32 arithmetic is IEEE binary32 with
round-to-nearest, the same as the kernel's __fmul_rn / __fsub_rn / __fadd_rn.
"""
import numpy as np

B = 1 << 30


def filt(dx1, dy1, dy2, dx2):
    f = np.float32
    t1 = dx1.astype(f) * dy1.astype(f)
    t2 = dy2.astype(f) * dx2.astype(f)
    df = t1 - t2
    E = f(2.0 ** -21) * (np.abs(t1) + np.abs(t2))
    return df, np.abs(df) > E


def exact(dx1, dy1, dy2, dx2):
    return dx1.astype(np.int64) * dy1 - dy2.astype(np.int64) * dx2


def triples(rng, n, near):
    a = rng.integers(0, B + 1, (n, 2))
    b = rng.integers(0, B + 1, (n, 2))
    if near:
        # p close to the line ab: a + t (b - a), rounded, nudged by a few units
        t = rng.random(n)
        p = np.rint(a + t[:, None] * (b - a)).astype(np.int64) + rng.integers(-2, 3, (n, 2))
        p = np.clip(p, 0, B - 1)
    else:
        p = rng.integers(0, B, (n, 2))
    return (b[:, 0] - a[:, 0], p[:, 1] - a[:, 1], b[:, 1] - a[:, 1], p[:, 0] - a[:, 0])


def test_filter_never_missigns_random():
    rng = np.random.default_rng(1)
    for _ in range(20):
        dx1, dy1, dy2, dx2 = triples(rng, 200_000, near=False)
        df, ok = filt(dx1, dy1, dy2, dx2)
        d = exact(dx1, dy1, dy2, dx2)
        assert np.array_equal(np.sign(df[ok]).astype(np.int64), np.sign(d[ok]))
        assert ok.mean() > 0.999  # random triples almost never escalate


def test_filter_never_missigns_near_collinear():
    rng = np.random.default_rng(2)
    esc = 0
    n = 0
    for _ in range(20):
        dx1, dy1, dy2, dx2 = triples(rng, 200_000, near=True)
        df, ok = filt(dx1, dy1, dy2, dx2)
        d = exact(dx1, dy1, dy2, dx2)
        assert np.array_equal(np.sign(df[ok]).astype(np.int64), np.sign(d[ok]))
        assert not ok[d == 0].any()  # an exact zero is always escalated
        esc += int((~ok).sum())
        n += ok.size
    assert esc > 0  # the adversarial set does exercise the int64 fallback


def test_filter_extremes():
    # largest magnitudes and sign patterns
    v = np.array([B, -B, B - 1, -(B - 1), 1, -1, 0], dtype=np.int64)
    g = np.stack(np.meshgrid(v, v, v, v, indexing="ij"), -1).reshape(-1, 4)
    df, ok = filt(g[:, 0], g[:, 1], g[:, 2], g[:, 3])
    d = exact(g[:, 0], g[:, 1], g[:, 2], g[:, 3])
    assert np.array_equal(np.sign(df[ok]).astype(np.int64), np.sign(d[ok]))


def test_bound_is_needed():
    """A filter with a much smaller constant does mis-sign: the margin is not vacuous."""
    rng = np.random.default_rng(3)
    dx1, dy1, dy2, dx2 = triples(rng, 400_000, near=True)
    f = np.float32
    t1 = dx1.astype(f) * dy1.astype(f)
    t2 = dy2.astype(f) * dx2.astype(f)
    df = t1 - t2
    ok = np.abs(df) > f(2.0 ** -30) * (np.abs(t1) + np.abs(t2))
    d = exact(dx1, dy1, dy2, dx2)
    assert not np.array_equal(np.sign(df[ok]).astype(np.int64), np.sign(d[ok]))

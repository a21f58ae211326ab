"""CPU models of the FP32-pair arithmetic the CUDA kernels use (no GPU needed).

The kernels split FP64 values into unevaluated FP32 pairs on 32-bit words, form products and
sums error-free (TwoProduct via FMA, Knuth's TwoSum) and round each result once to FP64.
These tests rebuild the same sequences with NumPy float32 operations (each rounded to
nearest, as the _rn intrinsics) and check the error bounds the GPU parity tests rely on
against exact rational arithmetic: the split within 2^-48, the Jacobian apply within 2^-44
of the size of its terms.  They pin the algorithms, not the GPU; the parity tests check the
kernels themselves against the oracle.
"""
from fractions import Fraction

import numpy as np

f32 = np.float32


def _words(x):
    u = np.asarray(x, np.float64).view(np.uint64)
    return (u >> np.uint64(32)).astype(np.uint32), (u & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def d2f_round(x):
    """High half: round the FP64 magnitude at mantissa bit 29, rebias to FP32 (normal range)."""
    hi, lo = _words(x)
    lo2 = (lo + np.uint32(1 << 28)).astype(np.uint32)
    hi2 = (hi + (lo2 < lo).astype(np.uint32)).astype(np.uint32)
    ef = ((hi2 >> np.uint32(20)) & np.uint32(0x7FF)).astype(np.int64) - 896
    m = ((hi2 & np.uint32(0xFFFFF)) << np.uint32(3)) | (lo2 >> np.uint32(29))
    sign = hi2 & np.uint32(0x80000000)
    bits = np.where(ef <= 0, sign, sign | (np.clip(ef, 0, 255).astype(np.uint32) << np.uint32(23)) | m)
    return bits.astype(np.uint32).view(np.float32)


def u29_to_float(a):
    """a < 2^29 as a float: two exact halves joined by one rounding (the kernel's FMA)."""
    a = np.asarray(a, np.uint32)
    hi = ((np.uint32(0x4B000000) | (a >> np.uint32(14))).view(np.float32) - f32(8388608.0))
    lo = ((np.uint32(0x4B000000) | (a & np.uint32(0x3FFF))).view(np.float32) - f32(8388608.0))
    return (hi.astype(np.float64) * 16384.0 + lo.astype(np.float64)).astype(np.float32)


def d2f_low(x):
    """Low half: x - hi as a signed count of ulps of x from the low words, scaled."""
    hi, lo = _words(x)
    ex = ((hi >> np.uint32(20)) & np.uint32(0x7FF)).astype(np.int64)
    lr = (lo + np.uint32(1 << 28)).astype(np.uint32) & np.uint32(0xE0000000)
    dl = (lo - lr).astype(np.uint32).view(np.int32).astype(np.int64)
    mag = u29_to_float(np.abs(dl).astype(np.uint32))
    scale = np.ldexp(np.float32(1), np.clip(ex - 1075, -149, 127).astype(np.int32)).astype(np.float32)
    val = (mag * scale).astype(np.float32)
    neg = ((hi >> np.uint32(31)) == 1) ^ (dl < 0)
    val = np.where(neg, -val, val).astype(np.float32)
    return np.where((ex < 949) | (ex > 1202), f32(0), val).astype(np.float32)


def test_u29_to_float_is_correctly_rounded():
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.integers(0, 1 << 29, 200000), [0, 1, (1 << 24) + 1, (1 << 28),
                                                            (1 << 29) - 1]]).astype(np.uint32)
    assert (u29_to_float(a) == a.astype(np.float32)).all()


def test_split_on_words():
    rng = np.random.default_rng(2)
    xs = rng.standard_normal(200000) * 10.0 ** rng.uniform(-25, 8, 200000)
    xs = np.concatenate([xs, [0.0, -0.0, 1.0, -1.0, 0.1, 1.9999999999999998, 2.0 ** -74,
                              2.0 ** -70, -3.0000001]])
    h, l = d2f_round(xs), d2f_low(xs)
    normal = (np.abs(xs) >= 2.0 ** -70) & (np.abs(xs) < 2.0 ** 120)
    assert (h[normal] == xs[normal].astype(np.float32)).all()      # no exact ties drawn
    err = np.abs(h.astype(np.float64) + l.astype(np.float64) - xs)
    assert (err[normal] <= 2.0 ** -48 * np.abs(xs[normal])).all()
    tiny = np.abs(xs) < 2.0 ** -74
    assert (l[tiny] == 0).all() and (err[tiny] <= 2.0 ** -98).all()


def two_sum(a, b):
    s = f32(a + b)
    bv = f32(s - a)
    av = f32(s - bv)
    return s, f32(f32(a - av) + f32(b - bv))


def two_prod(a, b):
    p = f32(a * b)
    return p, f32(np.float64(a) * np.float64(b) - np.float64(p))    # fma(a, b, -p), exact


def fma32(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def low_part(x):
    return f32(x - np.float64(f32(x)))


def apply_pair_model(a, bb, tl, tr, dd, dt, gt):
    """Top row of the kernel's pair apply: dt a - gt (tl + tr) + D (a - bb), rounded once."""
    dh = f32(dd)
    dl = low_part(dd)
    d, ed = two_sum(a, -bb)
    p3, e3 = two_prod(dh, d)
    t3 = fma32(dl, d, fma32(dh, ed, e3))
    st, es = two_sum(tl, tr)
    p1, e1 = two_prod(f32(dt), a)
    p2, e2 = two_prod(f32(gt), st)
    u, eu = two_sum(p1, -p2)
    v, ev = two_sum(u, p3)
    lt = f32(f32(fma32(low_part(dt), a, e1) - fma32(low_part(gt), st, fma32(f32(gt), es, e2)))
             + f32(t3 + f32(eu + ev)))
    return np.float64(v) + np.float64(lt)


def test_pair_apply_within_bound_of_term_sizes():
    """Against exact rationals: within 2^-44 of |dt a| + gt (|tl| + |tr|) + D (|a| + |bb|),
    also for wire constants that are not FP32 numbers and for smooth (cancelling) inputs."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for trial in range(3000):
        a, bb, tl, tr = (f32(v) for v in rng.standard_normal(4) * 10.0 ** rng.uniform(-3, 0, 4))
        if trial % 2:
            tl = f32(a * (1 + 1e-4 * rng.standard_normal()))
            tr = f32(a * (1 + 1e-4 * rng.standard_normal()))
        dd = 10 ** rng.uniform(-6, -4)
        if trial % 3 == 0:
            dd = float(f32(dd))                    # an FP32 conductance, as after step 1
        dt = [2.0, 1.0 + 1e-3 * rng.uniform(), 1.7, 1.3 + 1.0 / 3.0][trial % 4]
        gt = [1.0, 0.7, 1.0 / 3.0][trial % 3]
        w = apply_pair_model(a, bb, tl, tr, dd, dt, gt)
        F = Fraction
        exact = (F(dt) * F(float(a)) - F(gt) * (F(float(tl)) + F(float(tr)))
                 + F(dd) * (F(float(a)) - F(float(bb))))
        size = abs(dt * a) + gt * (abs(float(tl)) + abs(float(tr))) + dd * (abs(float(a)) + abs(float(bb)))
        worst = max(worst, abs(float(F(w) - exact)) / size)
    assert worst <= 2.0 ** -44, worst

"""The arithmetic premise of the rank-16 tensor-core pass's parity bar, checked
in numpy (FP64 reference): a value split as hi = bf16(v), lo = bf16(v - hi)
is represented to within 2^-16 |v| (each BF16 rounding keeps 8 significant
bits, an error of at most 2^-8 of the rounded value: |v - hi| <= 2^-8 |v|,
|v - hi - lo| <= 2^-8 |v - hi|), so a product of two split values is within
2 * 2^-16 ~ 3.05e-5 (the bar's factor on cond); and a contraction
of length L formed from the four products hi*hi, hi*lo, lo*hi, lo*lo with FP32
accumulation is within 1e-5 relative of the exact one for the lengths the pass
uses (L = 512 rows per CTA, L = 16 columns per tile)."""
import numpy as np


def bf16_rn(x):
    """Round FP32 values to BF16 (round to nearest, ties to even), as FP32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def split(v):
    v = np.asarray(v, dtype=np.float32)
    hi = bf16_rn(v)
    lo = bf16_rn(v - hi)
    return hi, lo


def test_bf16_rounding_is_nearest():
    g = np.random.default_rng(0)
    x = g.uniform(-4, 4, 100000).astype(np.float32)
    r = bf16_rn(x)
    # the two BF16 neighbours of x bracket it, and r is the nearer one
    err = np.abs(r.astype(np.float64) - x)
    ulp = 2.0 ** (np.floor(np.log2(np.abs(x.astype(np.float64)))) - 7)
    assert np.all(err <= 0.5 * ulp * (1 + 1e-12))
    assert np.all(bf16_rn(r) == r)                      # idempotent


def test_split_represents_value_to_2_pow_minus_16():
    g = np.random.default_rng(1)
    v = (g.uniform(0, 1, 200000) * 10.0 ** g.uniform(-6, 3, 200000)).astype(np.float32)
    hi, lo = split(v)
    rep = hi.astype(np.float64) + lo.astype(np.float64)
    rel = np.abs(rep - v.astype(np.float64)) / v.astype(np.float64)
    assert rel.max() <= 2.0 ** -16
    assert np.median(rel) <= 2.0 ** -18          # typical: both roundings far from their worst case
    assert np.all(np.abs(lo) <= 2.0 ** -8 * np.abs(hi) + 1e-45)
    # the worst case is reached: v just above a power of two, both roundings half an ulp
    w = np.float32(1.0 + 2.0 ** -8 + 2.0 ** -17 + 2.0 ** -23)
    h, l = split(np.array([w]))
    assert abs(float(h[0]) + float(l[0]) - float(w)) / float(w) > 2.0 ** -18


def _four_product_dot(a, b):
    """sum_i (ah + al)(bh + bl) with every product and partial sum in FP32."""
    ah, al = split(a)
    bh, bl = split(b)
    acc = np.float32(0)
    for x, y in ((ah, bh), (ah, bl), (al, bh), (al, bl)):
        for xi, yi in zip(x, y):
            acc = np.float32(acc + np.float32(xi) * np.float32(yi))   # BF16 x BF16 is exact in FP32
    return float(acc)


def test_four_product_contraction_error():
    g = np.random.default_rng(2)
    for L in (16, 512):
        worst = 0.0
        for _ in range(20):
            a = g.uniform(0, 1, L).astype(np.float32)           # nonnegative, as M, X and Y are
            b = g.uniform(0, 1, L).astype(np.float32)
            exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
            worst = max(worst, abs(_four_product_dot(a, b) - exact) / exact)
        assert worst <= 1e-5, (L, worst)

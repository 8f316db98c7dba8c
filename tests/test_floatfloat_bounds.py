"""Error bounds of the float-float operations the flux kernels use in the
RMHD_FLOATFLOAT form (paper_1808_09721_gb300/csrc/ffloat.cuh).

The steps of each operation -- Knuth's TwoSum, Dekker's FastTwoSum, the FMA
TwoProduct, and the sum, product, fused multiply-add and divide built from
them -- are transcribed here in IEEE float32 (numpy; fmaf as the exact
a*b + c rounded once) and checked against exact rational arithmetic on
random operands over 16 decades: the bounds the header states (about 2^-46
for sum, product and fma relative to the operands, 2^-42 for the divide with
a pessimistic model of the approximate FP32 reciprocal). The GPU tests check
the kernels themselves against the FP64 oracle."""
from fractions import Fraction as Fr

import numpy as np

f32 = np.float32


def fadd(a, b):
    return f32(f32(a) + f32(b))


def fmul(a, b):
    return f32(f32(a) * f32(b))


def fmaf(a, b, c):
    """a * b + c rounded once to float32."""
    return f32(float(Fr(float(a)) * Fr(float(b)) + Fr(float(c))))


def two_sum(a, b):
    s = fadd(a, b)
    bb = fadd(s, -a)
    return s, fadd(fadd(a, -fadd(s, -bb)), fadd(b, -bb))


def fast_two_sum(a, b):
    s = fadd(a, b)
    return s, fadd(b, -fadd(s, -a))


def ff_of(x):
    hi = f32(x)
    return hi, f32(x - float(hi))


def val(a):
    return Fr(float(a[0])) + Fr(float(a[1]))


def add(a, b):
    s = two_sum(a[0], b[0])
    return fast_two_sum(s[0], fadd(s[1], fadd(a[1], b[1])))


def product_parts(a, b):
    p = fmul(a[0], b[0])
    e = fmaf(a[0], b[0], -p)
    e = fmaf(a[0], b[1], e)
    return p, fmaf(a[1], b[0], e)


def mul(a, b):
    return fast_two_sum(*product_parts(a, b))


def fma3(a, b, c):
    p, e = product_parts(a, b)
    s = two_sum(p, c[0])
    return fast_two_sum(s[0], fadd(s[1], fadd(e, c[1])))


def div(a, x):
    y = f32(1.0 / float(x[0]))
    y = f32(float(y) * (1 + 2**-22))  # the approximate reciprocal's error, modelled pessimistically
    q1 = fmul(a[0], y)
    p = fmul(x[0], q1)
    pe = fmaf(x[1], q1, fmaf(x[0], q1, -p))
    r = fadd(fadd(fadd(a[0], -p), -pe), a[1])
    return fast_two_sum(q1, fmul(r, y))


def test_floatfloat_error_bounds():
    rng = np.random.default_rng(0)
    worst = dict.fromkeys(("conv", "add", "sub_near", "mul", "fma", "div"), 0.0)
    for _ in range(2000):
        x, y, z = (rng.uniform(-1, 1) * 10.0 ** rng.integers(-8, 8) for _ in range(3))
        a, b, c = ff_of(x), ff_of(y), ff_of(z)
        worst["conv"] = max(worst["conv"], abs(float(val(a) - Fr(x))) / abs(x))
        r = add(a, b)
        worst["add"] = max(worst["add"], abs(float(val(r) - (val(a) + val(b)))) / (abs(x) + abs(y)))
        bn = ff_of(x * (1 + rng.uniform(-1e-6, 1e-6)))
        r = add(a, (-bn[0], -bn[1]))
        worst["sub_near"] = max(worst["sub_near"], abs(float(val(r) - (val(a) - val(bn)))) / abs(x))
        r = mul(a, b)
        ex = val(a) * val(b)
        worst["mul"] = max(worst["mul"], abs(float(val(r) - ex)) / abs(float(ex)))
        r = fma3(a, b, c)
        ex = val(a) * val(b) + val(c)
        worst["fma"] = max(worst["fma"], abs(float(val(r) - ex)) / (abs(float(val(a) * val(b))) + abs(z)))
        xp = ff_of(abs(y) + 1e-3)
        r = div(a, xp)
        ex = val(a) / val(xp)
        worst["div"] = max(worst["div"], abs(float(val(r) - ex)) / abs(float(ex)))
    assert worst["conv"] <= 2.0 ** -48, worst
    for k in ("add", "sub_near", "mul", "fma"):
        assert worst[k] <= 2.0 ** -45, worst
    assert worst["div"] <= 2.0 ** -41, worst

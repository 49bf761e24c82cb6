"""A CPU model of the float-float sums of squares that the statistics kernels keep on the FP32 pipe
(hi + lo pairs: TwoProd residual of each square through an exact product, TwoSum into hi, the
residuals into lo; Fast2Sum renormalisation every `renorm` terms; a second float-float level that
takes the first every `fold` terms; one FP64 conversion at the end).  IEEE binary32 arithmetic is
numpy's float32; the product residual a*a - RN32(a*a) is taken exactly through float64 (a*a of a
float32 is exact in float64).  Checked against the correctly rounded FP64 sum (math.fsum of the
exact squares): the relative error stays below the 1e-12 the GPU parity tests allow, for the
schedules the kernels use and for inputs spanning 2^-60 .. 2^60."""
import math

import numpy as np
import pytest

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bp = f32(s - a)
    e = f32(f32(a - f32(s - bp)) + f32(b - bp))
    return s, e


class FF:
    def __init__(self):
        self.hi = f32(0.0)
        self.lo = f32(0.0)

    def add_sq(self, v):
        v = f32(v)
        pr = f32(v * v)
        pe = f32(np.float64(v) * np.float64(v) - np.float64(pr))  # the exact TwoProd residual
        t, e = two_sum(self.hi, pr)
        self.hi = t
        self.lo = f32(self.lo + f32(e + pe))

    def renorm(self):
        s = f32(self.hi + self.lo)
        self.lo = f32(self.lo - f32(s - self.hi))
        self.hi = s

    def add(self, o):
        t, e = two_sum(self.hi, o.hi)
        self.hi = t
        self.lo = f32(self.lo + f32(e + o.lo))

    def value(self):
        return float(np.float64(self.hi) + np.float64(self.lo))


def ff_sum_of_squares(x, renorm, fold):
    acc, tot = FF(), FF()
    for i, v in enumerate(x, 1):
        acc.add_sq(v)
        if i % renorm == 0:
            acc.renorm()
        if i % fold == 0:
            tot.add(acc)
            tot.renorm()
            acc = FF()
    acc.renorm()
    tot.add(acc)
    tot.renorm()
    return tot.value()


@pytest.mark.parametrize("renorm,fold", [(16, 64), (32, 128), (8, 32)])
@pytest.mark.parametrize("kind", ["gaussian", "wide", "one_big"])
def test_float_float_sum_of_squares_accuracy(renorm, fold, kind):
    rng = np.random.default_rng(1000 * renorm + fold + {"gaussian": 1, "wide": 2, "one_big": 3}[kind])
    n = 6000
    if kind == "gaussian":
        x = rng.standard_normal(n)
    elif kind == "wide":
        x = rng.standard_normal(n) * 2.0 ** rng.integers(-60, 60, n)
    else:
        x = rng.standard_normal(n)
        x[n // 2] = 2.0 ** 20  # one term dwarfing the rest: the others live in lo
    x = x.astype(np.float32)
    exact = math.fsum(float(v) * float(v) for v in x)
    got = ff_sum_of_squares(x, renorm, fold)
    assert abs(got - exact) <= 1e-12 * exact, (got, exact, abs(got - exact) / exact)


def test_plain_fp32_sum_would_not_do():
    # the reason for the pairs: an FP32 running sum of the same squares misses the 1e-12 tolerance
    rng = np.random.default_rng(3)
    x = rng.standard_normal(6000).astype(np.float32)
    exact = math.fsum(float(v) * float(v) for v in x)
    s = f32(0.0)
    for v in x:
        s = f32(s + f32(v * v))
    assert abs(float(s) - exact) > 1e-9 * exact

"""Host checks of the two numeric schemes the accurate passes are built on,
restated in numpy float32 (every operation rounds to float32 exactly as the
device's explicitly rounded intrinsics do):

  * the lazily normalised compensated sum (Sum2 / Dot2 of Ogita, Rump and Oishi,
    SIAM J. Sci. Comput. 26, 2005): over the stretches a pass accumulates between
    renormalisations, hi + lo carries the error bound of a sum in twice the
    working precision, u |s| + gamma_n^2 sum |terms| with u = 2^-24 and
    gamma_n = n u / (1 - n u);
  * the float32 -> float64 conversion by re-encoding the IEEE fields with integer
    operations (exponent rebiased by 1023 - 127, fraction moved up 29 bits).

The CUDA kernels themselves are checked against the oracle by the -m gpu tests."""
from fractions import Fraction

import numpy as np
import pytest

F = np.float32
U = 2.0 ** -24


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    return s, F(F(a - F(s - bb)) + F(b - bb))


def two_prod(a, b):
    p = F(a * b)
    # the exact product of two float32 numbers is a float64; its error term is a float32
    return p, F(float(a) * float(b) - float(p))


class DSum:
    def __init__(self):
        self.hi, self.lo = F(0), F(0)

    def add(self, x):
        s, e = two_sum(self.hi, F(x))
        self.hi, self.lo = s, F(self.lo + e)

    def add_prod(self, u, v):
        p, pe = two_prod(F(u), F(v))
        s, e = two_sum(self.hi, p)
        self.hi, self.lo = s, F(self.lo + F(e + pe))

    def norm(self):
        self.hi, self.lo = two_sum(self.hi, self.lo)

    def value(self):
        return Fraction(float(self.hi)) + Fraction(float(self.lo))


@pytest.mark.parametrize("cancel", [False, True])
def test_compensated_dot_meets_the_twice_working_precision_bound(cancel):
    rng = np.random.default_rng(3)
    for trial in range(200):
        n = int(rng.integers(1, 65))
        u = rng.standard_normal(n).astype(F)
        v = rng.uniform(-1, 1, n).astype(F)
        if cancel:   # a second half that nearly cancels the first
            h = n // 2
            u[h:2 * h] = -u[:h] * F(1 + 1e-6)
            v[h:2 * h] = v[:h]
        acc = DSum()
        for k in range(n):
            acc.add_prod(u[k], v[k])
            if k % 4 == 3:
                acc.norm()   # the passes renormalise once per 4-sample group
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, v))
        absum = float(sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(u, v)))
        g = n * U / (1 - n * U)
        err = abs(float(acc.value() - exact))
        assert err <= U * abs(float(exact)) + g * g * absum + 1e-300, (trial, n, err)


def test_compensated_sum_beats_plain_float32_by_the_precision_squared():
    rng = np.random.default_rng(4)
    x = (rng.standard_normal(48) * 10.0 ** rng.integers(-3, 4, 48)).astype(F)
    exact = sum(Fraction(float(t)) for t in x)
    acc, plain = DSum(), F(0)
    for t in x:
        acc.add(t)
        plain = F(plain + t)
    e_ds = abs(float(acc.value() - exact))
    e_32 = abs(float(Fraction(float(plain)) - exact))
    assert e_ds <= 1e-6 * max(e_32, 1e-30) or e_ds == 0.0


def f64_of_f32(f):
    """The device's integer re-encoding of a float32 as a float64."""
    u = int(np.array(f, dtype=F).view(np.uint32))
    sign, e, m = u & 0x80000000, (u >> 23) & 0xFF, u & 0x7FFFFF
    hi, lo = sign, 0
    if e == 0xFF:
        hi, lo = sign | 0x7FF00000 | (m >> 3), (m << 29) & 0xFFFFFFFF
    elif e != 0:
        hi, lo = sign | ((e + 896) << 20) | (m >> 3), (m << 29) & 0xFFFFFFFF
    return float(np.array((hi << 32) | lo, dtype=np.uint64).view(np.float64))


def test_integer_reencoding_is_the_exact_float64_of_every_normal_float32():
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2 ** 32, 200_000, dtype=np.uint64).astype(np.uint32)
    vals = bits.view(F)
    for f in list(vals[:20000]) + [F(1.0), F(-2.5), F(3.4028235e38), F(1.1754944e-38), F(0.0),
                                   F(-0.0)]:
        got = f64_of_f32(f)
        if np.isnan(f):
            assert np.isnan(got)
        elif f != 0 and abs(float(f)) < 1.1754943508222875e-38:
            assert got == 0.0 and np.signbit(got) == np.signbit(f)   # subnormals flush to signed zero
        else:
            assert got == float(f) and np.signbit(got) == np.signbit(f), (f, got)
    assert f64_of_f32(F(np.inf)) == np.inf and f64_of_f32(F(-np.inf)) == -np.inf

"""The arithmetic that replaces FP64 divisions and comparisons in the kernels, checked on the host by
emulating its steps (IEEE double bit patterns with numpy, the FP32 reciprocal in numpy's float32, the
fused multiply-adds in exact rational arithmetic rounded once): the one-step reciprocal seed within
2^-45 relative, the two-step reciprocal and the corrected quotient within an ulp of the correctly
rounded results, and the order keys of doubles ordering like the values (-0 just below +0).  The GPU
test tests/test_gpu_arith.py checks the device code itself against CUDA's operations."""
from fractions import Fraction

import numpy as np


def _bits(x):
    """The IEEE pattern of a double as an unsigned integer."""
    return int(np.array(x, dtype=np.float64).view(np.uint64))


def _double(bits):
    return float(np.array(bits, dtype=np.uint64).view(np.float64))


def _fma(a, b, c):
    """a * b + c with one rounding (exact rational arithmetic; finite operands)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def recip_seed(d):
    """The device reciprocal: the 24 leading mantissa bits (rounded) as an FP32 value in [1, 2],
    its FP32 reciprocal, the exponent of 1/|d| from the two exponents, one Newton step."""
    b = _bits(d)
    e = (b >> 52) & 0x7FF
    m23 = (b >> 29) & 0x7FFFFF
    up = np.float32(2.0 ** -23) if (b >> 28) & 1 else np.float32(0.0)
    m = np.float32(1.0 + m23 * 2.0 ** -23) + up
    rb = int(np.array(np.float32(1.0) / m, dtype=np.float32).view(np.uint32))
    ed = (rb >> 23) - 127 + 2046 - e
    if e == 0 or e == 0x7FF or ed <= 0 or ed >= 0x7FF:
        return 1.0 / d
    x = _double((b & (1 << 63)) | (ed << 52) | ((rb & 0x7FFFFF) << 29))
    return _fma(x, _fma(-d, x, 1.0), x)


def recip2(d):
    x = recip_seed(d)
    return _fma(x, _fma(-d, x, 1.0), x)


def quot(n, d):
    x = recip_seed(d)
    q = n * x
    return _fma(x, _fma(-d, q, n), q)


def ord_key(x):
    """The device order key: the signed pattern, magnitude bits flipped for negative values."""
    b = int(np.array(x, dtype=np.float64).view(np.int64))
    return b if b >= 0 else b ^ 0x7FFFFFFFFFFFFFFF


def _ulps(x, exact):
    return abs(Fraction(x) - exact) / Fraction(float(np.spacing(abs(float(exact)))))


def _random(rng, n, emin, emax):
    return [float(s * np.ldexp(m, e)) for s, m, e in zip(rng.choice([-1.0, 1.0], n), rng.uniform(1.0, 2.0, n),
                                                           rng.integers(emin, emax + 1, n))]


def test_reciprocal_seed_and_refinements():
    rng = np.random.default_rng(46)
    ds = _random(rng, 3000, -500, 500) + [1.0, 1.5, 2.0 - 2.0 ** -52, 1.0 + 2.0 ** -52, 3.0, 7.0]
    worst_seed = worst2 = 0.0
    for d in ds:
        exact = 1 / Fraction(d)
        x = recip_seed(d)
        worst_seed = max(worst_seed, float(abs(Fraction(x) / exact - 1)))
        worst2 = max(worst2, float(_ulps(recip2(d), exact)))
    print(f'seed {worst_seed:.3e} relative, two steps {worst2:.3f} ulp')
    assert worst_seed <= 2.0 ** -45
    assert worst2 <= 1.0


def test_corrected_quotient_within_an_ulp():
    rng = np.random.default_rng(52)
    ns = _random(rng, 3000, -300, 300)
    ds = _random(rng, 3000, -300, 300)
    ns[:500] = [d * (1 + 1e-13 * k) for k, d in enumerate(ds[:500])]        # near-equal pairs
    worst = 0.0
    for n, d in zip(ns, ds):
        worst = max(worst, float(_ulps(quot(n, d), Fraction(n) / Fraction(d))))
    print(f'quotient {worst:.3f} ulp')
    assert worst <= 1.0


def test_order_keys_order_like_the_values():
    rng = np.random.default_rng(7)
    xs = _random(rng, 2000, -1074, 1023) + [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308,
                                               -2.2250738585072014e-308, float('inf'), float('-inf'), 1.0, -1.0]
    keyed = sorted(xs, key=ord_key)
    assert all(a <= b for a, b in zip(keyed, keyed[1:]))                     # the values' order
    assert ord_key(-0.0) == ord_key(0.0) - 1                                 # -0 just below +0
    for a, b in zip(xs[:1000], xs[1000:2000]):
        assert (ord_key(a) < ord_key(b)) == (a < b)

"""The fixed-point digit split behind the FP64-class tensor-core GEMM, checked on
the CPU from its definition (no GPU, no library code):

* a df32 value x = hi + lo in a chunk whose largest |hi| is below 2^e is
  x 2^(7-e) = sum_{i<6} s_i 2^(-8i) + r with integers |s_i| <= 128 and a
  remainder |r| <= 2^-41 (half a unit of the sixth digit);
* every digit s_i 2^(-8i) is exact in TF32 and in BF16 (at most 8 significant
  bits), so the BF16 planes hold the same values as the TF32 ones;
* the digit-pair sums of levels 0 and 1 over a 512-wide chunk are exact in FP32
  in any summation order;
* the chunk product from the kept pairs (i + j < 6) is the exact product to
  within 2^-47 K max|a| max|b| on random data, and five digits are not.
"""
from fractions import Fraction

import numpy as np
import pytest

S, KC = 6, 512


def _df32(rng, n, spread=20):
    """n df32 values (hi, lo) with magnitudes over 2^spread, as float64 hi + lo."""
    v = rng.standard_normal(n) * np.exp2(rng.integers(-spread, 1, n))
    hi = v.astype(np.float32).astype(np.float64)
    lo = (v - hi).astype(np.float32).astype(np.float64)
    return hi, lo


def _split(hi, lo):
    """Digits of one chunk: exponent e (max |hi| < 2^e) and the integer digits s[i, k]."""
    m = np.max(np.abs(hi))
    e = int(np.floor(np.log2(m))) + 1
    t = np.ldexp(hi, 7 - e) + np.ldexp(lo, 7 - e)  # exact: at most 48 significant bits
    s = np.empty((S, hi.size))
    for i in range(S):
        s[i] = np.rint(t)
        t = (t - s[i]) * 256.0  # exact in float64
    return e, s, t


def _bf16_exact(x):
    """True where the float32 value of x is a BF16 value (its low 16 bits are zero)."""
    f = x.astype(np.float32)
    assert np.all(f.astype(np.float64) == x)
    return (f.view(np.uint32) & 0xFFFF) == 0


def test_digits_are_small_integers_and_the_remainder_is_tiny():
    rng = np.random.default_rng(0)
    hi, lo = _df32(rng, KC)
    e, s, r = _split(hi, lo)
    assert np.all(np.abs(s) <= 128)
    # after six digits the remainder, scaled back, is at most half a unit of the last digit
    assert np.max(np.abs(r)) <= 128.0 + 1e-9
    x = hi + lo
    back = np.ldexp(sum(s[i] * np.exp2(-8.0 * i) for i in range(S)), e - 7)
    assert np.max(np.abs(back - x)) <= np.ldexp(0.5, e - 7 - 8 * (S - 1))


def test_digits_are_exact_in_bf16():
    rng = np.random.default_rng(1)
    hi, lo = _df32(rng, KC)
    _, s, _ = _split(hi, lo)
    for i in range(S):
        d = s[i] * np.exp2(-8.0 * i)
        assert np.all(_bf16_exact(d)), i


@pytest.mark.parametrize("level", [0, 1])
def test_leading_levels_sum_exactly_in_fp32(level):
    rng = np.random.default_rng(2 + level)
    ha, la = _df32(rng, KC)
    hb, lb = _df32(rng, KC)
    _, sa, _ = _split(ha, la)
    _, sb, _ = _split(hb, lb)
    terms = sum(sa[i] * sb[level - i] for i in range(level + 1)) * np.exp2(-8.0 * level)
    exact = float(np.sum(terms))  # integers times 2^-8, well inside float64
    for order in (np.arange(KC), rng.permutation(KC), np.argsort(-np.abs(terms))):
        acc = np.float32(0.0)
        for t in terms[order]:
            acc = np.float32(acc + np.float32(t))
        assert float(acc) == exact


def _chunk_product(ea, sa, eb, sb, digits):
    """The chunk's dot product from the digit pairs i + j < digits, in exact rational arithmetic."""
    g = Fraction(0)
    for i in range(digits):
        for j in range(digits - i):
            g += Fraction(2) ** (-8 * (i + j)) * sum(Fraction(int(x)) * int(y) for x, y in zip(sa[i], sb[j]))
    return g * Fraction(2) ** (ea + eb - 14)


def test_kept_pairs_give_the_product_to_fp64_class_accuracy():
    """Each term of the kept pairs is within ~2^-42 max|a| max|b| of the exact product (the
    dropped pairs and the remainders weigh 2^-48 of 2^(ea+eb) each); on random signs the chunk
    sum lands near 2^-50 of K max|a| max|b| (seeds 5-10: 2^-50.5 to 2^-53.5). With five digits
    it is 2^-43 to 2^-45, so the bound 2^-47 also tells a dropped level."""
    rng = np.random.default_rng(5)
    ha, la = _df32(rng, KC, spread=4)
    hb, lb = _df32(rng, KC, spread=4)
    ea, sa, _ = _split(ha, la)
    eb, sb, _ = _split(hb, lb)
    a, b = ha + la, hb + lb
    ref = sum(Fraction(x) * Fraction(y) for x, y in zip(a, b))
    scale = float(np.max(np.abs(a)) * np.max(np.abs(b)) * KC)
    err6 = abs(float(_chunk_product(ea, sa, eb, sb, S) - ref))
    err5 = abs(float(_chunk_product(ea, sa, eb, sb, S - 1) - ref))
    assert err6 <= 2.0 ** -47 * scale
    assert err5 > 2.0 ** -47 * scale

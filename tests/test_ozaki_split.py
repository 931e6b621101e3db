"""The arithmetic claims behind the FP64 factor's tensor-core updates (Ozaki
scheme, BF16 slices), checked in exact integer and numpy arithmetic on the
CPU, independent of the kernels (which the GPU tests compare with the oracle):

* balanced base-256 digits of X = round(x 2^(55-e)), |x| < 2^e: D_1..D_6 in
  [-128, 127], |D_0| <= 129, all exactly representable in BF16;
* over a 128-column window the products of each diagonal i + j = d <= 4 sum to
  fewer than 2^24 units of 2^(-8d), so FP32 accumulation in any order is exact;
* the window's dot product rebuilt from the exact diagonals, the FP32-rounded
  diagonals 5-6 and without i + j >= 7 stays within the FP64 dot-product bound
  K u max|a| max|b| (u = 2^-53), also for adversarial (all-maximal) digits.
"""
from fractions import Fraction

import numpy as np
import pytest

P, K = 7, 128


def digits(x, e):
    """Balanced base-256 digits (top first) of round(x 2^(55-e)), exact."""
    X = [int(round(v * 2.0 ** (55 - e))) for v in x]
    out = np.zeros((len(x), P), dtype=np.int64)
    for r, v in enumerate(X):
        for i in range(P - 1, 0, -1):
            d = ((v & 0xFF) ^ 0x80) - 0x80  # signed low byte
            out[r, i] = d
            v = (v - d) >> 8
        out[r, 0] = v
    return out


def bf16_exact(v):
    """v representable with 8 significant bits (BF16) times a power of two."""
    v = abs(int(v))
    while v and v % 2 == 0:
        v //= 2
    return v < 256


def window(rng, kind):
    if kind == "random":
        a, b = rng.standard_normal(K), rng.standard_normal(K)
    elif kind == "spread":  # entries over 12 decades within the window
        a = rng.standard_normal(K) * 10.0 ** rng.uniform(-12, 0, K)
        b = rng.standard_normal(K) * 10.0 ** rng.uniform(-12, 0, K)
    else:  # every entry just below the window's largest power of two
        a = np.full(K, 1.0 - 2.0 ** -53)
        b = np.full(K, -(1.0 - 2.0 ** -53))
    return a, b


def exponent(x):
    return int(np.frexp(np.max(np.abs(x)))[1])  # |x| < 2^e


@pytest.mark.parametrize("kind", ["random", "spread", "maximal"])
def test_digit_ranges_and_reconstruction(kind):
    rng = np.random.default_rng(7)
    for _ in range(20):
        a, _ = window(rng, kind)
        e = exponent(a)
        D = digits(a, e)
        assert D[:, 1:].min() >= -128 and D[:, 1:].max() <= 127
        assert np.abs(D[:, 0]).max() <= 129
        assert all(bf16_exact(v) for v in D.ravel())
        X = sum(D[:, i].astype(object) * 256 ** (P - 1 - i) for i in range(P))
        # the digits rebuild round(x 2^(55-e)) exactly
        want = [int(round(v * 2.0 ** (55 - e))) for v in a]
        assert list(X) == want


def test_exact_diagonals_fit_fp32_worst_case():
    """All-maximal digits of one sign: the largest sums the accumulators can hold."""
    top, low = 129, 128
    for d in range(5):
        n_top = (1 if d == 0 else 2)  # pairs with one index 0
        n_low = (d + 1) - n_top if d > 0 else 0
        bound = K * (n_top * top * (top if d == 0 else low) + n_low * low * low)
        assert bound < 2 ** 24, (d, bound)


@pytest.mark.parametrize("kind", ["random", "spread", "maximal"])
def test_window_product_within_fp64_bound(kind):
    rng = np.random.default_rng(11)
    u = 2.0 ** -53
    for _ in range(20):
        a, b = window(rng, kind)
        ea, eb = exponent(a), exponent(b)
        Da, Db = digits(a, ea), digits(b, eb)
        # exact integer sums per diagonal (what the FP32 accumulators hold for d <= 4)
        N = [sum(int(Da[k, i]) * int(Db[k, d - i]) for k in range(K)
                 for i in range(max(0, d - P + 1), min(d, P - 1) + 1)) for d in range(5)]
        # diagonals 5 and 6 accumulated in FP32 in the tensor core's column order
        tail = np.float32(0.0)
        for k in range(K):
            for d in (5, 6):
                for i in range(d + 1):
                    if d - i < P:
                        tail = np.float32(tail + np.float32(float(Da[k, i] * Db[k, d - i]) * 2.0 ** (-8 * d)))
        # W in units of 2^-40 (tail rounded to that unit), then the scale
        W = sum(N[d] * 2 ** (40 - 8 * d) for d in range(5)) + int(round(float(tail) * 2.0 ** 40))
        got = Fraction(W) * Fraction(2) ** (ea + eb - 54)
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
        bound = Fraction(K) * Fraction(u) * Fraction(float(np.max(np.abs(a)))) * \
            Fraction(float(np.max(np.abs(b))))
        assert abs(got - exact) <= bound, (kind, float(got - exact), float(bound))

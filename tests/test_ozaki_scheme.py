"""The splitting behind the FP64-accurate products on the BF16 tensor cores (Ozaki, Ogita,
Oishi and Rump 2012), restated in exact integer arithmetic and checked on the CPU: the
balanced base-256 digits of a value scaled to 56 fraction bits, the exactness of the FP32
accumulation of their products, and the error of the recombined result against the exact
product.  It pins the scheme as the kernels use it (rows of M equalised by powers of two,
per-row bounds of A' = A diag(2^mu), per-column bounds of M' = diag(2^-mu) M, digit pairs of
order s + t <= 6 kept), not the kernels themselves; those are held to the FP64 parity bound
by the GPU tests."""
import math
from fractions import Fraction

import numpy as np
import pytest

NDIG = 7          # digits per value
MASK64 = (1 << 64) - 1


def bexp(x: float) -> int:
    """e with |x| < 2^e (frexp's exponent); None for zero."""
    return None if x == 0.0 else math.frexp(x)[1]


def digits(x: float, e: int):
    """T = trunc(x 2^(56 - e)) as 7 balanced digits d_0 .. d_6, T = sum d_s 2^(48 - 8 s):
    adding 128 at each of the six low byte positions turns every low byte into d_s + 128."""
    T = math.trunc(Fraction(x) * Fraction(2) ** (56 - e))
    V = (T + 0x808080808080) & MASK64
    d = [0] * NDIG
    for s in range(1, NDIG):
        d[s] = ((V >> (48 - 8 * s)) & 0xFF) - 128
    v = V - (1 << 64) if V >> 63 else V
    d[0] = v >> 48
    return T, d


def test_digits_are_exact_balanced_and_bf16_representable():
    rng = np.random.default_rng(7)
    for _ in range(3000):
        x = float(rng.standard_normal() * 2.0 ** rng.integers(-60, 60))
        e = bexp(x) + int(rng.integers(0, 3))          # any bound at or above |x|
        T, d = digits(x, e)
        assert sum(ds * 2 ** (48 - 8 * s) for s, ds in enumerate(d)) == T
        assert -256 <= d[0] <= 256 and all(-128 <= ds <= 127 for ds in d[1:])
        # at most 8 significant bits: exact in BF16
        assert all(abs(ds) < 2 ** 8 or abs(ds) == 256 for ds in d)
        assert abs(Fraction(x) * Fraction(2) ** (56 - e) - T) < 1


def test_fp32_accumulation_is_exact_for_64_terms():
    """Accumulator g sums the pairs (s, t), s + t = g, over at most 64 terms: the largest
    possible partial sum stays below 2^24, so FP32 adds them exactly."""
    for g in range(NDIG):
        worst = sum((256 if s == 0 else 128) * (256 if g - s == 0 else 128)
                    for s in range(g + 1))
        assert 64 * worst < 2 ** 24, g


def ozaki_product(A, M):
    """Y = A M by the splitting, in exact integers, with the per-accumulator partial sums."""
    R, K = A.shape
    N = M.shape[1]
    mu = [max((bexp(v) for v in M[k] if v != 0.0), default=None) for k in range(K)]
    f = [max((bexp(M[k, n]) - mu[k] for k in range(K) if M[k, n] != 0.0), default=None)
         for n in range(N)]
    Y = np.zeros((R, N))
    peak = 0
    for r in range(R):
        terms = [bexp(A[r, k]) + mu[k] for k in range(K) if A[r, k] != 0.0 and mu[k] is not None]
        if not terms:
            continue
        er = max(terms)
        da = [digits(A[r, k], er - mu[k])[1] if mu[k] is not None else [0] * NDIG for k in range(K)]
        for n in range(N):
            if f[n] is None:
                continue
            dm = [digits(M[k, n], f[n] + mu[k])[1] if mu[k] is not None else [0] * NDIG
                  for k in range(K)]
            D = [0] * NDIG
            for k in range(K):
                for g in range(NDIG):
                    D[g] += sum(da[k][s] * dm[k][g - s] for s in range(g + 1))
                    peak = max(peak, abs(D[g]))
            J = sum(D[g] << (40 - 8 * g) for g in range(NDIG - 1)) + (D[NDIG - 1] >> 8)
            Y[r, n] = float(Fraction(J) * Fraction(2) ** (er + f[n] - 56))
    return Y, peak, mu, f


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_recombined_product_is_within_a_few_units_of_2_minus_56(seed):
    rng = np.random.default_rng(seed)
    R, K, N = 6, 40, 5
    A = rng.standard_normal((R, K)) * 2.0 ** rng.integers(-30, 30, size=(R, K))
    M = rng.standard_normal((K, N)) * 2.0 ** rng.integers(-20, 20, size=(K, N))
    A[0, 3] = 0.0
    M[5, :] = 0.0                              # a zero row of M drops its column of A
    Y, peak, mu, f = ozaki_product(A, M)
    assert peak < 2 ** 24
    for r in range(R):
        er = max(bexp(A[r, k]) + mu[k] for k in range(K) if A[r, k] != 0.0 and mu[k] is not None)
        for n in range(N):
            exact = sum(Fraction(A[r, k]) * Fraction(M[k, n]) for k in range(K))
            scale = Fraction(2) ** (er + f[n])          # max|A'[r, :]| max|M'[:, n]| < scale
            err = abs(Fraction(Y[r, n]) - exact)
            ulp = Fraction(math.ulp(float(exact))) if exact != 0 else Fraction(0)
            assert err <= 8 * K * scale * Fraction(2) ** -56 + ulp / 2, (r, n, float(err / scale))

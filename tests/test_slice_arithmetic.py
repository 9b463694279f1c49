"""The arithmetic facts the tensor-core path rests on, checked on the CPU.

The five-slice scheme cuts a coefficient vector a (|a_n| < 1) and a basis
column T (|T_n| < 1) into slices A_p 2^-8p, T_q 2^-8q with integer A_p, T_q,
|A_0|, |T_0| <= 256 and |A_p|, |T_q| <= 128 for p, q >= 1.  The claims:

1. level k, D'_k = sum_{p+q=k} sum_n (A_p 2^-8p)(T_q 2^-8q), accumulates exactly
   in FP32 in any order for K <= 64 terms (every partial sum is a multiple of
   2^-8k below 2^(24-8k));
2. the cascade m = fl(fl(fl(fl(D'_0 + D'_1) + D'_2) + D'_3) + D'_4) with
   fast two-sums has exact error terms: m + e1 + e2 + e3 + e4 equals
   sum_k D'_k exactly;
3. the five levels hold sum_n a_n T_n to about 2^-40 per term of the scale
   max|a| max|T| to which both operands are normalised.

Emulated with numpy float32 round-to-nearest operations and checked with
exact rational arithmetic; the worst-case magnitudes are included.
"""
from fractions import Fraction

import numpy as np

S = 5


def slices(x):
    """Fixed-point slices of x (|x| < 1) as the device cuts them: integer q_p
    times 2^-8p, from r = 256 x, q = rint(r), r = 256 (r - q)."""
    r = np.asarray(x, dtype=np.float64) * 256.0
    out = []
    for p in range(S):
        q = np.rint(r)
        out.append(q * 2.0 ** (-8 * p))
        r = (r - q) * 256.0
    return out


def f32_sum(vals):
    acc = np.float32(0.0)
    for v in vals:
        acc = np.float32(acc + np.float32(v))
    return acc


def fast_two_sum(a, b):
    s = np.float32(a + b)
    e = np.float32(b - np.float32(s - a))
    return s, e


def levels(A, T, order):
    """D'_k accumulated in FP32 over (p, q, n) in the given order of n."""
    D = []
    for k in range(S):
        terms = []
        for p in range(k + 1):
            q = k - p
            for n in order:
                terms.append(np.float32(A[p][n]) * np.float32(T[q][n]))  # exact products
        D.append((f32_sum(terms), sum(Fraction(float(t)) for t in terms)))
    return D


def test_levels_exact_and_cascade_exact_on_random_columns():
    rng = np.random.default_rng(5)
    for trial in range(40):
        K = 64
        # wide dynamic range and strong cancellation, as in the Chebyshev sums
        a = rng.uniform(-1, 1, K) * np.exp(rng.uniform(-20, 0, K))
        T = rng.uniform(-1, 1, K) * np.exp(rng.uniform(-20, 0, K))
        a /= 1.01 * np.max(np.abs(a))
        T /= 1.01 * np.max(np.abs(T))
        A, B = slices(a), slices(T)
        for p in range(S):  # slice ranges of the scheme
            lim = 256 if p == 0 else 128
            assert np.all(np.abs(A[p] * 2.0 ** (8 * p)) <= lim) and np.all(np.abs(B[p] * 2.0 ** (8 * p)) <= lim)
        order = rng.permutation(K)
        D = levels(A, B, order)
        for k, (d32, exact) in enumerate(D):
            assert Fraction(float(d32)) == exact, (trial, k)
        d = [dd for dd, _ in D]
        m, e1 = fast_two_sum(d[0], d[1])
        m, e2 = fast_two_sum(m, d[2])
        m, e3 = fast_two_sum(m, d[3])
        m, e4 = fast_two_sum(m, d[4])
        W = sum(Fraction(float(x)) for x in d)
        assert Fraction(float(m)) + sum(Fraction(float(x)) for x in (e1, e2, e3, e4)) == W
        # five levels reproduce sum a_n T_n to about 2^-40 per term of the scale
        # max|a| max|T| (< 1 here), the truncated slices and dropped pairs p + q > 4;
        # W carries the factor 256 x 256 of the two slicings
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, T))
        assert abs(float(W / 65536 - exact)) <= K * 2.0 ** -40


def test_worst_case_magnitudes_stay_exact():
    K = 64
    for sign_pattern in range(4):
        rng = np.random.default_rng(sign_pattern)
        sg = rng.choice([-1.0, 1.0], size=(2, S, K)) if sign_pattern else np.ones((2, S, K))
        A = [sg[0, p] * (256.0 if p == 0 else 128.0) * 2.0 ** (-8 * p) for p in range(S)]
        B = [sg[1, p] * (256.0 if p == 0 else 128.0) * 2.0 ** (-8 * p) for p in range(S)]
        D = levels(A, B, range(K))
        for k, (d32, exact) in enumerate(D):
            assert abs(exact) < Fraction(2) ** (24 - 8 * k)
            assert Fraction(float(d32)) == exact
        d = [dd for dd, _ in D]
        m, e1 = fast_two_sum(d[0], d[1])
        m, e2 = fast_two_sum(m, d[2])
        m, e3 = fast_two_sum(m, d[3])
        m, e4 = fast_two_sum(m, d[4])
        W = sum(Fraction(float(x)) for x in d)
        assert Fraction(float(m)) + sum(Fraction(float(x)) for x in (e1, e2, e3, e4)) == W

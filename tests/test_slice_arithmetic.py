"""The arithmetic facts the tensor-core path rests on, checked on the CPU.

The five-slice scheme cuts a coefficient vector a (|a_n| < 1) and a basis
column T (|T_n| < 1) into slices A_p 2^-8p, T_q 2^-8q with integer A_p, T_q,
|A_0|, |T_0| <= 256 and |A_p|, |T_q| <= 128 for p, q >= 1.  The claims:

1. level k, D'_k = sum_{p+q=k} sum_n (A_p 2^-8p)(T_q 2^-8q), accumulates exactly
   in FP32 in any order for K <= 96 terms (every partial sum is a multiple of
   2^-8k below 2^(24-8k));
2. the epilogue's combination m = fl(fl(D'_0 + D'_1) + D'_2) with fast
   two-sums has exact error terms (m + e1 + e2 = D'_0 + D'_1 + D'_2), and
   lo = fl(fl(e1 + e2) + fl(D'_3 + D'_4)) leaves W' = m + lo within 2^-21 of
   the exact sum W = sum_k D'_k;
3. levels 3 and 4 could share one FP32 accumulator (the kernel keeps all five
   levels apart, for both orders <= 64 and <= 96, so this is margin only):
   with one rounding per K = 16 MMA step the merged level stays within 2^-17
   of D'_3 + D'_4, far below the slices' truncation (next item);
4. the five levels hold sum_n a_n T_n to about 2^-40 per term of the scale
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


def combine(d):
    """m, lo of the epilogue from the five levels (FP32 round to nearest)."""
    m, e1 = fast_two_sum(d[0], d[1])
    m, e2 = fast_two_sum(m, d[2])
    lo = np.float32(np.float32(e1 + e2) + np.float32(d[3] + d[4]))
    return m, e1, e2, lo


def merged_low_levels(A, T, K):
    """Levels 3 and 4 in one FP32 accumulator, each K = 16 step's products
    summed exactly and added with one rounding (the MMA's accumulation)."""
    acc = np.float32(0.0)
    for p in range(S):
        for q in range(S - p):
            if p + q < 3:
                continue
            for k0 in range(0, K, 16):
                blk = sum(Fraction(float(A[p][n])) * Fraction(float(T[q][n])) for n in range(k0, min(K, k0 + 16)))
                acc = np.float32(float(Fraction(float(acc)) + blk))
    return acc


def check_column(a, T, rng, K):
    A, B = slices(a), slices(T)
    for p in range(S):  # slice ranges of the scheme
        lim = 256 if p == 0 else 128
        assert np.all(np.abs(A[p] * 2.0 ** (8 * p)) <= lim) and np.all(np.abs(B[p] * 2.0 ** (8 * p)) <= lim)
    D = levels(A, B, rng.permutation(K))
    for k, (d32, exact) in enumerate(D):
        assert Fraction(float(d32)) == exact, k
    d = [dd for dd, _ in D]
    m, e1, e2, lo = combine(d)
    assert Fraction(float(m)) + Fraction(float(e1)) + Fraction(float(e2)) == D[0][1] + D[1][1] + D[2][1]
    W = sum(ex for _, ex in D)
    assert abs(float(Fraction(float(m)) + Fraction(float(lo)) - W)) <= 2.0 ** -21
    d34 = merged_low_levels(A, B, K)
    assert abs(float(Fraction(float(d34)) - D[3][1] - D[4][1])) <= 2.0 ** -17
    return a, T, W


def test_levels_exact_and_combination_on_random_columns():
    rng = np.random.default_rng(5)
    for trial in range(40):
        K = 64 if trial % 2 else 96
        # wide dynamic range and strong cancellation, as in the Chebyshev sums
        a = rng.uniform(-1, 1, K) * np.exp(rng.uniform(-20, 0, K))
        T = rng.uniform(-1, 1, K) * np.exp(rng.uniform(-20, 0, K))
        a /= 1.01 * np.max(np.abs(a))
        T /= 1.01 * np.max(np.abs(T))
        a, T, W = check_column(a, T, rng, K)
        # five levels reproduce sum a_n T_n to about 2^-40 per term of the scale
        # max|a| max|T| (< 1 here), the truncated slices and dropped pairs p + q > 4;
        # W carries the factor 256 x 256 of the two slicings
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, T))
        assert abs(float(W / 65536 - exact)) <= K * 2.0 ** -40


def test_worst_case_magnitudes_stay_exact():
    K = 96
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
        m, e1, e2, lo = combine(d)
        assert Fraction(float(m)) + Fraction(float(e1)) + Fraction(float(e2)) == D[0][1] + D[1][1] + D[2][1]
        W = sum(ex for _, ex in D)
        assert abs(float(Fraction(float(m)) + Fraction(float(lo)) - W)) <= 2.0 ** -21

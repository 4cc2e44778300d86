"""CPU check of the arithmetic behind the tensor-core residual (no GPU): the
digit splitting of float64 values and the grouping of digit products by
weight, emulated with Python integers.

For random block rows L (m x 3m) and panels X (3m x r): every value is scaled
by the power of two above its row's (column's) largest magnitude and cut into
nine base-64 digits from its bits (truncated below 2^-54); products of digit
matrices are grouped by s + t <= 11.  Checked: each group's partial sums are
integers below 2^24 (so float32 accumulation is exact), and the recombined
product differs from the exact one by at most 3m 2^-50 max|row| max|column|."""
import math
from fractions import Fraction

import numpy as np
import pytest

BETA, SLICES, DMAX = 6, 9, 11


def scale_exp(vals):
    mx = max(abs(v) for v in vals)
    return math.frexp(mx)[1] if mx > 0 else -1021


def digits(v, e):
    """sign, nine digits d_s with |v| 2^-e = sum d_s 2^(-6s) + tail, tail < 2^-54."""
    y = Fraction(abs(v)) / Fraction(2) ** e
    assert y < 1
    Y = math.floor(y * 2 ** (BETA * SLICES))
    ds = [(Y >> (BETA * (SLICES - 1 - s))) & 63 for s in range(SLICES)]
    return (-1 if v < 0 else 1), ds


@pytest.mark.parametrize("m,r,seed", [(5, 1, 0), (32, 4, 1), (64, 16, 2), (128, 8, 3)])
def test_digit_products_exact_and_bounded(m, r, seed):
    rng = np.random.default_rng(seed)
    K = 3 * m
    rows = min(m, 6)  # a few rows suffice for the bound; all K terms are used
    L = rng.standard_normal((rows, K)) * np.exp(rng.uniform(-8, 8, size=(rows, K)))
    X = rng.standard_normal((K, r)) * np.exp(rng.uniform(-8, 8, size=(K, r)))
    L[0, 3] = 0.0
    X[2, 0] = 5e-320  # a subnormal
    for i in range(rows):
        e = scale_exp(L[i])
        Ld = [digits(v, e) for v in L[i]]
        for c in range(r):
            f = scale_exp(X[:, c])
            Xd = [digits(v, f) for v in X[:, c]]
            total = Fraction(0)
            for d in range(2, DMAX + 1):
                acc = absacc = 0
                for k in range(K):
                    (sl, dl), (sx, dx) = Ld[k], Xd[k]
                    for s in range(1, SLICES + 1):
                        t = d - s
                        if 1 <= t <= SLICES:
                            term = sl * sx * dl[s - 1] * dx[t - 1]
                            acc += term
                            absacc += abs(term)
                # any summation order: every partial sum is an integer below 2^24
                assert absacc < 2 ** 24
                total += Fraction(acc) * Fraction(2) ** (-BETA * d)
            approx = total * Fraction(2) ** (e + f)
            exact = sum(Fraction(float(L[i, k])) * Fraction(float(X[k, c])) for k in range(K))
            bound = Fraction(3 * m) * Fraction(2) ** -50 * Fraction(float(np.abs(L[i]).max())) * \
                Fraction(float(np.abs(X[:, c]).max()))
            assert abs(approx - exact) <= bound


def test_worst_case_group_sum_below_2_24():
    """The largest possible group: 9 digit pairs of 63 x 63 over K = 3 * 128."""
    assert 9 * 63 * 63 * 3 * 128 < 2 ** 24
    assert 9 * 63 * 63 * 3 * 256 >= 2 ** 24  # why the kernel stops at m = 128

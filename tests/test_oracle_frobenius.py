"""Pins of the oracle's F = ||A||_F^2 (CPU only).

Section 1 draws row i with probability ||a_i||^2/||A||_F^2.  The oracle takes
F as the exact sum of the row weights w_i rounded once to the nearest double
(ties to even), so F does not depend on an order of summation.  It is pinned
against two references that share nothing with it: Python's math.fsum (a
correctly rounded sum of doubles) and the exact rational sum of
fractions.Fraction converted back by float() (also correctly rounded).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _exact_rounded(v):
    return float(sum((Fraction(float(x)) for x in v), Fraction(0)))


def _cases():
    rng = np.random.default_rng(11)
    tiny = np.full(5000, 2.0**-54)
    tiny[0] = 1.0                              # a plain running sum stays at 1
    yield "many terms below half an ulp", tiny
    yield "wide dynamic range", np.exp(40.0 * rng.standard_normal(20000))
    yield "subnormals", np.array([5e-324] * 9 + [2.0**-1022 - 2.0**-1074])
    yield "tie to even, down", np.array([1.0, 2.0**-53])
    yield "tie to even, up", np.array([1.0 + 2.0**-52, 2.0**-53])
    yield "tie broken by a far bit", np.array([1.0, 2.0**-53, 2.0**-1074])
    yield "carry into a new binade", np.array([2.0**53 - 1.0, 0.5, 0.5])
    yield "largest finite", np.array([1.7976931348623157e308, 9.9e291])
    yield "lognormal row weights", np.exp(2.0 * rng.standard_normal(100000))
    yield "zeros", np.zeros(7)
    yield "empty", np.zeros(0)


@pytest.mark.parametrize("name,v", list(_cases()), ids=[c[0] for c in _cases()])
def test_exact_sum_is_the_correctly_rounded_sum(name, v):
    got = oracle.exact_sum(v)
    assert got == _exact_rounded(v)
    assert got == math.fsum(v)
    # the order of the terms does not matter
    assert oracle.exact_sum(v[::-1]) == got
    perm = np.random.default_rng(3).permutation(v.size)
    assert oracle.exact_sum(v[perm]) == got


def test_overflow_is_infinite():
    assert oracle.exact_sum(np.array([1.7976931348623157e308, 1e292])) == math.inf
    assert oracle.exact_sum(np.array([2.0**1023, 2.0**1023])) == math.inf


def test_row_weights_frobenius_is_exact():
    # rows with one entry each, so w_i = val_i^2 exactly for powers of two;
    # a plain running sum and a sum in blocks of 2048 both lose the small rows
    m = 9000
    val = np.full(m, 2.0**-27)
    val[[0, 4097, 8191]] = [1.0, 4.0, 0.5]
    row_ptr = np.arange(m + 1, dtype=np.int64)
    w, F = oracle.row_weights(m, row_ptr, val)
    np.testing.assert_array_equal(w, val * val)
    assert F == math.fsum(w) == _exact_rounded(w)
    naive = 0.0
    for x in w:
        naive += x
    assert naive != F  # the case does separate an exact from a running sum


def test_row_weights_are_squared_norms_in_csr_order():
    rng = np.random.default_rng(4)
    m = 200
    lens = rng.integers(1, 30, size=m)
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    val = rng.standard_normal(int(row_ptr[-1])) * np.exp(rng.standard_normal(int(row_ptr[-1])))
    w, F = oracle.row_weights(m, row_ptr, val)
    for i in range(m):
        s = 0.0
        for k in range(row_ptr[i], row_ptr[i + 1]):
            s += val[k] * val[k]
        assert w[i] == s
    assert F == math.fsum(w)

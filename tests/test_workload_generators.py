"""The Mandelbrot coefficient generator of the benchmark (workloads.mandelbrot_fast,
C with OpenMP) against its definition (workloads.mandelbrot: the direct
convolution of every term in Python), and both against the recurrence itself
at small n: p_n(c) computed by iterating p <- p^2 + c in exact rationals."""
from fractions import Fraction

import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("n", [1, 2, 3, 6, 9, 12])
def test_mandelbrot_fast_matches_definition(n):
    a, b = W.mandelbrot(n), W.mandelbrot_fast(n)
    assert np.array_equal(a.e2[a.re != 0], b.e2[a.re != 0])
    assert np.array_equal(a.re == 0, b.re == 0)
    rel = np.abs(a.re - b.re) / np.where(a.re != 0, np.abs(a.re), 1.0)
    assert rel.max() < 1e-14


@pytest.mark.parametrize("n", [3, 5])
def test_mandelbrot_coefficients_are_the_iterate(n):
    """Small n: the coefficients are exact integers; sum a_k c^k equals the
    iterate p_n(c) at rational c exactly."""
    coef = W.mandelbrot_fast(n)
    ak = [int(round(float(m) * 2.0 ** int(e))) if m != 0 else 0 for m, e in zip(coef.re, coef.e2)]
    for c in (Fraction(1, 3), Fraction(-7, 5), Fraction(2)):
        p = c
        for _ in range(n):
            p = p * p + c
        assert sum(a * c ** k for k, a in enumerate(ak)) == p

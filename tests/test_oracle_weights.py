"""Pins of the oracle's weight generators against values fixed by the paper or
by mathematics (no comparison of the oracle with itself)."""
import math

import numpy as np
import pytest

from oracle import weights as W

ALPHAS = [1.1, 1.5, 1.9]


@pytest.mark.parametrize("alpha", ALPHAS)
def test_riesz_1d_closed_form_vs_integral(alpha):
    # Sec. 2 eq. "single coefficient discrete Riesz": the closed Gamma form
    # must equal the Fourier coefficient integral, evaluated independently by
    # the Bessel subordination integral.
    a = W.riesz_1d(alpha, 40)
    for i in [0, 1, 2, 3, 7, 17, 39]:
        assert abs(a[i] - W.riesz_1d_bessel(alpha, i)) < 1e-12 * max(1.0, abs(a[i])) + 1e-14


@pytest.mark.parametrize("alpha", ALPHAS)
def test_riesz_1d_generating_function(alpha):
    # sum_i a_i e^{i i eta} = (4 sin^2(eta/2))^{alpha/2}: a long truncated sum
    # at eta = pi/2 and pi (the tail decays like i^{-1-alpha}; alternating at pi).
    n = 200000
    a = W.riesz_1d(alpha, n)
    i = np.arange(n)
    for eta, tol in [(np.pi, 1e-9), (np.pi / 2, 2e-5)]:
        s = a[0] + 2.0 * np.sum(a[1:] * np.cos(i[1:] * eta))
        assert abs(s - (4 * math.sin(eta / 2) ** 2) ** (alpha / 2)) < tol


def test_riesz_1d_alpha2_second_difference():
    np.testing.assert_array_equal(W.riesz_1d(2.0, 5), [2.0, -1.0, 0.0, 0.0, 0.0])
    # the generic formula approaches the same limit
    a = W.riesz_1d(1.999999, 5)
    np.testing.assert_allclose(a, [2.0, -1.0, 0.0, 0.0, 0.0], atol=1e-5)


def test_trapezoid_cosine_shortcut_equals_bruteforce_dft():
    # the DCT-I evaluation of the M x M trapezoid sum equals the literal 2D DFT
    for alpha in [1.3, 1.7]:
        A = W.lap2d_trap_single(alpha, 9, 64)
        B = W.lap2d_trap_bruteforce(alpha, 9, 64)
        assert np.abs(A - B).max() < 1e-15


def test_trapezoid_blocked_evaluation_equals_bruteforce_dft():
    # the blocked, threaded evaluation (ragged last block) sums the same
    # trapezoid rule: it must equal the literal 2D DFT as well
    for alpha, N, M, chunk in [(1.3, 9, 64, 5), (1.6, 20, 128, 7), (1.9, 33, 128, 64)]:
        A = W.lap2d_trap_single(alpha, N, M, chunk=chunk, workers=3)
        B = W.lap2d_trap_bruteforce(alpha, N, M)
        assert np.abs(A - B).max() < 1e-15, (alpha, N, M, chunk)


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_lap2d_trapezoid_vs_bessel_integral(alpha):
    # Sec. 2 eq. "center discretization": W1 (trapezoid + Richardson) against
    # the independent one-dimensional integral W2, including the far corner.
    N = 63
    A = W.lap2d_trap(alpha, N)
    for (i, j) in [(0, 0), (1, 0), (0, 1), (1, 1), (5, 3), (20, 7), (N - 1, N - 1)]:
        ref = W.lap2d_bessel(alpha, i, j)
        assert abs(A[i, j] - ref) < 1e-12, (i, j, A[i, j], ref)


def test_lap2d_symmetry_and_alpha2():
    A = W.lap2d_trap(1.6, 31)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-15)
    # alpha = 2: the symbol 4 - 2cos(eta) - 2cos(xi) is a trigonometric
    # polynomial, so the trapezoid is exact: the 5-point stencil.
    A2 = W.lap2d_trap(2.0, 6)
    ref = np.zeros((6, 6))
    ref[0, 0] = 4.0
    ref[1, 0] = ref[0, 1] = -1.0
    assert np.abs(A2 - ref).max() < 1e-14


@pytest.mark.parametrize("alpha", [1.3, 1.5, 1.8])
def test_lap2d_far_field_constant(alpha):
    # For large rho = |(i,j)|, h^-alpha a_ij matches the kernel of the singular
    # integral in Sec. 1 (d = 2): a_ij rho^{2+alpha} -> -2^alpha Gamma(1+alpha/2)
    # / (pi |Gamma(-alpha/2)|).
    A = W.lap2d_trap(alpha, 127)
    C = 2 ** alpha * math.gamma(1 + alpha / 2) / (math.pi * abs(math.gamma(-alpha / 2)))
    for (i, j) in [(30, 40), (50, 0), (36, 36), (100, 20)]:
        rho = math.hypot(i, j)
        assert abs(A[i, j] * rho ** (2 + alpha) + C) < 0.01 * C


def test_lap2d_diagonal_sum_rule():
    # sum over all of Z^2 of a_ij equals the symbol at the origin, 0; the
    # M x M trapezoid coefficients sum to f(0, 0) = 0 exactly (inverse DFT at
    # the origin).  Checked on the full periodic set with the brute-force DFT.
    M = 64
    A = np.fft.fft2((lambda t: ((4 * np.sin(t / 2) ** 2)[:, None]
                                + (4 * np.sin(t / 2) ** 2)[None, :]) ** 0.75)(
        2 * np.pi * np.arange(M) / M)).real / M ** 2
    assert abs(A.sum()) < 1e-13
    # and the truncated N x N block of W1 approaches zero like N^-alpha
    alpha = 1.5
    sums = []
    for N in (32, 64, 128):
        a = W.lap2d_trap(alpha, N)
        full = a[0, 0] + 2 * a[1:, 0].sum() + 2 * a[0, 1:].sum() + 4 * a[1:, 1:].sum()
        sums.append(full)
    assert sums[0] > sums[1] > sums[2] > 0
    assert 2 ** 1.3 < sums[0] / sums[1] < 2 ** 1.7


def test_bessel_integral_large_argument_branch():
    # the Hankel expansion that replaces scipy's ive above z = 1e8 agrees with
    # it just below the switch, for orders up to the largest grid offset
    import scipy.special as sp
    z = 0.99 * W._IVE_SWITCH
    saved = W._IVE_SWITCH
    try:
        W._IVE_SWITCH = 0.0
        for n in (0, 1, 17, 1000, 8190):
            assert abs(W._ive(n, z) - sp.ive(n, z)) <= 1e-14 * sp.ive(n, z), n
    finally:
        W._IVE_SWITCH = saved


@pytest.mark.parametrize("alpha", [1.2, 1.6, 1.9])
def test_bessel_weights_far_field_constant(alpha):
    # far from the origin a_ij -> -C rho^-(2+alpha) with the kernel constant of
    # the fractional Laplacian in two dimensions, C = 2^alpha Gamma(1 + alpha/2)
    # / (pi |Gamma(-alpha/2)|) (Sec. 1); the relative correction is O(rho^-2),
    # so at rho >= 3000 the Bessel-integral weights must match to 1e-5.  This
    # pins the integrator where the integrand peaks at t ~ rho^2 / 4.
    C = 2 ** alpha * math.gamma(1 + alpha / 2) / (math.pi * abs(math.gamma(-alpha / 2)))
    for (i, j) in [(3000, 0), (3000, 4000), (8190, 0), (8190, 8190)]:
        rho = math.hypot(i, j)
        a = W.lap2d_bessel(alpha, i, j)
        assert abs(a * rho ** (2 + alpha) / -C - 1.0) < 1e-5, (i, j, a)

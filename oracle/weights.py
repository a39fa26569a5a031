"""Fractional-difference weights (oracle, FP64, test infrastructure only).

* ``riesz_1d``      -- a_i of the fractional centred difference (Sec. 2, eq.
                       "single coefficient discrete Riesz"): the closed Gamma-
                       function form printed there.
* ``lap2d_trap``    -- a_ij of the 2D discrete fractional Laplacian (Sec. 2, eq.
                       "center discretization"), the Fourier coefficients of
                       (4 sin^2(eta/2) + 4 sin^2(xi/2))^(alpha/2).  The paper
                       gives no algorithm for them (it defers to its reference
                       on the discretisation); we take the trapezoid rule on an
                       M x M grid followed by one Richardson step on the leading
                       M^-(2+alpha) aliasing term (method W1).
* ``lap2d_bessel``  -- the same coefficients from a one-dimensional integral
                       (method W2), an independent cross check used only by the
                       pins: with s = alpha/2,
                       lambda^s = s/Gamma(1-s) * int_0^inf (1 - e^{-t lambda}) t^{-1-s} dt
                       and the Fourier coefficients of e^{-2t(1-cos eta)} being
                       e^{-2t} I_n(2t) (modified Bessel generating function).
* ``riesz_1d_bessel`` -- the 1D analogue of W2, which pins the closed form.

Parity: all four pinned (tests/test_oracle_weights.py).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft
import scipy.integrate
import scipy.special as sp


def riesz_1d(alpha: float, n: int) -> np.ndarray:
    """a_0 .. a_{n-1}: (-1)^i Gamma(alpha+1) / (Gamma(alpha/2-i+1) Gamma(alpha/2+i+1)).

    Sec. 2, eq. "single coefficient discrete Riesz".  Evaluated in log-Gamma
    form with explicit signs so that large i neither overflows nor underflows.
    """
    i = np.arange(n, dtype=np.float64)
    z1 = alpha / 2.0 - i + 1.0
    z2 = alpha / 2.0 + i + 1.0
    lg = sp.gammaln(alpha + 1.0) - sp.gammaln(z1) - sp.gammaln(z2)
    sign = np.where(i % 2 == 0, 1.0, -1.0) * sp.gammasgn(z1) * sp.gammasgn(z2)
    out = sign * np.exp(lg)
    if alpha == 2.0:
        # Gamma(alpha/2 - i + 1) has poles for i >= 2: the weights are exactly
        # the second difference (2, -1, 0, ...).
        out = np.zeros(n)
        out[0] = 2.0
        if n > 1:
            out[1] = -1.0
    return out


def trap_grid_size(N: int) -> int:
    """Trapezoid grid M used by method W1 for an N x N interior grid.

    M = max(1024, 8 * N'), N' the smallest power of two >= N; the Richardson
    partner grid is 2M.  (The paper is silent on how a_ij is evaluated.)
    """
    np2 = 1
    while np2 < N:
        np2 *= 2
    return max(1024, 8 * np2)


def _symbol(alpha: float, M: int, c0: int = 0, c1: int | None = None) -> np.ndarray:
    """Samples of (4 sin^2(eta/2) + 4 sin^2(xi/2))^(alpha/2) on the half grid
    eta_k = 2 pi k / M, xi_l = 2 pi l / M, 0 <= k <= M/2, c0 <= l < c1 (the
    symbol is even in both variables, so the half grid carries the full M x M
    sample set; c0, c1 select a block of its columns, default all)."""
    t = 2.0 * np.pi * np.arange(M // 2 + 1) / M
    s = 4.0 * np.sin(t / 2.0) ** 2
    c1 = M // 2 + 1 if c1 is None else c1
    lam = s[:, None] + s[None, c0:c1]
    return lam ** (alpha / 2.0)


def lap2d_trap_single(alpha: float, N: int, M: int, chunk: int | None = None,
                      workers: int | None = None) -> np.ndarray:
    """A_M(i, j), 0 <= i, j < N: the M x M trapezoid rule for the Fourier
    coefficient integral of Sec. 2, eq. "center discretization":

        A_M(i, j) = M^-2 sum_{k,l=0}^{M-1} f(2 pi k/M, 2 pi l/M) exp(-1j(i eta_k + j xi_l)).

    f is real and even in each variable, so the double sum equals a product of
    two type-I cosine transforms of the half-grid samples (scipy's DCT-I:
    y_i = x_0 + (-1)^i x_{M/2} + 2 sum_{m=1}^{M/2-1} x_m cos(2 pi i m / M),
    which is exactly sum_{k=0}^{M-1} f_k cos(2 pi i k / M) for even f).

    chunk: evaluate each transform over blocks of that many independent
    columns (rows) at a time, so that large M needs O(N M) memory instead of
    O(M^2); workers: threads for the blocks and the transforms.  Neither
    changes what is summed.
    """
    H = M // 2 + 1
    if chunk is None:
        F = _symbol(alpha, M)
        G = scipy.fft.dct(F, type=1, axis=0, workers=workers)[:N, :]
        A = scipy.fft.dct(G, type=1, axis=1, workers=workers)[:, :N]
        return A / float(M) ** 2
    G = np.empty((N, H))

    def col_block(c0):
        c1 = min(H, c0 + chunk)
        G[:, c0:c1] = scipy.fft.dct(_symbol(alpha, M, c0, c1), type=1, axis=0)[:N, :]

    def row_block(r0):
        r1 = min(N, r0 + chunk)
        A[r0:r1, :] = scipy.fft.dct(G[r0:r1, :], type=1, axis=1)[:, :N]

    import concurrent.futures as cf
    nw = max(1, workers or 1)
    with cf.ThreadPoolExecutor(max_workers=nw) as ex:
        list(ex.map(col_block, range(0, H, chunk)))
        A = np.empty((N, N))
        list(ex.map(row_block, range(0, N, chunk)))
    return A / float(M) ** 2


def lap2d_trap(alpha: float, N: int, M: int | None = None, chunk: int | None = None,
               workers: int | None = None) -> np.ndarray:
    """a_ij, 0 <= i, j < N, by method W1 (trapezoid on M and 2M, one Richardson
    step on the M^-(2+alpha) term).  a_ij = a_ji = a_{-i,j}.  chunk / workers:
    see lap2d_trap_single (memory and threads only)."""
    if M is None:
        M = trap_grid_size(N)
    A1 = lap2d_trap_single(alpha, N, M, chunk, workers)
    A2 = lap2d_trap_single(alpha, N, 2 * M, chunk, workers)
    q = 2.0 ** (2.0 + alpha)
    return (q * A2 - A1) / (q - 1.0)


def lap2d_trap_bruteforce(alpha: float, N: int, M: int) -> np.ndarray:
    """The M x M trapezoid sum written literally with the full complex 2D DFT
    (used only to pin the cosine-transform shortcut at small M)."""
    t = 2.0 * np.pi * np.arange(M) / M
    s = 4.0 * np.sin(t / 2.0) ** 2
    F = (s[:, None] + s[None, :]) ** (alpha / 2.0)
    A = np.fft.fft2(F) / float(M) ** 2
    return A.real[:N, :N]


_IVE_SWITCH = 1e8


def _ive(n: int, z: float) -> float:
    """Exponentially scaled modified Bessel function I_n(z) e^{-z}, z >= 0.

    scipy's ``ive`` below z = 1e8; above, where it returns NaN, the
    large-argument (Hankel) expansion I_n(z) e^{-z} ~ (2 pi z)^{-1/2}
    sum_k (-1)^k prod_{m=1..k} (mu - (2m - 1)^2) / (k! (8z)^k), mu = 4n^2
    (Abramowitz & Stegun 9.7.1), summed until its terms stop mattering
    (for n <= 16384 and z >= 1e8, mu / 8z <= 1.1 and 30 terms reach 1e-17)."""
    if z < _IVE_SWITCH:
        return float(sp.ive(n, z))
    mu = 4.0 * float(n) * float(n)
    term, acc = 1.0, 1.0
    for k in range(1, 60):
        term *= -(mu - (2 * k - 1) ** 2) / (k * 8.0 * z)
        acc += term
        if abs(term) < 1e-18 * abs(acc):
            break
    return acc / math.sqrt(2.0 * math.pi * z)


def _quad_inf(fun_over_t, s, a_break=1.0):
    """int_0^inf fun_over_t(t) * t^{-s} dt.

    On [0, a_break] the algebraic factor t^{-s} is integrated exactly by QAWS
    (scipy ``weight='alg'``), so the endpoint singularity costs no accuracy;
    [a_break, T) is cut at a_break 2^k (k = 1 .. 40) and each piece gets
    adaptive Gauss-Kronrod, which keeps a narrow peak of the integrand far out
    (large |i|, |j|: the Bessel factors are negligible until t ~ (i^2 + j^2)/4)
    from falling between quadrature nodes; the tail [T, inf) is integrated in
    the variable u = log(t / T), in which it decays like exp(-s u).
    """
    v, _ = scipy.integrate.quad(fun_over_t, 0.0, a_break, weight="alg", wvar=(-s, 0.0),
                                limit=400, epsabs=0.0, epsrel=2e-14)
    f = lambda t: fun_over_t(t) * t ** (-s)
    lo = a_break
    for _ in range(40):
        hi = 2.0 * lo
        v += scipy.integrate.quad(f, lo, hi, limit=200, epsabs=0.0, epsrel=2e-14)[0]
        lo = hi

    def tail(u):
        t = lo * math.exp(min(u, 600.0))
        return f(t) * t if math.isfinite(t) else 0.0
    v += scipy.integrate.quad(tail, 0.0, np.inf, limit=200, epsabs=0.0, epsrel=2e-14)[0]
    return v


def lap2d_bessel(alpha: float, i: int, j: int) -> float:
    """a_ij by the subordination integral (method W2; pins W1).

    (i, j) != (0, 0):  a_ij = -(s/Gamma(1-s)) int_0^inf ive(i,2t) ive(j,2t) t^{-1-s} dt
    (0, 0):            a_00 =  (s/Gamma(1-s)) int_0^inf (1 - ive(0,2t)^2) t^{-1-s} dt
    with s = alpha / 2 and ive the exponentially scaled modified Bessel function.
    """
    s = alpha / 2.0
    c = s / math.gamma(1.0 - s)
    i, j = abs(int(i)), abs(int(j))
    if i == 0 and j == 0:
        # 1 - ive(0,2t)^2 loses digits for small t: use -expm1(2 log ive).
        def f(t):  # limit 4 at t = 0
            return 4.0 if t == 0.0 else -np.expm1(2.0 * np.log(_ive(0, 2.0 * t))) / t
        return c * _quad_inf(f, s)

    def g(t):  # limit 1 at t = 0 when i + j = 1, else 0
        if t == 0.0:
            return 1.0 if i + j == 1 else 0.0
        return _ive(i, 2.0 * t) * _ive(j, 2.0 * t) / t
    brk = max(1.0, 0.25 * (i * i + j * j) ** 0.5)
    return -c * _quad_inf(g, s, brk)


def riesz_1d_bessel(alpha: float, i: int) -> float:
    """1D analogue of W2: a_i = -(s/Gamma(1-s)) int_0^inf ive(i,2t) t^{-1-s} dt, i != 0;
    a_0 = (s/Gamma(1-s)) int_0^inf (1 - ive(0,2t)) t^{-1-s} dt."""
    s = alpha / 2.0
    c = s / math.gamma(1.0 - s)
    i = abs(int(i))
    if i == 0:
        def f(t):  # limit 2 at t = 0
            return 2.0 if t == 0.0 else -np.expm1(np.log(_ive(0, 2.0 * t))) / t
        return c * _quad_inf(f, s)

    def g(t):  # limit 1 at t = 0 when i = 1, else 0
        if t == 0.0:
            return 1.0 if i == 1 else 0.0
        return _ive(i, 2.0 * t) / t
    return -c * _quad_inf(g, s, max(1.0, 0.25 * i))

"""Pins of the diffusion S-ADI oracle (oracle/diffusion.py) against what the
scheme's definition and the mathematics fix, not against itself:
* the factored step equals the unfactored scheme solved densely;
* alpha = 2, g = 0: a Dirichlet sine mode follows the scheme's closed scalar
  recursion (its factor, start step and extrapolation written out);
* g = 0: second-order convergence in tau to the exact solution of the
  semi-discrete problem, u(t) = exp(-kappa t L_h) phi1, computed from the
  eigendecomposition of the dense L_h (no time stepping involved);
* stability at time steps far beyond any explicit limit: the solution decays;
* a manufactured nonlinear forced solution converges at second order."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import diffusion as D
from oracle import sadi as S
from paper_2312_06206_gb300 import workloads as WL


def _rng(seed):
    return np.random.default_rng(20231206 + seed)


@pytest.mark.parametrize("N,alpha,g", [(1, 1.5, S.G_NEG_CUBE), (2, 1.3, S.G_NEG_SIN), (3, 1.8, S.G_ZERO),
                                       (5, 1.5, S.G_GENERAL), (7, 1.1, S.G_NEG_SIN)])
def test_factored_step_equals_unfactored_scheme(N, alpha, g):
    P = S.Problem(N, alpha, 0.7, 0.05, -1.0, 1.0, g, gc=(-1.2, -0.3, 0.6))
    Dp = D.Diffusion(P)
    ops = S.dense_operators(P)
    rng = _rng(30 + N)
    u0 = rng.uniform(-1, 1, (N, N))
    f0, f1 = rng.uniform(-1, 1, (N, N)), rng.uniform(-1, 1, (N, N))
    u1f = D.step(Dp, None, u0, True, f0)
    u1l = D.step_literal(Dp, ops, None, u0, True, f0)
    assert np.abs(u1f - u1l).max() < 1e-12 * np.abs(u1l).max()
    u2f = D.step(Dp, u0, u1f, False, f1)
    u2l = D.step_literal(Dp, ops, u0, u1f, False, f1)
    assert np.abs(u2f - u2l).max() < 1e-12 * np.abs(u2l).max()


def test_alpha2_sine_mode_recursion():
    # alpha = 2, g = 0: delta_x, delta_y and L_h = delta_x + delta_y act on the
    # mode (k, l) as mu_k, mu_l (mu_m = (4/h^2) sin^2(m pi / (2(N+1)))), so
    # u^n = c_n mode with F = (1 + kappa tau mu_k/2)(1 + kappa tau mu_l/2),
    # lam = kappa (mu_k + mu_l):  c_1 = c_0 - tau lam c_0 / F,
    # F (c_{n+1} - 2c_n + c_{n-1}) = -tau lam (3c_n - c_{n-1})/2 - (c_n - c_{n-1})
    N, kap, tau = 15, 0.8, 0.004
    P = S.Problem(N, 2.0, kap, tau)
    Dp = D.Diffusion(P)
    h = P.h
    X, Y = WL.coords(N, -1.0, 1.0)
    for (k, l) in [(1, 2), (4, 1), (7, 7)]:
        mode = np.sin(k * np.pi * (X + 1) / 2) * np.sin(l * np.pi * (Y + 1) / 2)
        mu = lambda m: 4 / h ** 2 * math.sin(m * math.pi / (2 * (N + 1))) ** 2
        F = (1 + tau * kap * mu(k) / 2) * (1 + tau * kap * mu(l) / 2)
        lam = kap * (mu(k) + mu(l))
        c = [0.7]
        c.append(c[0] - tau * lam * c[0] / F)
        for n in range(1, 40):
            c.append(2 * c[n] - c[n - 1] + (-tau * lam * (1.5 * c[n] - 0.5 * c[n - 1]) - (c[n] - c[n - 1])) / F)
        u = D.run(Dp, 0.7 * mode, 40)
        assert np.abs(u - c[40] * mode).max() < 1e-12 * abs(c[0])


@pytest.mark.parametrize("alpha", [1.3, 1.7])
def test_second_order_to_the_exact_semidiscrete_solution(alpha):
    N, kap, T = 12, 1.0, 0.05
    P0 = S.Problem(N, alpha, kap, 0.01)
    _, _, L = S.dense_operators(P0)
    w, V = scipy.linalg.eigh(L)                      # L_h is symmetric (positive definite)
    phi1 = WL.gaussian_bumps(N, 3, WL.SEED_BASE + 33)
    exact = (V @ (np.exp(-kap * T * w) * (V.T @ phi1.reshape(-1)))).reshape(N, N)
    errs = []
    for M in (10, 20, 40, 80):
        P = S.Problem(N, alpha, kap, T / M)
        errs.append(np.abs(D.run(D.Diffusion(P), phi1, M) - exact).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(3)]
    assert all(1.9 < o < 2.1 for o in orders[1:]), (orders, errs)


def test_stable_far_beyond_the_explicit_limit():
    # kappa tau / h^alpha = 10^3 .. 10^4: an explicit scheme would blow up.  As
    # with Crank-Nicolson, the scheme damps its stiffest modes only slowly
    # (amplification |z| < 1 but near 1 there), so what is fixed is that the
    # norm never exceeds its initial value and decays overall
    N, alpha = 31, 1.6
    for tau in (1.0, 10.0):
        P = S.Problem(N, alpha, 1.0, tau)
        Dp = D.Diffusion(P)
        phi1 = WL.gaussian_bumps(N, 5, WL.SEED_BASE + 34)
        norms = [np.linalg.norm(phi1)]
        u_prev, u = None, phi1
        for n in range(200):
            u_prev, u = u, D.step(Dp, u_prev, u, n == 0, tier="fft")
            norms.append(np.linalg.norm(u))
        assert max(norms[1:]) <= norms[0] and norms[-1] < 0.1 * norms[0], (tau, norms[-1] / norms[0])


def test_fft_tier_equals_direct_tier():
    P = S.Problem(25, 1.4, 0.9, 0.01, g=S.G_NEG_SIN)
    Dp = D.Diffusion(P)
    phi1 = WL.gaussian_bumps(25, 4, 9)
    a = D.run(Dp, phi1, 8, tier="direct")
    b = D.run(Dp, phi1, 8, tier="fft")
    assert S.rel_l2(b, a) < 1e-12


def test_manufactured_forced_solution_second_order():
    # U = exp(-beta r^2) cos(omega t) (r from a fixed centre), forced by
    # f = U_t + kappa L_h U - g(U) at the step midpoints t_{n+1/2}
    N, alpha, kap, T, om, beta = 31, 1.5, 1.0, 0.4, 3.0, 12.0
    coef = (-1.0, -0.5, 0.2)
    X, Y = WL.coords(N, -1.0, 1.0)
    prof = np.exp(-beta * ((X - 0.1) ** 2 + (Y + 0.05) ** 2))
    errs = []
    for M in (20, 40, 80):
        tau = T / M
        P = S.Problem(N, alpha, kap, tau, g=S.G_GENERAL, gc=coef)
        Lp = S.lh_direct(P, prof)

        def forcing(n):
            t = (n + 0.5) * tau
            U = prof * math.cos(om * t)
            return -om * math.sin(om * t) * prof + kap * math.cos(om * t) * Lp - S.g_eval(S.G_GENERAL, U, coef)
        u = D.run(D.Diffusion(P), prof, M, forcing=forcing)
        errs.append(np.abs(u - prof * math.cos(om * T)).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.85 < o < 2.15 for o in orders), (orders, errs)

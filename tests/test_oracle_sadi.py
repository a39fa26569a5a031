"""Pins of the S-ADI oracle (oracle/sadi.py) against what the paper and the
mathematics fix: brute-force sums, closed forms, the literal scheme as printed,
the energy identity of the stability theorem, the alpha -> 2 classical limit,
second-order convergence, and the paper's own error tables (Sec. 6)."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
import scipy.special as sp

from oracle import sadi as S
from oracle import weights as W
from paper_2312_06206_gb300 import workloads as WL


def _rng(k):
    return np.random.default_rng(1000 + k)


# ---------------------------------------------------------------- L_h -------

def test_lh_direct_equals_entrywise_sum():
    # the block-Toeplitz evaluation equals the defining double sum of Sec. 2
    P = S.Problem(5, 1.4, 1.0, 0.1)
    Dx, Dy, L = S.dense_operators(P)
    u = _rng(0).standard_normal((5, 5))
    lhs = S.lh_direct(P, u).reshape(-1)
    ref = np.zeros(25)
    for j in range(5):
        for i in range(5):
            acc = 0.0
            for jj in range(5):
                for ii in range(5):
                    acc += P.A2[abs(i - ii), abs(j - jj)] * u[jj, ii]
            ref[j * 5 + i] = acc / P.h ** P.alpha
    assert np.abs(lhs - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(L @ u.reshape(-1) - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N", [1, 2, 16, 31])
def test_lh_fft_equals_direct(N):
    P = S.Problem(N, 1.7, 1.0, 0.1)
    u = _rng(N).standard_normal((N, N))
    a, b = S.lh_fft(P, u), S.lh_direct(P, u)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("N,Q", [(16, 31), (16, 64), (31, 61), (31, 70), (1, 1)])
def test_lh_fft_any_circulant_size_equals_direct(N, Q):
    # Sec. 3: the block-circulant embedding reproduces the block-Toeplitz
    # product for every size Q >= 2N - 1 (the smallest one included)
    P = S.Problem(N, 1.4, 1.0, 0.1, fft_size=Q, fft_workers=2)
    u = _rng(N + Q).standard_normal((N, N))
    a, b = S.lh_fft(P, u), S.lh_direct(P, u)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()
    with pytest.raises(ValueError):
        S.lh_fft(S.Problem(N + 1, 1.4, 1.0, 0.1, fft_size=2 * N), u)


@pytest.mark.parametrize("alpha", [1.3, 1.7])
def test_lh_unit_disk_closed_form(alpha):
    # (-Delta)^{alpha/2} (1 - r^2)_+^{alpha/2} = 2^alpha Gamma(1 + alpha/2)^2 for
    # r < 1 (d = 2); L_h approaches it as h -> 0 (Sec. 5 consistency lemma).
    ex = 2 ** alpha * math.gamma(1 + alpha / 2) ** 2
    errs = []
    for N in (31, 63, 127):
        P = S.Problem(N, alpha, 1.0, 0.01)
        X, Y = WL.coords(N, -1.0, 1.0)
        r2 = X * X + Y * Y
        u = np.where(r2 < 1, (1 - np.minimum(r2, 1)) ** (alpha / 2), 0.0)
        Lu = S.lh_fft(P, u)
        m = r2 <= 0.25
        errs.append(np.abs(Lu[m] - ex).max() / ex)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-5


def test_lh_gaussian_second_order():
    # (-Delta)^{alpha/2} e^{-beta r^2} by its Hankel transform (the Fourier
    # transform of Sec. 5): (1/2pi) int k^alpha (pi/beta) e^{-k^2/4beta} J0(kr) k dk.
    # L_h converges to it at order 2 (Sec. 5 consistency lemma).
    alpha, beta = 1.5, 40.0

    def exact(r):
        f = lambda k: k ** alpha * (np.pi / beta) * np.exp(-k * k / (4 * beta)) * sp.j0(k * r) * k
        v, _ = scipy.integrate.quad(f, 0, 60 * np.sqrt(beta), limit=2000, epsabs=1e-13)
        return v / (2 * np.pi)
    ys = [0.0, 0.125, 0.25]
    ref = [exact(y) for y in ys]
    errs = []
    for N in (127, 255, 511):
        P = S.Problem(N, alpha, 1.0, 0.01)
        X, Y = WL.coords(N, -1.0, 1.0)
        Lu = S.lh_fft(P, np.exp(-beta * (X * X + Y * Y)))
        ic = (N - 1) // 2
        e = 0.0
        for y, r in zip(ys, ref):
            j = int(round((y + 1.0) * (N + 1) / 2.0)) - 1
            assert abs(Y[j, 0] - y) < 1e-12
            e = max(e, abs(Lu[j, ic] - r))
        errs.append(e)
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.9 < o < 2.1 for o in orders), orders


# --------------------------------------------------- SPD / lemma pins -------

@pytest.mark.parametrize("alpha", [1.2, 1.6, 1.95])
def test_operators_spd_and_remainder_nsd(alpha):
    # Sec. 4 lemmas: delta_x+delta_y, delta_x delta_y and L_h define inner
    # products; ||w||_A <= ||w||_At, i.e. L_h - delta_x - delta_y is NSD.
    P = S.Problem(7, alpha, 1.0, 0.1)
    Dx, Dy, L = S.dense_operators(P)
    for Mx in (Dx + Dy, Dx @ Dy, L):
        Ms = 0.5 * (Mx + Mx.T)
        assert np.abs(Mx - Mx.T).max() < 1e-10 * np.abs(Mx).max()
        assert np.linalg.eigvalsh(Ms).min() > 0
    R = L - Dx - Dy
    assert np.linalg.eigvalsh(0.5 * (R + R.T)).max() < 0
    # H is SPD with eigenvalues above one
    ev = np.linalg.eigvalsh(P.H)
    assert ev.min() > 1.0


# ---------------------------------------------------- Gohberg-Semencul -----

@pytest.mark.parametrize("N", [1, 2, 3, 8, 31, 64, 127])
def test_gs_algorithm1_equals_dense_solve(N):
    rng = _rng(N)
    alpha = rng.uniform(1.05, 1.95)
    s = rng.uniform(0.01, 5.0)
    a = W.riesz_1d(alpha, N)
    H = np.eye(N) + s * scipy.linalg.toeplitz(a)
    c = S.gs_generator(H)
    assert c[0] > 0
    # the generator itself: H c = e_1
    e1 = np.zeros(N)
    e1[0] = 1
    assert np.abs(H @ c - e1).max() < 1e-13
    V = rng.standard_normal((5, N))
    X = S.gs_solve(c, V)
    ref = np.linalg.solve(H, V.T).T
    assert np.abs(X - ref).max() < 1e-13 * np.abs(ref).max()


# ------------------------------------------------------------- scheme -------

@pytest.mark.parametrize("N,alpha,g", [(1, 1.5, S.G_NEG_CUBE), (2, 1.3, S.G_NEG_SIN),
                                       (3, 1.5, S.G_NEG_CUBE), (5, 1.8, S.G_NEG_SIN),
                                       (7, 1.1, S.G_ZERO)])
def test_factored_step_equals_literal_three_level_scheme(N, alpha, g):
    # Sec. 3 eq. "ADI scheme equivalent" (factored, with the full L_h in B)
    # reproduces eqs. "ADI scheme" and "ADI scheme initial" (remainder form,
    # Riesz average at n +- 1, perturbation delta_x delta_y), solved densely.
    P = S.Problem(N, alpha, 0.7, 0.3, -1.0, 1.0, g)
    ops = S.dense_operators(P)
    rng = _rng(10 + N)
    u0 = rng.uniform(-1, 1, (N, N))
    phi2 = rng.uniform(-1, 1, (N, N))
    u1f = S.step(P, None, u0, True, phi2)
    u1l = S.step_literal(P, ops, None, u0, True, phi2)
    assert np.abs(u1f - u1l).max() < 1e-12 * np.abs(u1l).max()
    u2f = S.step(P, u0, u1f, False)
    u2l = S.step_literal(P, ops, u0, u1f, False)
    assert np.abs(u2f - u2l).max() < 1e-12 * np.abs(u2l).max()


@pytest.mark.parametrize("tier", ["direct", "fft"])
def test_transposed_data_gives_the_transposed_solution(tier):
    # the scheme is symmetric in x and y (Sec. 3: the two factors act on
    # different indices and commute, and a_ij = a_ji), so data phi^T must give
    # u^T; asymmetric data and forcing make any x/y mix-up of the oracle show
    N, steps = 15, 4
    P = S.Problem(N, 1.6, 0.8, 0.05, -1.0, 1.0, 1)
    rng = _rng(77)
    phi1 = rng.uniform(-1, 1, (N, N))
    phi2 = 0.3 * rng.uniform(-1, 1, (N, N))
    u = S.run(P, phi1, phi2, steps, tier=tier)
    ut = S.run(P, phi1.T.copy(), phi2.T.copy(), steps, tier=tier)
    assert np.abs(u - u.T).max() > 1e-3 * np.abs(u).max()    # the data is asymmetric
    assert np.abs(ut - u.T).max() <= 1e-12 * np.abs(u).max()


def test_energy_conserved_without_nonlinearity():
    # Sec. 4 stability theorem: with g = 0, (H_n^2 - H_{n-1}^2)/tau = I_2 = 0,
    # so H_n is constant from n = 0 (the start step included).
    P = S.Problem(15, 1.5, 1.0, 0.2)
    phi1 = WL.gaussian(15, 5.0)
    phi2 = 0.3 * WL.random_field(15, 3)
    _, hist = S.run(P, phi1, phi2, 20, keep=True)
    Hn = [S.energy(P, hist[n], hist[n + 1]) for n in range(20)]
    assert max(Hn) - min(Hn) < 1e-13 * Hn[0]
    # and with g = -u^3 it is not (the pin is sensitive to the scheme)
    Pg = S.Problem(15, 1.5, 1.0, 0.2, g=S.G_NEG_CUBE)
    _, hg = S.run(Pg, 3 * phi1, phi2, 20, keep=True)
    Hg = [S.energy(Pg, hg[n], hg[n + 1]) for n in range(20)]
    assert max(Hg) - min(Hg) > 1e-6 * Hg[0]


def test_alpha2_single_sine_mode_recursion():
    # alpha = 2: L_h = delta_x + delta_y (5-point stencil), the remainder
    # vanishes, and a Dirichlet sine mode (k, l) is an eigenvector with
    # mu_k = (4/h^2) sin^2(k pi / (2(N+1))).  u^n = c_n * mode with
    # (1+t^2 k mu_k/2)(1+t^2 k mu_l/2)(c_{n+1}-2c_n+c_{n-1}) = -t^2 k (mu_k+mu_l) c_n,
    # and (...)(c_1 - c_0) = t d_0 - t^2/2 k (mu_k+mu_l) c_0 at the start.
    N, kap, tau = 15, 0.8, 0.05
    P = S.Problem(N, 2.0, kap, tau)
    h = P.h
    for (k, l) in [(1, 2), (3, 1), (7, 7)]:
        X, Y = WL.coords(N, -1.0, 1.0)
        mode = np.sin(k * np.pi * (X + 1) / 2) * np.sin(l * np.pi * (Y + 1) / 2)
        mu = lambda m: 4 / h ** 2 * math.sin(m * math.pi / (2 * (N + 1))) ** 2
        fac = (1 + tau ** 2 * kap * mu(k) / 2) * (1 + tau ** 2 * kap * mu(l) / 2)
        lam = mu(k) + mu(l)
        c0, d0 = 0.7, -0.4
        u_end = S.run(P, c0 * mode, d0 * mode, 30)
        c = [c0, c0 + (tau * d0 - 0.5 * tau ** 2 * kap * lam * c0) / fac]
        for n in range(1, 30):
            c.append(2 * c[n] - c[n - 1] - tau ** 2 * kap * lam * c[n] / fac)
        assert np.abs(u_end - c[30] * mode).max() < 1e-12 * abs(c[30])


def test_general_g_reduces_to_the_named_kinds():
    # g(u) = c1 u + c3 u^3 + cs sin u: (0, -1, 0) is the Klein-Gordon term and
    # (0, 0, -1) the sine-Gordon term of Sec. 6, exactly
    u = _rng(3).uniform(-3, 3, (7, 5))
    assert np.array_equal(S.g_eval(S.G_GENERAL, u, (0.0, -1.0, 0.0)), S.g_eval(S.G_NEG_CUBE, u))
    assert np.array_equal(S.g_eval(S.G_GENERAL, u, (0.0, 0.0, -1.0)), S.g_eval(S.G_NEG_SIN, u))
    assert np.array_equal(S.g_eval(S.G_GENERAL, u, (0.0, 0.0, 0.0)), np.zeros_like(u))
    assert np.array_equal(S.g_eval(S.G_GENERAL, u, (2.0, 0.0, 0.0)), 2.0 * u)


def test_alpha2_sine_mode_with_linear_g():
    # g(u) = c1 u keeps a Dirichlet sine mode a mode at alpha = 2: B^n gains
    # tau^2 c1 c_n, so (1+t^2 k mu_k/2)(1+t^2 k mu_l/2)(c_{n+1}-2c_n+c_{n-1})
    # = t^2 (c1 - k (mu_k + mu_l)) c_n, and the start step carries t^2/2 c1 c_0
    N, kap, tau, c1 = 15, 0.8, 0.05, -2.5
    P = S.Problem(N, 2.0, kap, tau, g=S.G_GENERAL, gc=(c1, 0.0, 0.0))
    h = P.h
    for (k, l) in [(1, 2), (5, 3)]:
        X, Y = WL.coords(N, -1.0, 1.0)
        mode = np.sin(k * np.pi * (X + 1) / 2) * np.sin(l * np.pi * (Y + 1) / 2)
        mu = lambda m: 4 / h ** 2 * math.sin(m * math.pi / (2 * (N + 1))) ** 2
        fac = (1 + tau ** 2 * kap * mu(k) / 2) * (1 + tau ** 2 * kap * mu(l) / 2)
        lam = kap * (mu(k) + mu(l)) - c1
        c0, d0 = 0.7, -0.4
        u_end = S.run(P, c0 * mode, d0 * mode, 30)
        c = [c0, c0 + (tau * d0 - 0.5 * tau ** 2 * lam * c0) / fac]
        for n in range(1, 30):
            c.append(2 * c[n] - c[n - 1] - tau ** 2 * lam * c[n] / fac)
        assert np.abs(u_end - c[30] * mode).max() < 1e-12 * abs(c[30])


@pytest.mark.parametrize("N,alpha", [(3, 1.5), (6, 1.7)])
def test_factored_step_equals_literal_scheme_general_g(N, alpha):
    P = S.Problem(N, alpha, 0.7, 0.3, -1.0, 1.0, S.G_GENERAL, gc=(-1.3, -0.4, 0.8))
    ops = S.dense_operators(P)
    rng = _rng(20 + N)
    u0 = rng.uniform(-1, 1, (N, N))
    phi2 = rng.uniform(-1, 1, (N, N))
    u1f = S.step(P, None, u0, True, phi2)
    u1l = S.step_literal(P, ops, None, u0, True, phi2)
    assert np.abs(u1f - u1l).max() < 1e-12 * np.abs(u1l).max()
    u2f = S.step(P, u0, u1f, False)
    u2l = S.step_literal(P, ops, u0, u1f, False)
    assert np.abs(u2f - u2l).max() < 1e-12 * np.abs(u2l).max()


def test_fft_tier_equals_direct_tier():
    P = S.Problem(31, 1.6, 1.0, 0.02, g=S.G_NEG_SIN)
    phi1 = WL.gaussian_bumps(31, 4, 7)
    phi2 = 0.5 * WL.gaussian(31, 10.0)
    a = S.run(P, phi1, phi2, 10, tier="direct")
    b = S.run(P, phi1, phi2, 10, tier="fft")
    assert S.rel_l2(b, a) < 1e-12


def test_manufactured_solution_second_order_in_time():
    # forcing f^n = U_tt + kappa L_h U - g(U) makes the smooth U(t) = cos(t) phi
    # a solution of the semi-discrete problem; the S-ADI scheme must converge
    # to it at O(tau^2) (Sec. 5 convergence theorem).
    N, alpha, kap = 31, 1.5, 1.0
    phi = WL.gaussian(N, 8.0)
    errs = []
    for M in (8, 16, 32):
        tau = 1.0 / M
        P = S.Problem(N, alpha, kap, tau, g=S.G_NEG_CUBE)
        Lphi = S.lh_direct(P, phi)

        def forcing(n, P=P, tau=tau):
            t = n * tau
            U = math.cos(t) * phi
            return -math.cos(t) * phi + kap * math.cos(t) * Lphi - S.g_eval(P.g, U)
        u = S.run(P, phi, 0 * phi, M, forcing=forcing)
        errs.append(np.abs(u - math.cos(1.0) * phi).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.9 < o < 2.15 for o in orders), orders


# ------------------------------------------ the paper's own error tables ----

@pytest.mark.parametrize("alpha,ref", [(1.1, 6.3150e-02), (1.5, 8.1276e-02), (1.9, 1.0716e-01)])
def test_paper_table2_example1_space_error(alpha, ref):
    # Sec. 6 Table 2, S-ADI, h = 1 (N = 19 vs N = 39), tau = 1/100, t = 5
    us = []
    for N in (19, 39):
        w = WL.paper_example1(N, alpha, 1 / 100)
        P = S.Problem(N, alpha, 1.0, w.tau, w.a, w.b, w.g)
        us.append(S.run(P, w.phi1, w.phi2, w.steps, tier="fft"))
    e = S.error2(20.0 / 20, us[0], us[1])
    # half a unit of the last printed digit (5 significant digits)
    assert abs(e - ref) <= 0.5 * 10 ** (math.floor(math.log10(ref)) - 4), (e, ref)


def test_paper_table4_example2_space_error():
    # Sec. 6 Table 4, S-ADI, alpha = 1.5, h = 2/5 (N = 49 vs 99), tau = 1/125, t = 8;
    # reproduced with phi1 = 2 sech(cosh(x^2+y^2)) (see workloads.paper_example2)
    alpha, ref = 1.5, 3.9151e-01
    us = []
    for N in (49, 99):
        w = WL.paper_example2(N, alpha, 1 / 125)
        P = S.Problem(N, alpha, 1.0, w.tau, w.a, w.b, w.g)
        us.append(S.run(P, w.phi1, w.phi2, w.steps, tier="fft"))
    e = S.error2(20.0 / 50, us[0], us[1])
    assert abs(e - ref) <= 0.5e-5, (e, ref)


@pytest.mark.slow
def test_paper_table1_example1_time_error():
    # Sec. 6 Table 1, S-ADI, alpha = 1.5, h = 1/40 (N = 799), tau = 1/10 vs 1/20, t = 5
    alpha, ref = 1.5, 8.9900e-03
    N = 799
    us = []
    A2 = W.lap2d_trap(alpha, N)
    for tau in (1 / 10, 1 / 20):
        w = WL.paper_example1(N, alpha, tau)
        P = S.Problem(N, alpha, 1.0, tau, w.a, w.b, w.g, A2=A2)
        us.append(S.run(P, w.phi1, w.phi2, w.steps, tier="fft"))
    e = S.error1(1 / 40, us[0], us[1])
    assert abs(e - ref) < 0.5e-7, (e, ref)

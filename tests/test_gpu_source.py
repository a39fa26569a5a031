"""The general nonlinearity g(u) = c1 u + c3 u^3 + cs sin u and the per-step
source field (sadi_step_source) through the C ABI.

* g: every step form against the oracle (FP64 <= 1e-10, FP32 forms <= 1e-5,
  relative L2 and element-wise), and at alpha = 2 with g = c1 u against the
  closed scalar recursion of a Dirichlet sine mode.
* f^n: arbitrary (non-separable) fields, one per step, given as device
  buffers of double or float, against the oracle's forcing; and a
  manufactured solution -- a Gaussian moving on a curve, U(x, y, t) -- driven by
  f^n = U_tt + kappa L_h U - g(U) (L_h the discrete operator, so only the time
  discretisation errs), which the scheme must follow to second order in tau."""
import math

import numpy as np
import pytest

from oracle import sadi as O
from paper_2312_06206_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

PRECS = [("SADI_PREC_FP64", 1e-10), ("SADI_PREC_FP32", 1e-5), ("SADI_PREC_FP32_DENSE", 1e-5)]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_06206_gb300 import build
    build.build()
    from paper_2312_06206_gb300 import sadi
    return sadi, torch


def _close(u, ref, tol, what):
    rel = O.rel_l2(u, ref)
    ew = np.abs(u - ref).max() / np.abs(ref).max()
    assert rel <= tol and ew <= tol, (what, rel, ew)


@pytest.mark.parametrize("prec_name,tol", PRECS)
@pytest.mark.parametrize("N,alpha,coef", [(31, 1.4, (-1.0, -1.0, 0.0)), (100, 1.7, (-2.0, 0.5, -0.7)),
                                          (255, 1.2, (0.3, -0.2, -1.5))])
def test_general_g_against_oracle(env, prec_name, tol, N, alpha, coef):
    S, _ = env
    kappa, tau, steps = 0.9, 0.02, 6
    phi1 = WL.gaussian_bumps(N, 5, WL.SEED_BASE + 80 + N)
    phi2 = 0.3 * WL.gaussian(N, 12.0)
    P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, O.G_GENERAL, gc=coef)
    ref = O.run(P, phi1, phi2, steps, tier="direct" if N <= 40 else "fft")
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(0, getattr(S, prec_name))
        s.sadi_set_nonlinearity(*coef)
        assert s.sadi_get_options()[0] == S.SADI_G_GENERAL
        s.set_initial(phi1, phi2)
        s.step(steps)
        u, _ = s.get()
    _close(u, ref, tol, (prec_name, N))


def test_linear_g_sine_mode_closed_recursion(env):
    # alpha = 2, g = c1 u: u^n = c_n mode with
    # (1 + t^2 k mu_k/2)(1 + t^2 k mu_l/2)(c_{n+1} - 2c_n + c_{n-1}) = t^2 (c1 - k(mu_k + mu_l)) c_n
    S, _ = env
    N, kap, tau, c1, k, l, M = 63, 0.8, 0.01, -3.0, 3, 5, 40
    X, Y = WL.coords(N, -1.0, 1.0)
    mode = np.sin(k * np.pi * (X + 1) / 2) * np.sin(l * np.pi * (Y + 1) / 2)
    h = 2.0 / (N + 1)
    mu = lambda m: 4 / h ** 2 * math.sin(m * math.pi / (2 * (N + 1))) ** 2
    fac = (1 + tau ** 2 * kap * mu(k) / 2) * (1 + tau ** 2 * kap * mu(l) / 2)
    lam = kap * (mu(k) + mu(l)) - c1
    c0, d0 = 0.7, -0.4
    c = [c0, c0 + (tau * d0 - 0.5 * tau ** 2 * lam * c0) / fac]
    for n in range(1, M):
        c.append(2 * c[n] - c[n - 1] - tau ** 2 * lam * c[n] / fac)
    with S.Sadi(N, 2.0, kap, tau) as s:
        s.set_options(0, S.SADI_PREC_FP64)
        s.sadi_set_nonlinearity(c1, 0.0, 0.0)
        s.set_initial(c0 * mode, d0 * mode)
        s.step(M)
        u, _ = s.get()
    assert np.abs(u - c[M] * mode).max() < 1e-12 * abs(c[M])


@pytest.mark.parametrize("prec_name,tol", PRECS)
@pytest.mark.parametrize("N,dtype", [(37, 0), (100, 1), (255, 0)])
def test_step_source_fields_against_oracle(env, prec_name, tol, N, dtype):
    S, torch = env
    alpha, kappa, tau, g, steps = 1.6, 1.1, 0.02, 2, 5
    rng = np.random.default_rng(WL.SEED_BASE + 90 + N)
    fields = [rng.uniform(-2, 2, (N, N)) for _ in range(steps)]
    if dtype == 1:   # the oracle gets the same values the float buffers hold
        fields = [f.astype(np.float32).astype(np.float64) for f in fields]
    phi1 = WL.gaussian_bumps(N, 5, WL.SEED_BASE + 91 + N)
    P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, g)
    ref = O.run(P, phi1, np.zeros_like(phi1), steps, tier="direct" if N <= 40 else "fft",
                forcing=lambda n: fields[n])
    tdt = torch.float64 if dtype == 0 else torch.float32
    dev = [torch.tensor(f, dtype=tdt, device="cuda") for f in fields]
    torch.cuda.synchronize()
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(g, getattr(S, prec_name))
        s.set_initial(phi1)
        for n in range(steps):
            s.sadi_step_source(dev[n].data_ptr(), dtype)
        u, k = s.get()
    assert k == steps
    _close(u, ref, tol, (prec_name, N, dtype))


def _moving_bump(X, Y, t, beta=30.0):
    """U = exp(-beta (X^2 + Y^2)), X = x - a(t), Y = y - b(t), a = 0.3 cos t,
    b = 0.2 sin 2t, with U_t = q U and U_tt = (q' + q^2) U."""
    a, da, dda = 0.3 * math.cos(t), -0.3 * math.sin(t), -0.3 * math.cos(t)
    b, db, ddb = 0.2 * math.sin(2 * t), 0.4 * math.cos(2 * t), -0.8 * math.sin(2 * t)
    Xs, Ys = X - a, Y - b
    U = np.exp(-beta * (Xs * Xs + Ys * Ys))
    q = 2 * beta * (Xs * da + Ys * db)
    dq = 2 * beta * (-da * da + Xs * dda - db * db + Ys * ddb)
    return U, q * U, (dq + q * q) * U


def test_step_source_manufactured_solution_second_order(env):
    S, torch = env
    N, alpha, kappa, T = 63, 1.5, 1.0, 0.5
    coef = (-1.0, -0.5, 0.0)
    X, Y = WL.coords(N, -1.0, 1.0)
    errs = []
    for M in (20, 40, 80):
        tau = T / M
        P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, O.G_GENERAL, gc=coef)
        fs = []
        for n in range(M):
            U, _, Utt = _moving_bump(X, Y, n * tau)
            fs.append(Utt + kappa * O.lh_fft(P, U) - O.g_eval(O.G_GENERAL, U, coef))
        dev = torch.tensor(np.stack(fs), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        U0, Ut0, _ = _moving_bump(X, Y, 0.0)
        with S.Sadi(N, alpha, kappa, tau) as s:
            s.set_options(0, S.SADI_PREC_FP64)
            s.sadi_set_nonlinearity(*coef)
            s.set_initial(U0, Ut0)
            for n in range(M):
                s.sadi_step_source(dev[n].data_ptr(), 0)
            u, _ = s.get()
        UT, _, _ = _moving_bump(X, Y, T)
        errs.append(np.abs(u - UT).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.85 < o < 2.15 for o in orders), (orders, errs)


def test_step_source_argument_errors(env):
    S, torch = env
    N = 15
    f = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    with S.Sadi(N, 1.5, 1.0, 0.01) as s:
        with pytest.raises(S.SadiError) as ei:          # before set_initial
            s.sadi_step_source(f.data_ptr(), 0)
        assert ei.value.status == S.SADI_ESTATE
        s.set_initial(np.zeros((N, N)))
        host = np.zeros((N, N))
        for ptr, dt in ((host.ctypes.data, 0), (f.data_ptr(), 2), (0, 0)):
            with pytest.raises(S.SadiError) as ei:
                s.sadi_step_source(ptr, dt)
            assert ei.value.status == S.SADI_EINVAL
        s.sadi_set_source(np.ones((N, N)), 1.0, 0.0)
        with pytest.raises(S.SadiError) as ei:          # a separable source is set
            s.sadi_step_source(f.data_ptr(), 0)
        assert ei.value.status == S.SADI_ESTATE

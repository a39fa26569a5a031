"""The diffusion S-ADI step (sadi_create_diffusion) through the C ABI against
the diffusion oracle (oracle/diffusion.py) and against what the mathematics
fixes: FP64 <= 1e-10 and the FP32 forms <= 1e-5 (relative L2 and
element-wise) on ragged sizes; the alpha = 2 sine-mode recursion; second
order in tau to the exact semi-discrete solution exp(-kappa t L_h) phi1 and
to a manufactured forced solution."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import diffusion as D
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


def _gpu(S, N, alpha, kappa, tau, g, phi1, steps, prec, coef=None):
    with S.Sadi(N, alpha, kappa, tau, equation="diffusion") as s:
        assert s.sadi_get_equation() == 1
        s.set_options(g, prec)
        if coef is not None:
            s.sadi_set_nonlinearity(*coef)
        s.set_initial(phi1)
        s.step(steps)
        u, n = s.get()
    assert n == steps
    return u


def _close(u, ref, tol, what):
    rel = O.rel_l2(u, ref)
    ew = np.abs(u - ref).max() / np.abs(ref).max()
    assert rel <= tol and ew <= tol, (what, rel, ew)


@pytest.mark.parametrize("prec_name,tol", PRECS)
@pytest.mark.parametrize("N,alpha,g", [(1, 1.5, 1), (7, 1.3, 2), (31, 1.8, 0), (100, 1.5, 3), (255, 1.2, 2)])
def test_diffusion_step_against_oracle(env, prec_name, tol, N, alpha, g):
    S, _ = env
    kappa, tau, steps = 0.8, 2e-4, 6
    coef = (1.0, -1.0, 0.0) if g == 3 else None          # Allen-Cahn type u - u^3
    phi1 = WL.gaussian_bumps(N, 5, WL.SEED_BASE + 100 + N) if N > 1 else np.array([[0.7]])
    P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, g, gc=coef or (0.0, 0.0, 0.0))
    ref = D.run(D.Diffusion(P), phi1, steps, tier="direct" if N <= 40 else "fft")
    u = _gpu(S, N, alpha, kappa, tau, g, phi1, steps, getattr(S, prec_name), coef)
    _close(u, ref, tol, (prec_name, N))


@pytest.mark.parametrize("prec_name", ["SADI_PREC_FP32", "SADI_PREC_FP32_DENSE"])
@pytest.mark.parametrize("N", [1023, 2047])
def test_diffusion_fp32_forms_track_fp64(env, prec_name, N):
    S, _ = env
    alpha, kappa, tau, g, steps = 1.6, 1.0, 3e-6, 1, 40     # s a_0 <= 0.17 (dense form)
    phi1 = WL.gaussian_bumps(N, 8, WL.SEED_BASE + 110 + N)
    u64 = _gpu(S, N, alpha, kappa, tau, g, phi1, steps, S.SADI_PREC_FP64)
    u32 = _gpu(S, N, alpha, kappa, tau, g, phi1, steps, getattr(S, prec_name))
    _close(u32, u64, 1e-5, (prec_name, N))


def test_diffusion_alpha2_sine_mode_recursion(env):
    S, _ = env
    N, kap, tau, M = 63, 0.8, 5e-4, 40
    h = 2.0 / (N + 1)
    X, Y = WL.coords(N, -1.0, 1.0)
    k, l = 3, 6
    mode = np.sin(k * np.pi * (X + 1) / 2) * np.sin(l * np.pi * (Y + 1) / 2)
    mu = lambda m: 4 / h ** 2 * math.sin(m * math.pi / (2 * (N + 1))) ** 2
    F = (1 + tau * kap * mu(k) / 2) * (1 + tau * kap * mu(l) / 2)
    lam = kap * (mu(k) + mu(l))
    c = [0.7, 0.7 - tau * lam * 0.7 / F]
    for n in range(1, M):
        c.append(2 * c[n] - c[n - 1] + (-tau * lam * (1.5 * c[n] - 0.5 * c[n - 1]) - (c[n] - c[n - 1])) / F)
    u = _gpu(S, N, 2.0, kap, tau, 0, 0.7 * mode, M, S.SADI_PREC_FP64)
    assert np.abs(u - c[M] * mode).max() < 1e-12 * 0.7


def test_diffusion_second_order_to_the_exact_semidiscrete_solution(env):
    S, _ = env
    N, alpha, kap, T = 12, 1.5, 1.0, 0.05
    P0 = O.Problem(N, alpha, kap, 0.01)
    _, _, L = O.dense_operators(P0)
    w, V = scipy.linalg.eigh(L)
    phi1 = WL.gaussian_bumps(N, 3, WL.SEED_BASE + 120)
    exact = (V @ (np.exp(-kap * T * w) * (V.T @ phi1.reshape(-1)))).reshape(N, N)
    errs = [np.abs(_gpu(S, N, alpha, kap, T / M, 0, phi1, M, S.SADI_PREC_FP64) - exact).max()
            for M in (20, 40, 80)]
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.9 < o < 2.1 for o in orders), (orders, errs)


def test_diffusion_manufactured_forced_solution(env):
    # U = exp(-beta r^2) cos(omega t), f^{n+1/2} = U_t + kappa L_h U - g(U) at
    # the step midpoints, given to sadi_step_source as device fields
    S, torch = env
    N, alpha, kap, T, om, beta = 63, 1.5, 1.0, 0.4, 3.0, 12.0
    coef = (-1.0, -0.5, 0.2)
    X, Y = WL.coords(N, -1.0, 1.0)
    prof = np.exp(-beta * ((X - 0.1) ** 2 + (Y + 0.05) ** 2))
    errs = []
    for M in (20, 40, 80):
        tau = T / M
        P = O.Problem(N, alpha, kap, tau, g=O.G_GENERAL, gc=coef)
        Lp = O.lh_fft(P, prof)
        fs = []
        for n in range(M):
            t = (n + 0.5) * tau
            U = prof * math.cos(om * t)
            fs.append(-om * math.sin(om * t) * prof + kap * math.cos(om * t) * Lp - O.g_eval(O.G_GENERAL, U, coef))
        dev = torch.tensor(np.stack(fs), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        with S.Sadi(N, alpha, kap, tau, equation="diffusion") as s:
            s.set_options(0, S.SADI_PREC_FP64)
            s.sadi_set_nonlinearity(*coef)
            s.set_initial(prof)
            for n in range(M):
                s.sadi_step_source(dev[n].data_ptr(), 0)
            u, _ = s.get()
        errs.append(np.abs(u - prof * math.cos(om * T)).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.85 < o < 2.15 for o in orders), (orders, errs)


def test_diffusion_rejects_phi2(env):
    S, _ = env
    with S.Sadi(15, 1.5, 1.0, 0.01, equation="diffusion") as s:
        with pytest.raises(S.SadiError) as ei:
            s.set_initial(np.zeros((15, 15)), np.zeros((15, 15)))
        assert ei.value.status == S.SADI_EINVAL
    with S.Sadi(15, 1.5, 1.0, 0.01) as s:
        assert s.sadi_get_equation() == 0

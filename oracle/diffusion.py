"""S-ADI for the fractional Laplacian diffusion equation (FP64 CPU oracle,
test infrastructure only).

Problem (the diffusion counterpart that the paper's conclusion, Sec. 7,
names as a further application of the S-ADI idea):
    u_t = -kappa (-Delta)^{alpha/2} u + g(u) + f   on Omega = (a, b)^2,
    u = 0 outside Omega,  u(., 0) = phi1,
discretised in space exactly as the wave equation (Sec. 2: L_h, delta_x,
delta_y on the N x N interior grid).

The paper states no scheme for it.  This oracle follows the reading that
carries the S-ADI construction of Secs. 2-3 over to a first-order-in-time
problem: split L_h = (delta_x + delta_y) + R (R the remainder), treat the
split Riesz parts implicitly by Crank-Nicolson, R and g explicitly at
t_{n+1/2} by extrapolation u~ = (3u^n - u^{n-1})/2, and add the perturbation
(kappa^2 tau / 4) delta_x delta_y acting on the second difference so that
the implicit operator factors into two one-dimensional Toeplitz systems:

  n >= 1:
    (u^{n+1} - u^n)/tau = -kappa (delta_x + delta_y)(u^{n+1} + u^n)/2
                          - kappa R u~ + g(u~) + f^{n+1/2}
                          - (kappa^2 tau/4) delta_x delta_y (u^{n+1} - 2u^n + u^{n-1})
  n = 0 (no u^{-1}; u~ = u^0, first difference in the perturbation):
    (u^1 - u^0)/tau = -kappa (delta_x + delta_y)(u^1 + u^0)/2 - kappa R u^0
                      + g(u^0) + f^{1/2} - (kappa^2 tau/4) delta_x delta_y (u^1 - u^0)

Both are second order in tau overall (the first step's local error is
O(tau^2)).  With d^n = u^n - u^{n-1}, Delta = u^{n+1} - 2u^n + u^{n-1} and
H_d = I + kappa tau/(2 h^alpha) T(a_0 .. a_{N-1}) the factored form is
    (I + kappa tau/2 delta_x)(I + kappa tau/2 delta_y) Delta
        = tau (-kappa L_h u~ + g(u~) + f^{n+1/2}) - d^n,
    Delta = H_d^-1 B H_d^-1 (x sweep, then y sweep),  u^{n+1} = 2u^n - u^{n-1} + Delta,
and at n = 0  u^1 = u^0 + H_d^-1 [tau (-kappa L_h u^0 + g(u^0) + f^{1/2})] H_d^-1:
the wave step's operators and sweeps with tau in place of tau^2.

Parity: every function is pinned in tests/test_oracle_diffusion.py (the
literal unfactored scheme by dense solves, the closed recursion of a sine
mode at alpha = 2, second-order convergence to the exact semi-discrete
solution exp(-kappa t L_h) phi1, and stability at large tau).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import sadi as S


class Diffusion:
    """The diffusion step's factor H_d of an S-ADI Problem (its grid,
    weights, kappa, tau, g): s_d = kappa tau / (2 h^alpha)."""

    def __init__(self, P: S.Problem):
        self.P = P
        self.s = P.kappa * P.tau / (2.0 * P.h ** P.alpha)
        self.H = np.eye(P.N) + self.s * scipy.linalg.toeplitz(P.a1)
        self._chol = scipy.linalg.cho_factor(self.H, lower=True)

    def solve_x(self, B: np.ndarray) -> np.ndarray:
        """B H_d^-1: H_d w = b on every row (x direction)."""
        return scipy.linalg.cho_solve(self._chol, B.T).T

    def solve_y(self, W: np.ndarray) -> np.ndarray:
        """H_d^-1 W: H_d w = b on every column (y direction)."""
        return scipy.linalg.cho_solve(self._chol, W)


def step(D: Diffusion, u_prev, u_cur, first: bool, f=None, tier="direct"):
    """One diffusion S-ADI step in the factored form (module docstring).
    first=True is the n = 0 step (u_prev ignored); f is f^{n+1/2} or None."""
    P = D.P
    lh = S.lh_direct if tier == "direct" else S.lh_fft
    if first:
        ut = u_cur
        d = np.zeros_like(u_cur)
    else:
        d = u_cur - u_prev
        ut = u_cur + 0.5 * d
    gu = S.g_eval(P.g, ut, P.gc)
    if f is not None:
        gu = gu + f
    B = P.tau * (-P.kappa * lh(P, ut) + gu) - d
    Delta = D.solve_y(D.solve_x(B))
    return u_cur + d + Delta


def run(D: Diffusion, phi1, M: int, tier="direct", forcing=None):
    """u^M after M steps from u^0 = phi1; forcing(n) -> f^{n+1/2} (or None)."""
    up = None
    uc = np.array(phi1, dtype=np.float64)
    for n in range(M):
        fn = forcing(n) if forcing else None
        un = step(D, up, uc, n == 0, fn, tier)
        up, uc = uc, un
    return uc


def step_literal(D: Diffusion, ops, u_prev, u_cur, first: bool, f=None):
    """The unfactored scheme of the module docstring, solved for u^{n+1}
    with one dense N^2 x N^2 solve (tiny N only); ops = sadi.dense_operators(P)."""
    P = D.P
    Dx, Dy, L = ops
    n2 = P.N * P.N
    k, t = P.kappa, P.tau
    R = L - Dx - Dy
    Ssum = Dx + Dy
    DxDy = Dx @ Dy
    un = u_cur.reshape(-1)
    ut = un if first else 1.5 * un - 0.5 * u_prev.reshape(-1)
    gt = S.g_eval(P.g, ut, P.gc) + (0.0 if f is None else f.reshape(-1))
    lhs = np.eye(n2) / t + 0.5 * k * Ssum + 0.25 * k * k * t * DxDy
    r = un / t - 0.5 * k * Ssum @ un - k * R @ ut + gt
    if first:
        r = r + 0.25 * k * k * t * DxDy @ un
    else:
        r = r + 0.25 * k * k * t * DxDy @ (2.0 * un - u_prev.reshape(-1))
    return np.linalg.solve(lhs, r).reshape(P.N, P.N)

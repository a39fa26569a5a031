"""Seeded synthetic inputs for the S-ADI workloads.

This module only builds initial data (phi_1, phi_2) and names workload
parameters; it contains none of the scheme's arithmetic, so both the CUDA-path
tests/bench and the CPU oracle tests may use it.

Grid: N interior points per direction on Omega = (a, b)^2, h = (b - a)/(N + 1),
x_i = a + i h for 1 <= i <= N (the paper's grid, Sec. 2).  Arrays are N x N,
row index = y, column index = x.

Gaussian bumps: A * exp(-|x - c|^2 / (2 w^2)); per bump the draws are, in
order, c_x, c_y ~ U(-0.6, 0.6), w ~ U(0.05, 0.2), A ~ U(-1, 1) from
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 20231206

G_ZERO, G_NEG_CUBE, G_NEG_SIN = 0, 1, 2


def coords(N: int, a: float, b: float):
    h = (b - a) / (N + 1)
    x = a + h * np.arange(1, N + 1, dtype=np.float64)
    return x[None, :], x[:, None]          # X (varies along columns), Y (along rows)


def gaussian_bumps(N: int, nbumps: int, seed: int, a: float = -1.0, b: float = 1.0,
                   centre=0.6, wlo=0.05, whi=0.2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    X, Y = coords(N, a, b)
    u = np.zeros((N, N))
    for _ in range(nbumps):
        cx = rng.uniform(-centre, centre)
        cy = rng.uniform(-centre, centre)
        w = rng.uniform(wlo, whi)
        A = rng.uniform(-1.0, 1.0)
        u += A * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * w * w))
    return u


def gaussian(N: int, beta: float, a: float = -1.0, b: float = 1.0) -> np.ndarray:
    X, Y = coords(N, a, b)
    return np.exp(-beta * (X * X + Y * Y))


def random_field(N: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """i.i.d. U(-scale, scale) values (stress inputs for parity tests)."""
    return np.random.default_rng(seed).uniform(-scale, scale, size=(N, N))


@dataclass
class Workload:
    name: str
    N: int
    alpha: float
    kappa: float
    tau: float
    steps: int
    g: int
    phi1: np.ndarray
    phi2: np.ndarray
    a: float = -1.0
    b: float = 1.0


def small_fp64(N: int = 63) -> Workload:
    """N=63, Omega=(-1,1)^2, alpha=1.5, kappa=1, tau=1/64, 64 steps, g=-u^3,
    phi1=exp(-20(x^2+y^2)), phi2=0 (single instance, FP64)."""
    p1 = gaussian(N, 20.0)
    return Workload("sadi-N63-a1.5-fp64", N, 1.5, 1.0, 1.0 / 64.0, 64, G_NEG_CUBE,
                    p1, np.zeros_like(p1))


def bumps_1023(alpha: float, N: int = 1023, steps: int = 1000) -> Workload:
    """N=1023, alpha in {1.2, 1.5, 1.8}, kappa=1, tau=1e-3, 1000 steps,
    g=-sin u, phi1 = 8 seeded Gaussian bumps, phi2 = 0."""
    p1 = gaussian_bumps(N, 8, SEED_BASE + 2)
    return Workload(f"sadi-N{N}-a{alpha}-bumps8", N, alpha, 1.0, 1e-3, steps, G_NEG_SIN,
                    p1, np.zeros_like(p1))


def paper_example1(N: int, alpha: float, tau: float, t_end: float = 5.0) -> Workload:
    """Sec. 6 Example 1 (sine-Gordon): Omega=(-10,10)^2, phi1=0,
    phi2=sech(sqrt(x^2+y^2)), g=-sin u, kappa=1, t=5."""
    X, Y = coords(N, -10.0, 10.0)
    p2 = 1.0 / np.cosh(np.sqrt(X * X + Y * Y))
    M = int(round(t_end / tau))
    return Workload(f"paper-ex1-N{N}-a{alpha}", N, alpha, 1.0, tau, M, G_NEG_SIN,
                    np.zeros((N, N)), p2, -10.0, 10.0)


def paper_example2(N: int, alpha: float, tau: float, t_end: float = 8.0,
                   amp: float = 2.0) -> Workload:
    """Sec. 6 Example 2 (Klein-Gordon): Omega=(-10,10)^2,
    phi1 = amp * sech(cosh(x^2+y^2)), phi2=0, g=-u^3, kappa=1, t=8.

    The paper prints phi1 = sech(cosh(x^2+y^2)); its Table 4 errors are
    reproduced only with amp = 2 (the printed formula drops the factor 2), so
    amp = 2 is the default."""
    X, Y = coords(N, -10.0, 10.0)
    with np.errstate(over="ignore"):
        p1 = amp / np.cosh(np.cosh(X * X + Y * Y))
    M = int(round(t_end / tau))
    return Workload(f"paper-ex2-N{N}-a{alpha}", N, alpha, 1.0, tau, M, G_NEG_CUBE,
                    p1, np.zeros((N, N)), -10.0, 10.0)

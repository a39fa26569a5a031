"""S-ADI scheme oracle (FP64 CPU, test infrastructure only).

Notation follows the paper: N interior points per direction, h = (b-a)/(N+1),
grid points x_i = a + i h (1 <= i <= N); a grid function is an N x N array
``u[j, i]`` with j the y index (row) and i the x index (contiguous).

Operators (Sec. 2):
  L_h^alpha v = h^-alpha sum_{i,j} a_ij v(x+ih, y+jh)        eq. "center discretization"
  delta_x v   = h^-alpha sum_i a_i v(x+ih, y)                  eq. "single discrete Riesz"
  delta_y v   = h^-alpha sum_i a_i v(x, y+ih)
with v = 0 outside the N x N interior (u = 0 on the complement of Omega).

Scheme (Sec. 3, eq. "ADI scheme equivalent"):
  (1 + tau^2 kappa/2 delta_x)(1 + tau^2 kappa/2 delta_y) uhat^n = B^n,
  uhat^n = u^{n+1} - 2u^n + u^{n-1} (n >= 1),  u^1 - u^0 (n = 0),
  B^n = -tau^2 kappa L_h u^n + tau^2 g(u^n)                              (n >= 1)
  B^0 = tau phi_2 - tau^2/2 kappa L_h u^0 + tau^2/2 g(u^0)               (n = 0)
In matrix form (Sec. 3) uhat = H^-1 B H^-1 with H = I + tau^2 kappa/2 A_x.  The
matrix A_x printed there omits the factor h^-alpha that delta_x carries; we
read H = I + kappa tau^2 / (2 h^alpha) T(a_0 .. a_{N-1}).

Two tiers (both plain FP64):
  * "direct": L_h by the direct O(N^4) block-Toeplitz sum, the two sweeps by
    dense Cholesky solves (the definition).
  * "fft":    L_h by zero-padded 2D FFT convolution (the BTTB-in-BCCB embedding
    of Sec. 3), sweeps by dense Cholesky (same definition); used for the large
    sizes and as the timed CPU baseline.  Pinned to "direct".
The literal three-level scheme (eqs. "ADI scheme", "ADI scheme initial") is
also here, for tiny N, to pin the factored form against the paper's own
statement.

Parity: every function is pinned in tests/test_oracle_sadi.py; none is
"parity unpinned".
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.fft
import scipy.linalg

from . import weights as W

G_ZERO, G_NEG_CUBE, G_NEG_SIN, G_GENERAL = 0, 1, 2, 3


def g_eval(kind: int, u: np.ndarray, coef=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Nonlinearity g(u) of the problem statement (Sec. 1): 0, -u^3
    (Klein-Gordon, Sec. 6 Ex. 2), -sin u (sine-Gordon, Ex. 1), or the general
    form c1 u + c3 u^3 + cs sin u with coef = (c1, c3, cs)."""
    if kind == G_ZERO:
        return np.zeros_like(u)
    if kind == G_NEG_CUBE:
        return -u * u * u
    if kind == G_NEG_SIN:
        return -np.sin(u)
    if kind == G_GENERAL:
        c1, c3, cs = coef
        return c1 * u + c3 * (u * u * u) + cs * np.sin(u)
    raise ValueError(f"unknown g kind {kind}")


def grid(N: int, a: float, b: float):
    """h = (b - a)/(N + 1) and the interior coordinates x_1..x_N (Sec. 2)."""
    h = (b - a) / (N + 1)
    x = a + h * np.arange(1, N + 1)
    return h, x


@dataclass
class Problem:
    """One S-ADI instance: sizes, parameters and the FP64 weights."""
    N: int
    alpha: float
    kappa: float
    tau: float
    a: float = -1.0
    b: float = 1.0
    g: int = G_ZERO
    A2: np.ndarray | None = field(default=None, repr=False)   # a_ij, 0<=i,j<N
    a1: np.ndarray | None = field(default=None, repr=False)   # a_i, 0<=i<N
    fft_size: int | None = None      # circulant size Q >= 2N - 1 of the fft tier (default 2N)
    fft_workers: int | None = None   # threads of its transforms (default 1)
    gc: tuple = (0.0, 0.0, 0.0)      # coefficients of the general g (kind 3)

    def __post_init__(self):
        self.h, self.x = grid(self.N, self.a, self.b)
        if self.a1 is None:
            self.a1 = W.riesz_1d(self.alpha, self.N)
        if self.A2 is None:
            if self.alpha == 2.0:
                A2 = np.zeros((self.N, self.N))
                A2[0, 0] = 4.0
                if self.N > 1:
                    A2[1, 0] = A2[0, 1] = -1.0
                self.A2 = A2
            else:
                self.A2 = W.lap2d_trap(self.alpha, self.N)
        self.s = self.kappa * self.tau ** 2 / (2.0 * self.h ** self.alpha)
        self.H = np.eye(self.N) + self.s * scipy.linalg.toeplitz(self.a1)
        self._chol = scipy.linalg.cho_factor(self.H, lower=True)


# ----------------------------------------------------------------------------
# The discrete fractional Laplacian L_h (Sec. 2, eq. "center discretization")
# ----------------------------------------------------------------------------

def lh_direct(P: Problem, u: np.ndarray) -> np.ndarray:
    """(L_h u)[q, p] = h^-alpha sum_{q', p'} a_{|p-p'|, |q-q'|} u[q', p'].

    The direct block-Toeplitz product: for each y offset d the Toeplitz matrix
    T_d = [a_{|p-p'|, d}]_{p,p'} acts on every row, and row q collects the
    rows q +- d.  O(N^4) flops, no FFT.
    """
    N = P.N
    out = np.zeros((N, N))
    for d in range(N):
        Td = scipy.linalg.toeplitz(P.A2[:, d])      # symmetric: a_{|p-p'|, d}
        Y = u @ Td                                  # Y[q', p] = sum_p' u[q', p'] a_{|p-p'|,d}
        if d == 0:
            out += Y
        else:
            out[d:, :] += Y[:-d, :]                 # q' = q - d
            out[:-d, :] += Y[d:, :]                 # q' = q + d
    return out / P.h ** P.alpha


def lh_fft(P: Problem, u: np.ndarray) -> np.ndarray:
    """L_h u by embedding the block-Toeplitz-Toeplitz-block matrix into a block
    circulant one of size Q x Q (Q >= 2N - 1) and multiplying with 2D FFTs
    (Sec. 3): the wrapped kernel holds a_{|i|,|j|} at (i mod Q, j mod Q) for
    |i|, |j| <= N - 1 and zero elsewhere.  Any Q >= 2N - 1 gives the same
    product (no wrapped term reaches the kept N x N block); Q = P.fft_size,
    default 2N.  The kernel's transform is computed once per Problem and Q."""
    N = P.N
    Q = P.fft_size or 2 * N
    if Q < 2 * N - 1:
        raise ValueError(f"circulant size {Q} < 2N - 1 = {2 * N - 1}")
    cache = P.__dict__.setdefault("_khat", {})
    if Q not in cache:
        dist = np.minimum(np.arange(Q), Q - np.arange(Q))     # |i| of the wrapped index
        ok = dist <= N - 1
        dc = np.minimum(dist, N - 1)
        K = np.where(ok[:, None] & ok[None, :], P.A2[dc[:, None], dc[None, :]], 0.0)
        cache[Q] = scipy.fft.rfft2(K, workers=P.fft_workers)
        del K
    U = np.zeros((Q, Q))
    U[:N, :N] = u
    conv = scipy.fft.irfft2(cache[Q] * scipy.fft.rfft2(U, workers=P.fft_workers), s=(Q, Q),
                            workers=P.fft_workers)
    return conv[:N, :N] / P.h ** P.alpha


def riesz_x(P: Problem, u: np.ndarray) -> np.ndarray:
    """delta_x u: h^-alpha T(a) acting along x (the contiguous index)."""
    return u @ scipy.linalg.toeplitz(P.a1) / P.h ** P.alpha


def riesz_y(P: Problem, u: np.ndarray) -> np.ndarray:
    """delta_y u: h^-alpha T(a) acting along y (the row index)."""
    return scipy.linalg.toeplitz(P.a1) @ u / P.h ** P.alpha


# ----------------------------------------------------------------------------
# The two sweeps (Sec. 3: uhat = H^-1 B H^-1)
# ----------------------------------------------------------------------------

def solve_x(P: Problem, B: np.ndarray) -> np.ndarray:
    """W = B H^-1: H w = b on every row (x direction); dense Cholesky."""
    return scipy.linalg.cho_solve(P._chol, B.T).T


def solve_y(P: Problem, W_: np.ndarray) -> np.ndarray:
    """H^-1 W: H w = b on every column (y direction); dense Cholesky."""
    return scipy.linalg.cho_solve(P._chol, W_)


# ----------------------------------------------------------------------------
# The S-ADI step (Sec. 3, factored increment form)
# ----------------------------------------------------------------------------

def rhs(P: Problem, u: np.ndarray, Lu: np.ndarray, first: bool, phi2=None, f=None) -> np.ndarray:
    """B^n of eq. "ADI scheme equivalent" (optionally with a source f^n added
    to g, for the manufactured-solution tests)."""
    gu = g_eval(P.g, u, P.gc)
    if f is not None:
        gu = gu + f
    if first:
        return P.tau * phi2 + 0.5 * P.tau ** 2 * (-P.kappa * Lu + gu)
    return P.tau ** 2 * (-P.kappa * Lu + gu)


def step(P: Problem, u_prev, u_cur, first: bool, phi2=None, f=None, tier="direct"):
    """One S-ADI step.  first=True is the n = 0 formula (u_prev ignored):
    returns u^1 = u^0 + uhat^0; otherwise u^{n+1} = 2u^n - u^{n-1} + uhat^n."""
    Lu = lh_direct(P, u_cur) if tier == "direct" else lh_fft(P, u_cur)
    B = rhs(P, u_cur, Lu, first, phi2, f)
    uhat = solve_y(P, solve_x(P, B))
    if first:
        return u_cur + uhat
    return 2.0 * u_cur - u_prev + uhat


def run(P: Problem, phi1, phi2, M: int, tier="direct", forcing=None, keep=False):
    """u^M after M steps from u^0 = phi1, d_t u^0 = phi2 (M = 0 returns phi1).
    forcing(n) -> f^n (or None).  keep=True also returns the list u^0..u^M."""
    u0 = np.array(phi1, dtype=np.float64)
    hist = [u0]
    if M == 0:
        return (u0, hist) if keep else u0
    f0 = forcing(0) if forcing else None
    u1 = step(P, None, u0, True, np.asarray(phi2, dtype=np.float64), f0, tier)
    hist.append(u1)
    up, uc = u0, u1
    for n in range(1, M):
        fn = forcing(n) if forcing else None
        un = step(P, up, uc, False, None, fn, tier)
        up, uc = uc, un
        if keep:
            hist.append(uc)
    return (uc, hist) if keep else uc


# ----------------------------------------------------------------------------
# The literal three-level scheme (Sec. 2), tiny N only: pins the factored form
# ----------------------------------------------------------------------------

def dense_operators(P: Problem):
    """N^2 x N^2 matrices of delta_x, delta_y and L_h acting on vec(u) with
    vec(u)[j*N + i] = u[j, i].  L_h is assembled entry by entry from its
    defining sum (no Toeplitz helper), so it also pins lh_direct."""
    N = P.N
    I = np.eye(N)
    T = scipy.linalg.toeplitz(P.a1)
    Dx = np.kron(I, T) / P.h ** P.alpha
    Dy = np.kron(T, I) / P.h ** P.alpha
    L = np.zeros((N * N, N * N))
    for j in range(N):
        for i in range(N):
            for jj in range(N):
                for ii in range(N):
                    L[j * N + i, jj * N + ii] = P.A2[abs(i - ii), abs(j - jj)]
    L /= P.h ** P.alpha
    return Dx, Dy, L


def step_literal(P: Problem, ops, u_prev, u_cur, first: bool, phi2=None):
    """Solve eq. "ADI scheme" (n >= 1) or eq. "ADI scheme initial" (n = 0) as
    printed, for u^{n+1}, with one dense N^2 x N^2 solve."""
    Dx, Dy, L = ops
    N2 = P.N * P.N
    I = np.eye(N2)
    k, t = P.kappa, P.tau
    un = u_cur.reshape(-1)
    gn = g_eval(P.g, un, P.gc)
    R = L - Dx - Dy                                  # the explicit remainder
    S = Dx + Dy
    DxDy = Dx @ Dy
    if first:
        # (u1 - u0 - t phi2)/(t^2/2) = -k S u1 - k^2 t^2/2 DxDy (u1 - u0) - k R u0 + g(u0)
        lhs = 2.0 / t ** 2 * I + k * S + 0.5 * k ** 2 * t ** 2 * DxDy
        r = (2.0 / t ** 2) * (un + t * phi2.reshape(-1)) + 0.5 * k ** 2 * t ** 2 * DxDy @ un \
            - k * R @ un + gn
    else:
        um = u_prev.reshape(-1)
        # (u+ - 2u + u-)/t^2 = -k S (u+ + u-)/2 - k^2 t^2/4 DxDy (u+ - 2u + u-) - k R u + g(u)
        lhs = I / t ** 2 + 0.5 * k * S + 0.25 * k ** 2 * t ** 2 * DxDy
        r = (2.0 * un - um) / t ** 2 - 0.5 * k * S @ um \
            + 0.25 * k ** 2 * t ** 2 * DxDy @ (2.0 * un - um) - k * R @ un + gn
    return np.linalg.solve(lhs, r).reshape(P.N, P.N)


# ----------------------------------------------------------------------------
# Gohberg-Semencul (Proposition 1, Algorithm 1)
# ----------------------------------------------------------------------------

def gs_generator(H: np.ndarray) -> np.ndarray:
    """c = H^-1 e_1 (the paper uses PCG; any exact solver gives the same c).
    Levinson recursion via scipy.linalg.solve_toeplitz."""
    e1 = np.zeros(H.shape[0])
    e1[0] = 1.0
    return scipy.linalg.solve_toeplitz(H[:, 0], e1)


def gs_solve(c: np.ndarray, v: np.ndarray) -> np.ndarray:
    """H^-1 v by Algorithm 1 (Proposition 1 with the circulant/skew-circulant
    diagonalisations of Sec. 3), numpy fft/ifft conventions (ifft carries 1/N),
    Q = diag(exp(-i pi k / N)).  v may be a 1D vector or a stack of rows."""
    N = c.shape[0]
    p1 = c[0]
    s = np.concatenate(([c[0]], -c[:0:-1]))        # [p1, -p_N, ..., -p_2]
    k = np.arange(N)
    q = np.exp(-1j * np.pi * k / N)
    lam_c = np.fft.fft(c)
    lam_s = np.fft.fft(q * s)
    v = np.asarray(v, dtype=np.float64)
    v1 = (v + 1j * v[..., ::-1]) / (2.0 * p1)
    v2 = np.conj(q) * np.fft.ifft(lam_s * np.fft.fft(q * v1, axis=-1), axis=-1)
    v3 = np.fft.ifft(lam_c * np.fft.fft(v2, axis=-1), axis=-1)
    return v3.real + v3.imag[..., ::-1]


# ----------------------------------------------------------------------------
# Discrete energy (Sec. 4, stability theorem) and error estimators (Sec. 6)
# ----------------------------------------------------------------------------

def energy(P: Problem, u_n: np.ndarray, u_np1: np.ndarray, tier="direct") -> float:
    """H_n of the stability proof, evaluated on the numerical solution itself:
    H_n^2 = ||d||^2 + tau^2 kappa/2 (||d||_At^2 - ||d||_A^2)
            + kappa/2 (||u^{n+1}||_A^2 + ||u^n||_A^2) + kappa^2 tau^4/4 ||d||_B^2,
    d = (u^{n+1} - u^n)/tau, <v, w> = h^2 sum v w, ||w||_A^2 = <L_h w, w>,
    ||w||_At^2 = <(delta_x + delta_y) w, w>, ||w||_B^2 = <delta_x delta_y w, w>.
    With g = 0 it is constant in n (the identity (H_n^2 - H_{n-1}^2)/tau = I_2 = 0)."""
    h2 = P.h ** 2
    lh = lh_direct if tier == "direct" else lh_fft

    def ip(v, w):
        return h2 * float(np.sum(v * w))
    d = (u_np1 - u_n) / P.tau
    nA = lambda w: ip(lh(P, w), w)
    nAt = lambda w: ip(riesz_x(P, w) + riesz_y(P, w), w)
    nB = lambda w: ip(riesz_x(P, riesz_y(P, w)), w)
    k, t = P.kappa, P.tau
    H2 = ip(d, d) + 0.5 * t * t * k * (nAt(d) - nA(d)) + 0.5 * k * (nA(u_np1) + nA(u_n)) \
        + 0.25 * k * k * t ** 4 * nB(d)
    return float(np.sqrt(H2))


def error1(h: float, u_tau: np.ndarray, u_tau_half: np.ndarray) -> float:
    """Error_1 of Sec. 6: sqrt(h^2 sum |u^M(tau,h) - u^{2M}(tau/2,h)|^2)."""
    return float(np.sqrt(h * h * np.sum((u_tau - u_tau_half) ** 2)))


def error2(h: float, u_h: np.ndarray, u_h_half: np.ndarray) -> float:
    """Error_2 of Sec. 6: sqrt(h^2 sum |u_ij(tau,h) - u_{2i,2j}(tau,h/2)|^2);
    fine point 2i (1-based) is fine array index 2i - 1."""
    fine = u_h_half[1::2, 1::2]
    assert fine.shape == u_h.shape
    return float(np.sqrt(h * h * np.sum((u_h - fine) ** 2)))


def rel_l2(u: np.ndarray, ref: np.ndarray) -> float:
    """||u - ref||_2 / ||ref||_2 over the N^2 grid."""
    return float(np.linalg.norm(u - ref) / np.linalg.norm(ref))

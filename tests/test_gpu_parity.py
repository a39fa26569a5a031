"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 path <= 1e-10 relative L2 (element-wise 1e-10 of the max for
setup tables); FP32 path <= 1e-5 relative L2.  Inputs are seeded and
synthetic (workloads.py)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import sadi as O
from oracle import weights as OW
from paper_2312_06206_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_06206_gb300 import build
    build.build()
    from paper_2312_06206_gb300 import sadi
    return sadi


def _run_gpu(S, N, alpha, kappa, tau, g, phi1, phi2, steps, prec, dom=(-1.0, 1.0)):
    with S.Sadi(N, alpha, kappa, tau, dom) as s:
        s.set_options(g, prec)
        s.set_initial(phi1, phi2)
        s.step(steps)
        u, n = s.get()
    assert n == steps
    return u


# ------------------------------------------------------------- setup -------

@pytest.mark.parametrize("N,alpha", [(1, 1.5), (7, 1.3), (63, 1.5), (100, 1.8), (255, 1.2)])
def test_setup_tables_match_oracle(S, N, alpha):
    tau, kappa = 0.01, 1.0
    with S.Sadi(N, alpha, kappa, tau) as s:
        Np, r = s.sadi_get_info()
        a1 = s.sadi_get_setup(0)
        a2 = s.sadi_get_setup(1)
        c = s.sadi_get_setup(2)
        lam = s.sadi_get_setup(3)
    assert Np >= max(N, 8) and Np & (Np - 1) == 0 and r == Np - N
    ref1 = OW.riesz_1d(alpha, N)
    assert np.abs(a1 - ref1).max() <= 1e-13 * np.abs(ref1).max()
    ref2 = OW.lap2d_trap(alpha, N, OW.trap_grid_size(N))
    assert np.abs(a2 - ref2).max() <= 1e-13 * np.abs(ref2).max()
    # generator of the bordered matrix H' = I + s T(a_0..a_{Np-1})
    h = 2.0 / (N + 1)
    s_ = kappa * tau ** 2 / (2 * h ** alpha)
    Hp = np.eye(Np) + s_ * scipy.linalg.toeplitz(OW.riesz_1d(alpha, Np))
    cref = np.linalg.solve(Hp, np.eye(Np)[:, 0])
    assert np.abs(c - cref).max() <= 1e-13 * np.abs(cref).max()
    # symbol of the 2Np x 2Np block-circulant embedding
    P = 2 * Np
    dist = np.minimum(np.arange(P), P - np.arange(P))
    ok = dist <= N - 1
    dc = np.minimum(dist, N - 1)
    K = np.where(ok[:, None] & ok[None, :], ref2[dc[:, None], dc[None, :]], 0.0)
    Lref = np.fft.fft2(K).real[:Np + 1, :Np + 1]
    assert np.abs(lam - Lref).max() <= 1e-12 * np.abs(Lref).max()


# -------------------------------------------------------------- steps -------

def test_config_small_fp64_full_run(S):
    # N=63, alpha=1.5, kappa=1, tau=1/64, 64 steps, g=-u^3, phi1=exp(-20 r^2)
    w = WL.small_fp64(63)
    P = O.Problem(w.N, w.alpha, w.kappa, w.tau, w.a, w.b, w.g)
    ref = O.run(P, w.phi1, w.phi2, w.steps, tier="direct")
    u = _run_gpu(S, w.N, w.alpha, w.kappa, w.tau, w.g, w.phi1, w.phi2, w.steps, S.SADI_PREC_FP64)
    assert O.rel_l2(u, ref) <= 1e-10


@pytest.mark.parametrize("N,alpha,g", [(1, 1.5, 1), (2, 1.3, 2), (3, 1.9, 1), (5, 1.5, 0), (7, 1.1, 2),
                                       (8, 1.6, 1), (9, 1.4, 2), (16, 1.5, 1), (31, 1.7, 2), (33, 1.2, 1),
                                       (64, 1.5, 2), (100, 1.8, 1), (2, 2.0, 0), (15, 2.0, 1)])
def test_fp64_step_parity_ragged_sizes(S, N, alpha, g):
    kappa, tau = 0.9, 0.05
    phi1 = WL.random_field(N, 11 + N)
    phi2 = 0.5 * WL.random_field(N, 97 + N)
    steps = 3
    P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, g)
    ref = O.run(P, phi1, phi2, steps, tier="direct")
    u = _run_gpu(S, N, alpha, kappa, tau, g, phi1, phi2, steps, S.SADI_PREC_FP64)
    assert O.rel_l2(u, ref) <= 1e-10, O.rel_l2(u, ref)
    # element-wise as well
    assert np.abs(u - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("N,alpha,g", [(63, 1.5, 1), (64, 1.4, 0), (100, 1.3, 2), (128, 1.6, 1), (255, 1.8, 2)])
def test_fp32_step_parity(S, N, alpha, g):
    kappa, tau = 1.0, 0.02
    phi1 = WL.gaussian_bumps(N, 8, 5 + N)
    phi2 = 0.2 * WL.gaussian(N, 10.0)
    steps = 10
    P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, g)
    ref = O.run(P, phi1, phi2, steps, tier="fft")
    u = _run_gpu(S, N, alpha, kappa, tau, g, phi1, phi2, steps, S.SADI_PREC_FP32)
    assert O.rel_l2(u, ref) <= 1e-5, O.rel_l2(u, ref)
    assert np.abs(u - ref).max() <= 1e-5 * np.abs(ref).max()   # element-wise too


def test_full_size_1023_fp64_and_fp32(S):
    # N=1023, alpha=1.5, kappa=1, tau=1e-3, g=-sin u, 8 seeded bumps: a few
    # steps against the oracle (FFT tier, itself pinned to the direct tier)
    w = WL.bumps_1023(1.5, steps=4)
    P = O.Problem(w.N, w.alpha, w.kappa, w.tau, w.a, w.b, w.g)
    ref = O.run(P, w.phi1, w.phi2, w.steps, tier="fft")
    u64 = _run_gpu(S, w.N, w.alpha, w.kappa, w.tau, w.g, w.phi1, w.phi2, w.steps, S.SADI_PREC_FP64)
    assert O.rel_l2(u64, ref) <= 1e-10, O.rel_l2(u64, ref)
    u32 = _run_gpu(S, w.N, w.alpha, w.kappa, w.tau, w.g, w.phi1, w.phi2, w.steps, S.SADI_PREC_FP32)
    assert O.rel_l2(u32, ref) <= 1e-5, O.rel_l2(u32, ref)
    assert np.abs(u32 - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.abs(u64 - ref).max() <= 1e-10 * np.abs(ref).max()


def test_rerun_is_bitwise_identical_and_symmetric(S):
    N = 63
    phi1 = WL.gaussian(N, 12.0)            # symmetric under x <-> y
    us = [_run_gpu(S, N, 1.6, 1.0, 0.03, 2, phi1, None, 8, S.SADI_PREC_FP64) for _ in range(2)]
    assert np.array_equal(us[0], us[1])
    assert np.abs(us[0] - us[0].T).max() <= 1e-13 * np.abs(us[0]).max()


def test_state_errors(S):
    with S.Sadi(15, 1.5, 1.0, 0.1) as s:
        with pytest.raises(S.SadiError) as ei:
            s.step(1)
        assert ei.value.status == S.SADI_ESTATE
        with pytest.raises(S.SadiError) as ei:
            s.set_options(7, 0)
        assert ei.value.status == S.SADI_EINVAL
        s.set_initial(np.zeros((15, 15)))
        with pytest.raises(S.SadiError) as ei:
            s.set_options(0, 1)
        assert ei.value.status == S.SADI_ESTATE
        with pytest.raises(S.SadiError):
            s.step(-1)
        s.step(0)
        u, n = s.get()
        assert n == 0 and not u.any()


def test_batch_step_matches_single_contexts(S):
    # FP32 contexts of equal FFT length (N = 63, 50, 33 -> N' = 64) go through
    # one batched launch per kernel; an FP64 context steps on its own.  The
    # batch must reproduce single-context stepping bitwise.
    specs = [(63, 1.5, 1.0, 0.02, 1, 1), (50, 1.2, 0.7, 0.03, 2, 1), (33, 1.8, 1.3, 0.01, 0, 1),
             (40, 1.6, 1.0, 0.02, 1, 0)]

    def make():
        out = []
        for k, (N, al, ka, ta, g, prec) in enumerate(specs):
            s = S.Sadi(N, al, ka, ta)
            s.set_options(g, prec)
            s.set_initial(WL.gaussian_bumps(N, 4, 300 + k), 0.3 * WL.random_field(N, 400 + k))
            out.append(s)
        return out
    single = make()
    for s in single:
        s.step(6)
    ref = [s.get()[0] for s in single]
    batch = make()
    S.sadi_batch_step(batch, 6)
    for s, r in zip(batch, ref):
        u, n = s.get()
        assert n == 6 and np.array_equal(u, r)
    for s in single + batch:
        s.close()


def test_dense_batch_over_two_gemm_launches_matches_single_contexts(S):
    # ten dense-form contexts of one FFT length (N' = 64): the B^n kernel of
    # the batch zeroes every member's GEMM counters, the first sweep GEMM
    # (eight members) runs as its programmatic dependent, the second (two
    # members) after it; stepped directly and by graph replay, the batch must
    # reproduce single-context stepping bitwise
    specs = [(40 + 2 * k, 1.2 + 0.06 * k, 1.0, 0.02, k % 3) for k in range(10)]

    import torch
    st = torch.cuda.Stream()

    def make():
        out = []
        for k, (N, al, ka, ta, g) in enumerate(specs):
            s = S.Sadi(N, al, ka, ta)
            s.set_options(g, S.SADI_PREC_FP32_DENSE)
            s.set_stream(st.cuda_stream)                  # a graph needs one stream
            s.set_initial(WL.gaussian_bumps(N, 4, 500 + k), 0.3 * WL.random_field(N, 600 + k))
            out.append(s)
        return out
    single = make()
    for s in single:
        s.step(5)
    ref = [s.get()[0] for s in single]
    batch = make()
    S.sadi_batch_step(batch, 5)
    for s, r in zip(batch, ref):
        u, n = s.get()
        assert n == 5 and np.array_equal(u, r)
    replay = make()
    S.sadi_batch_step(replay, 1)
    g = S.SadiGraph(replay, 1)
    g.launch(4)
    g.close()
    for s, r in zip(replay, ref):
        u, n = s.get()
        assert n == 5 and np.array_equal(u, r)
    for s in single + batch + replay:
        s.close()


@pytest.mark.parametrize("engine", ["register", "shared"])
def test_dense_batch_at_2048_matches_single_contexts(S, engine):
    # dense-form contexts of FFT length 2048: on the register path (the
    # default) one launch per FFT kernel covers all of them; with explicit
    # tiles they stay on the shared-memory engine, whose FFT kernels run one
    # context after another.  Both sweeps of all of them in one GEMM launch;
    # bitwise equal to single-context stepping either way.
    specs = [(1500, 1.4, 1.0, 1e-3, 1), (1100, 1.7, 0.8, 1e-3, 2), (2047, 1.2, 1.2, 5e-4, 0)]

    def make():
        out = []
        for k, (N, al, ka, ta, g) in enumerate(specs):
            s = S.Sadi(N, al, ka, ta)
            s.set_options(g, S.SADI_PREC_FP32_DENSE)
            if engine == "shared":
                s.sadi_set_tiles(*s.sadi_get_tiles())
            s.set_initial(WL.gaussian_bumps(N, 4, 700 + k))
            out.append(s)
        return out
    single = make()
    for s in single:
        s.step(3)
    ref = [s.get()[0] for s in single]
    batch = make()
    S.sadi_batch_step(batch, 3)
    for s, r in zip(batch, ref):
        u, n = s.get()
        assert n == 3 and np.array_equal(u, r)
    for s in single + batch:
        s.close()


def test_batch_step_rejects_bad_batches(S):
    a = S.Sadi(31, 1.5, 1.0, 0.1)
    b = S.Sadi(31, 1.5, 1.0, 0.1)
    a.set_initial(np.zeros((31, 31)))
    with pytest.raises(S.SadiError):
        S.sadi_batch_step([a, a], 1)          # duplicate
    with pytest.raises(S.SadiError):
        S.sadi_batch_step([a, b], 1)          # b not initialised
    a.close()
    b.close()


@pytest.mark.parametrize("alpha,ref", [(1.1, 6.3150e-02), (1.5, 8.1276e-02), (1.9, 1.0716e-01)])
def test_paper_table2_through_the_c_abi(S, alpha, ref):
    # Sec. 6 Table 2 (Example 1, sine-Gordon, S-ADI): h = 1 (N = 19) against
    # h = 1/2 (N = 39), tau = 1/100, t = 5, on Omega = (-10, 10)^2, FP64 path.
    # N' = 32 and 64: border ranks r = 13 and 25 exercise the rank-r correction.
    us = []
    for N in (19, 39):
        w = WL.paper_example1(N, alpha, 1 / 100)
        us.append(_run_gpu(S, N, alpha, w.kappa, w.tau, w.g, w.phi1, w.phi2, w.steps, S.SADI_PREC_FP64,
                           dom=(w.a, w.b)))
    e = O.error2(1.0, us[0], us[1])
    assert abs(e - ref) <= 0.5 * 10 ** (np.floor(np.log10(ref)) - 4), (e, ref)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_source_term_parity(S, prec, tol):
    # f^n = cos(omega t_n + phase) F enters B^n like g(u^n) (oracle `forcing`)
    N, alpha, kappa, tau, g = 31, 1.4, 0.8, 0.04, 2
    F = WL.random_field(N, 77)
    om, ph = 2.3, 0.4
    phi1 = WL.gaussian_bumps(N, 3, 78)
    phi2 = 0.2 * WL.random_field(N, 79)
    P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, g)
    ref = O.run(P, phi1, phi2, 7, tier="direct", forcing=lambda n: np.cos(om * n * tau + ph) * F)
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(g, prec)
        s.sadi_set_source(F, om, ph)
        s.set_initial(phi1, phi2)
        s.step(7)
        u, _ = s.get()
    assert O.rel_l2(u, ref) <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_manufactured_solution_second_order_on_gpu(S, prec):
    # U(t) = cos(t) phi solves u_tt = -kappa L_h u + f with g = 0 and
    # f = cos(t) (kappa L_h phi - phi); the S-ADI step must converge to it at
    # O(tau^2) (Sec. 5 convergence theorem).
    N, alpha, kappa = 63, 1.5, 1.0
    phi = WL.gaussian(N, 8.0)
    errs = []
    for M in (8, 16, 32):
        tau = 1.0 / M
        P = O.Problem(N, alpha, kappa, tau)
        F = kappa * O.lh_direct(P, phi) - phi
        with S.Sadi(N, alpha, kappa, tau) as s:
            s.set_options(0, prec)
            s.sadi_set_source(F, 1.0, 0.0)
            s.set_initial(phi, None)
            s.step(M)
            u, _ = s.get()
        errs.append(np.abs(u - np.cos(1.0) * phi).max())
    orders = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.9 < o < 2.15 for o in orders), (orders, errs)


@pytest.mark.parametrize("N,alpha,g,steps", [(2047, 1.4, 1, 5), (4095, 1.7, 1, 3)])
def test_large_n_fp32_against_fp64(S, N, alpha, g, steps):
    # N' = 2048 (the GS form) and 4096 run on the shared-memory FFT engine;
    # the FP64 path is itself checked against the oracle at N = 2047 (2 steps).
    tau, kappa = 5e-4, 0.5
    phi1 = WL.gaussian_bumps(N, 8, 2000 + N)
    u64 = _run_gpu(S, N, alpha, kappa, tau, g, phi1, None, steps, S.SADI_PREC_FP64)
    u32 = _run_gpu(S, N, alpha, kappa, tau, g, phi1, None, steps, S.SADI_PREC_FP32)
    assert O.rel_l2(u32, u64) <= 1e-5, O.rel_l2(u32, u64)
    if N == 2047:
        P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, g)
        ref = O.run(P, phi1, np.zeros_like(phi1), 2, tier="fft")
        u2 = _run_gpu(S, N, alpha, kappa, tau, g, phi1, None, 2, S.SADI_PREC_FP64)
        assert O.rel_l2(u2, ref) <= 1e-10, O.rel_l2(u2, ref)


@pytest.mark.parametrize("N,alpha,g,steps", [(2047, 1.4, 1, 5), (4095, 1.7, 2, 3)])
@pytest.mark.parametrize("prec_name", ["SADI_PREC_FP32", "SADI_PREC_FP32_DENSE"])
def test_three_pass_convolution_against_fp64(S, N, alpha, g, steps, prec_name):
    # conv_cols = -1: the column convolution as three passes of a four-step
    # FFT (64-point transforms over strided rows, R1 = 32 at N' = 2048 and 64
    # at N' = 4096; R1 = 128 at N' = 8192 is the default there and covered by
    # the full-size tests), against the FP64 path with the FP32 forms'
    # tolerance and against the single-pass kernel (rounding only)
    prec = getattr(S, prec_name)
    tau, kappa = 5e-4, 0.5
    phi1 = WL.gaussian_bumps(N, 8, 2100 + N)
    phi2 = 0.1 * WL.gaussian_bumps(N, 3, 2200 + N)
    u64 = _run_gpu(S, N, alpha, kappa, tau, g, phi1, phi2, steps, S.SADI_PREC_FP64)
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(g, prec)
        t = s.sadi_get_tiles()
        s.sadi_set_tiles(t[0], -1, t[2])
        assert s.sadi_get_tiles()[1] == -1
        s.set_initial(phi1, phi2)
        s.step(steps)
        u3, _ = s.get()
    assert O.rel_l2(u3, u64) <= 1e-5, O.rel_l2(u3, u64)
    u1 = _run_gpu(S, N, alpha, kappa, tau, g, phi1, phi2, steps, prec)
    assert O.rel_l2(u3, u1) <= 1e-6, O.rel_l2(u3, u1)


def test_three_pass_convolution_rejected_where_it_does_not_apply(S):
    # FP64, and the register path (N' <= 1024), have no three-pass form
    for N, prec in ((2047, S.SADI_PREC_FP64), (1023, S.SADI_PREC_FP32)):
        with S.Sadi(N, 1.5, 1.0, 1e-3) as s:
            s.set_options(0, prec)
            t = s.sadi_get_tiles()
            with pytest.raises(S.SadiError) as ei:
                s.sadi_set_tiles(t[0], -1, t[2])
            assert ei.value.status == S.SADI_EINVAL
            assert s.sadi_get_tiles() == t

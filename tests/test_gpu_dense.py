"""The dense-inverse form (SADI_PREC_FP32_DENSE): both sweeps as split-BF16
tensor-core GEMMs with H^-1 = I + E, against the FP64 oracle.

Tolerances: the stored E (a BF16 pair) to 2^-16 of each entry; whole steps
1e-5 relative L2 as for the FP32 form."""
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


def _run(S, N, alpha, kappa, tau, g, phi1, phi2, steps, prec, dom=(-1.0, 1.0), F=None, om=0.0, ph=0.0):
    with S.Sadi(N, alpha, kappa, tau, dom) as s:
        s.set_options(g, prec)
        if F is not None:
            s.sadi_set_source(F, om, ph)
        s.set_initial(phi1, phi2)
        s.step(steps)
        u, n = s.get()
    assert n == steps
    return u


@pytest.mark.parametrize("N,alpha,tau", [(1, 1.5, 0.1), (7, 1.3, 0.05), (63, 1.5, 0.02), (200, 1.8, 0.01),
                                         (1023, 1.2, 1e-3)])
def test_dense_inverse_matches_oracle_inverse(S, N, alpha, tau):
    kappa = 1.0
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(0, S.SADI_PREC_FP32_DENSE)
        E = s.sadi_get_setup(4)
    h = 2.0 / (N + 1)
    sc = kappa * tau ** 2 / (2 * h ** alpha)
    H = np.eye(N) + sc * scipy.linalg.toeplitz(OW.riesz_1d(alpha, N))
    Eref = scipy.linalg.cho_solve(scipy.linalg.cho_factor(H), np.eye(N)) - np.eye(N)
    # the BF16 pair keeps 16 bits of each entry (plus the FP64 recurrence error)
    assert np.all(np.abs(E - Eref) <= 2.0 ** -16 * np.abs(Eref) + 1e-13 * np.abs(Eref).max())
    assert np.array_equal(E, E.T)


def test_dense_setup_requires_the_dense_form(S):
    with S.Sadi(15, 1.5, 1.0, 0.1) as s:
        with pytest.raises(S.SadiError) as ei:
            s.sadi_get_setup(4)
        assert ei.value.status == S.SADI_ESTATE
    with S.Sadi(15, 1.5, 1.0, 0.1) as s:
        with pytest.raises(S.SadiError) as ei:
            s.set_options(0, 7)
        assert ei.value.status == S.SADI_EINVAL


@pytest.mark.parametrize("N,alpha,g", [(1, 1.5, 1), (2, 1.3, 2), (5, 1.9, 0), (8, 1.6, 1), (9, 1.4, 2),
                                       (31, 1.7, 2), (33, 1.2, 1), (63, 1.5, 1), (64, 1.4, 2), (100, 1.3, 2),
                                       (128, 1.6, 1), (255, 1.8, 2), (257, 1.5, 1)])
def test_dense_step_parity(S, N, alpha, g):
    kappa, tau = 1.0, 0.02
    phi1 = WL.gaussian_bumps(N, 8, 5 + N)
    phi2 = 0.2 * WL.gaussian(N, 10.0)
    steps = 10
    P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, g)
    ref = O.run(P, phi1, phi2, steps, tier="fft" if N > 40 else "direct")
    u = _run(S, N, alpha, kappa, tau, g, phi1, phi2, steps, S.SADI_PREC_FP32_DENSE)
    assert O.rel_l2(u, ref) <= 1e-5, O.rel_l2(u, ref)
    assert np.abs(u - ref).max() <= 1e-5 * np.abs(ref).max()   # element-wise too


def test_dense_full_size_1023(S):
    w = WL.bumps_1023(1.8, steps=4)
    P = O.Problem(w.N, w.alpha, w.kappa, w.tau, w.a, w.b, w.g)
    ref = O.run(P, w.phi1, w.phi2, w.steps, tier="fft")
    u = _run(S, w.N, w.alpha, w.kappa, w.tau, w.g, w.phi1, w.phi2, w.steps, S.SADI_PREC_FP32_DENSE)
    assert O.rel_l2(u, ref) <= 1e-5, O.rel_l2(u, ref)
    assert np.abs(u - ref).max() <= 1e-5 * np.abs(ref).max()   # element-wise too


@pytest.mark.parametrize("N,alpha,g,steps", [(2047, 1.4, 1, 5), (4095, 1.7, 1, 3)])
def test_dense_large_n_against_fp64(S, N, alpha, g, steps):
    # N' = 2048: the FFT part on the register path; N' = 4096: on the
    # shared-memory engine; the sweeps as 8 x 16 and 16 x 32 tiles of 128 x 256
    tau, kappa = 5e-4, 0.5
    phi1 = WL.gaussian_bumps(N, 8, 2000 + N)
    u64 = _run(S, N, alpha, kappa, tau, g, phi1, None, steps, S.SADI_PREC_FP64)
    ud = _run(S, N, alpha, kappa, tau, g, phi1, None, steps, S.SADI_PREC_FP32_DENSE)
    assert O.rel_l2(ud, u64) <= 1e-5, O.rel_l2(ud, u64)


@pytest.mark.parametrize("N,alpha,g", [(1025, 1.3, 2), (1100, 1.7, 1)])
def test_dense_fft_engines_at_2048_against_oracle(S, N, alpha, g):
    # N' = 2048 (ragged: N = 1025 is the smallest N of that length): the
    # dense form's FFT part on the register path (64 elements per lane) by
    # default, on the shared-memory engine with explicit tiles; both against
    # the oracle element by element, and against each other
    kappa, tau, steps = 0.8, 1e-3, 3
    phi1 = WL.gaussian_bumps(N, 6, 900 + N)
    phi2 = 0.2 * WL.random_field(N, 901 + N)
    P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, g)
    ref = O.run(P, phi1, phi2, steps, tier="fft")
    us = {}
    for engine in ("register", "shared"):
        with S.Sadi(N, alpha, kappa, tau) as s:
            s.set_options(g, S.SADI_PREC_FP32_DENSE)
            if engine == "shared":
                s.sadi_set_tiles(*s.sadi_get_tiles())
            s.set_initial(phi1, phi2)
            s.step(steps)
            us[engine], n = s.get()
        assert n == steps
        u = us[engine]
        assert O.rel_l2(u, ref) <= 1e-5, (engine, O.rel_l2(u, ref))
        assert np.abs(u - ref).max() <= 1e-5 * np.abs(ref).max(), engine
    # different kernels (rounding order), the same scheme
    assert not np.array_equal(us["register"], us["shared"])
    assert O.rel_l2(us["register"], us["shared"]) <= 1e-6


def test_dense_engine_choice_at_2048(S):
    # explicit tiles move a dense N' = 2048 context to the shared-memory
    # engine and zeros move it back, before sadi_set_initial only; the FP64
    # path's tiles and the GS form are unaffected
    N, alpha, kappa, tau = 1100, 1.5, 1.0, 1e-3
    phi1 = WL.gaussian_bumps(N, 4, 950)

    def run(tiles_seq):
        with S.Sadi(N, alpha, kappa, tau) as s:
            s.set_options(1, S.SADI_PREC_FP32_DENSE)
            for t in tiles_seq:
                s.sadi_set_tiles(*t)
            s.set_initial(phi1)
            s.step(2)
            return s.get()[0]
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(1, S.SADI_PREC_FP32_DENSE)
        t = s.sadi_get_tiles()
    u_reg = run([])
    u_shared = run([t])
    assert not np.array_equal(u_reg, u_shared)
    assert np.array_equal(run([t, (0, 0, 0)]), u_reg)
    # three passes need the shared-memory engine: explicit tiles give it
    assert O.rel_l2(run([(t[0], -1, t[2])]), u_shared) <= 1e-6
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(1, S.SADI_PREC_FP32_DENSE)
        s.set_initial(phi1)
        with pytest.raises(S.SadiError) as ei:     # would re-lay the state
            s.sadi_set_tiles(*t)
        assert ei.value.status == S.SADI_ESTATE
        s.step(1)                                  # still steps on the register path
    # tiles set for the FP64 path do not move the dense form later
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.sadi_set_tiles(*s.sadi_get_tiles())
        s.set_options(1, S.SADI_PREC_FP32_DENSE)
        s.set_initial(phi1)
        s.step(2)
        assert np.array_equal(s.get()[0], u_reg)


def test_dense_source_term_and_second_order(S):
    N, alpha, kappa, tau, g = 31, 1.4, 0.8, 0.04, 2
    F = WL.random_field(N, 77)
    om, ph = 2.3, 0.4
    phi1 = WL.gaussian_bumps(N, 3, 78)
    phi2 = 0.2 * WL.random_field(N, 79)
    P = O.Problem(N, alpha, kappa, tau, -1.0, 1.0, g)
    ref = O.run(P, phi1, phi2, 7, tier="direct", forcing=lambda n: np.cos(om * n * tau + ph) * F)
    u = _run(S, N, alpha, kappa, tau, g, phi1, phi2, 7, S.SADI_PREC_FP32_DENSE, F=F, om=om, ph=ph)
    assert O.rel_l2(u, ref) <= 1e-5
    # manufactured solution U = cos(t) phi (g = 0): O(tau^2) convergence
    N, alpha, kappa = 63, 1.5, 1.0
    phi = WL.gaussian(N, 8.0)
    errs = []
    for M in (8, 16, 32):
        tau = 1.0 / M
        P = O.Problem(N, alpha, kappa, tau)
        Fm = kappa * O.lh_direct(P, phi) - phi
        u = _run(S, N, alpha, kappa, tau, 0, phi, None, M, S.SADI_PREC_FP32_DENSE, F=Fm, om=1.0)
        errs.append(np.abs(u - np.cos(1.0) * phi).max())
    orders = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.9 < o < 2.15 for o in orders), (orders, errs)


def test_dense_batch_matches_single_contexts(S):
    # dense contexts of one FFT length (N' = 64) batch their FFT kernels and
    # their GEMMs (different N: 1 x 1 tiles each); an FP32 context of the same
    # N' and a dense N' = 512 context join the same call
    specs = [(63, 1.5, 1.0, 0.02, 1, 2), (50, 1.2, 0.7, 0.03, 2, 2), (33, 1.8, 1.3, 0.01, 0, 2),
             (40, 1.6, 1.0, 0.02, 1, 1), (300, 1.3, 1.0, 0.01, 2, 2)]

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


@pytest.mark.parametrize("N", [1023, 2047])
def test_long_run_fp32_forms_track_fp64(S, N):
    # 250 steps of the N=4095 precision workload's parameters (alpha 1.7,
    # kappa 0.5, tau 5e-4, g = -u^3): both FP32 forms stay within 1e-6 of the
    # FP64 path.  N = 1023 runs the register FFT path; at N = 2047 the GS
    # form runs on the shared-memory engine (the dense form's FFT part on the
    # register path), whose packed k1 = 0 / k1 = N' column must keep
    # the small low-frequency symbol free of cancellation (before that was
    # fixed the drift here was about 4e-6).
    alpha, kappa, tau, g, steps = 1.7, 0.5, 5e-4, 1, 250
    phi1 = WL.gaussian_bumps(N, 8, WL.SEED_BASE + 3)
    u64 = _run(S, N, alpha, kappa, tau, g, phi1, None, steps, S.SADI_PREC_FP64)
    for prec in (S.SADI_PREC_FP32, S.SADI_PREC_FP32_DENSE):
        u = _run(S, N, alpha, kappa, tau, g, phi1, None, steps, prec)
        assert O.rel_l2(u, u64) <= 1e-6, (prec, O.rel_l2(u, u64))


def test_wide_row_blocks_match_narrow_ones_bitwise(S):
    # three N' = 1024 instances per form exceed one wave of the narrow row
    # blocks (4 rows, 4 per SM), so the batch takes the wide ones (21 rows,
    # one per SM) for the row transform, the B^n kernel and the GS x sweep;
    # a context stepped alone takes the narrow ones.  Every row's arithmetic
    # is the same either way: the fields agree bitwise.
    specs = [(1023, 1.2, 1.0, 1e-3, 2, 2), (1023, 1.5, 1.0, 1e-3, 2, 2), (1001, 1.8, 0.9, 1e-3, 1, 2),
             (1023, 1.4, 0.9, 1e-3, 1, 1), (900, 1.6, 1.1, 1e-3, 2, 1), (1023, 1.3, 0.8, 1e-3, 2, 1)]

    def make():
        out = []
        for k, (N, al, ka, ta, g, prec) in enumerate(specs):
            s = S.Sadi(N, al, ka, ta)
            s.set_options(g, prec)
            s.set_initial(WL.gaussian_bumps(N, 6, 1300 + k), 0.3 * WL.random_field(N, 1400 + k))
            out.append(s)
        return out
    single = make()
    for s in single:
        s.step(4)
    ref = [s.get()[0] for s in single]
    batch = make()
    S.sadi_batch_step(batch, 4)
    for k, (s, r) in enumerate(zip(batch, ref)):
        u, n = s.get()
        assert n == 4
        assert np.array_equal(u, r), f"instance {k} {specs[k]}"
    for s in single + batch:
        s.close()


def test_bench_launch_configuration_against_the_oracle(S):
    # the N = 1023 workload as the benchmark steps it: its three alpha
    # instances batched in the dense form (one launch per kernel, the wide row
    # blocks, both sweeps of all three in one GEMM launch), each instance
    # against the oracle's FFT tier
    ws = [WL.bumps_1023(al, steps=4) for al in (1.2, 1.5, 1.8)]
    ctxs = []
    for w in ws:
        s = S.Sadi(w.N, w.alpha, w.kappa, w.tau, (w.a, w.b))
        s.set_options(w.g, S.SADI_PREC_FP32_DENSE)
        s.set_initial(w.phi1, w.phi2)
        ctxs.append(s)
    S.sadi_batch_step(ctxs, 4)
    for w, s in zip(ws, ctxs):
        u, n = s.get()
        s.close()
        assert n == 4
        P = O.Problem(w.N, w.alpha, w.kappa, w.tau, w.a, w.b, w.g)
        ref = O.run(P, w.phi1, w.phi2, w.steps, tier="fft")
        err = O.rel_l2(u, ref)
        assert err <= 1e-5, (w.alpha, err)
        ew = np.abs(u - ref).max() / np.abs(ref).max()
        assert ew <= 1e-5, (w.alpha, ew)   # element-wise too

"""Failure detection through the C ABI, with nothing that can fault or hang
the GPU: the failures are made on the host (a NaN planted in the initial
data) or by a wait for a count that nothing raises, under a short limit.

* The state watchdog: a NaN in phi1 must come back as SADI_ENONFINITE from
  the first synchronising call after the first check, for every step form,
  stepped directly, batched or by graph replay; the context then needs new
  data and steps normally again.  With finite data the watchdog's norm is
  the discrete L2 norm of the state it checked.
* The dense form's bounded device waits: sadi_debug_expire_waits makes the
  y-sweep tiles of one GEMM launch wait for a panel count that is never
  reached, under a 10 ms limit.  The launch returns, sadi_get reports
  SADI_ETIMEOUT, the context refuses further work, and a new context in the
  same process steps to the same bits as one run before the failure."""
import numpy as np
import pytest

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


PRECS = ["SADI_PREC_FP64", "SADI_PREC_FP32", "SADI_PREC_FP32_DENSE"]


def _status(S, fn, *args):
    try:
        fn(*args)
    except S.SadiError as e:
        return e.status
    return S.SADI_OK


@pytest.mark.parametrize("prec_name", PRECS)
@pytest.mark.parametrize("N", [63, 1023])
def test_watchdog_reports_nonfinite_state(S, prec_name, N):
    prec = getattr(S, prec_name)
    phi1 = WL.gaussian_bumps(N, 4, WL.SEED_BASE + 60)
    bad = phi1.copy()
    bad[N // 3, N // 2] = np.nan
    with S.Sadi(N, 1.5, 1.0, 1e-3) as s:
        s.set_options(1, prec)
        s.sadi_set_watchdog(4)
        s.set_initial(bad)
        s.step(3)                                   # n = 3: no check yet
        assert _status(S, s.get) == S.SADI_OK
        s.step(1)                                   # n = 4: checked
        st = _status(S, s.get)
        assert st == S.SADI_ENONFINITE, st
        assert "step 4" in s.sadi_last_error()
        assert _status(S, s.step, 1) == S.SADI_ESTATE   # new data needed
        s.set_initial(phi1)                          # clears the flag
        s.step(8)
        u, n = s.get()
        assert n == 8 and np.isfinite(u).all()
        norm, at = s.sadi_get_watchdog()
        h = 2.0 / (N + 1)
        ref = h * np.linalg.norm(u)
        assert at == 8 and abs(norm - ref) <= (1e-12 if prec == S.SADI_PREC_FP64 else 1e-6) * ref
    # switched off: nothing is reported
    with S.Sadi(N, 1.5, 1.0, 1e-3) as s:
        s.set_options(1, prec)
        s.sadi_set_watchdog(0)
        s.set_initial(bad)
        s.step(5)
        u, _ = s.get()
        assert not np.isfinite(u).all()


def test_watchdog_in_batches_and_graph_replays(S):
    N = 255
    phi1 = WL.gaussian_bumps(N, 4, WL.SEED_BASE + 61)
    bad = phi1.copy()
    bad[7, 9] = np.inf
    import torch
    stream = torch.cuda.Stream()
    ctxs = [S.Sadi(N, a, 1.0, 2e-3) for a in (1.3, 1.7)]
    try:
        for s, p in zip(ctxs, (bad, phi1)):
            s.set_stream(stream.cuda_stream)            # a graph's contexts share one stream
            s.set_options(1, S.SADI_PREC_FP32)
            s.sadi_set_watchdog(3)
            s.set_initial(p)
        S.sadi_batch_step(ctxs, 2)                  # n = 2
        assert all(_status(S, s.sadi_wait) == S.SADI_OK for s in ctxs)
        g = S.SadiGraph(ctxs, 1)
        g.launch(1)                                 # n = 3: checked after the replay
        g.close()
        assert _status(S, ctxs[0].sadi_wait) == S.SADI_ENONFINITE
        assert _status(S, ctxs[1].sadi_wait) == S.SADI_OK
        u, n = ctxs[1].get()
        assert n == 3 and np.isfinite(u).all()
    finally:
        for s in ctxs:
            s.close()


def _dense_run(S, N, phi1, steps):
    with S.Sadi(N, 1.5, 1.0, 2e-3) as s:
        s.set_options(2, S.SADI_PREC_FP32_DENSE)
        s.set_initial(phi1)
        s.step(steps)
        return s.get()[0]


@pytest.mark.parametrize("N", [63, 1023])
def test_dense_sweep_waits_run_out_and_are_reported(S, N):
    phi1 = WL.gaussian_bumps(N, 6, WL.SEED_BASE + 62)
    before = _dense_run(S, N, phi1, 3)
    with S.Sadi(N, 1.5, 1.0, 2e-3) as s:
        s.set_options(2, S.SADI_PREC_FP32_DENSE)
        s.set_initial(phi1)
        s.step(2)
        assert _status(S, s.sadi_wait) == S.SADI_OK
        s.sadi_debug_expire_waits(10_000_000)        # 10 ms
        s.step(1)
        st = _status(S, s.get)
        assert st == S.SADI_ETIMEOUT, st
        assert _status(S, s.step, 1) == S.SADI_ESTATE
    # the process and the GPU carry on: a new context gives the same bits
    after = _dense_run(S, N, phi1, 3)
    assert np.array_equal(before, after)


def test_expiry_hook_arguments(S):
    with S.Sadi(31, 1.5, 1.0, 1e-2) as s:
        assert _status(S, s.sadi_debug_expire_waits, 10_000_000) == S.SADI_EUNSUPPORTED   # FP64
        s.set_options(0, S.SADI_PREC_FP32_DENSE)
        for bad in (0, 99_999, 1_000_000_001):
            assert _status(S, s.sadi_debug_expire_waits, bad) == S.SADI_EINVAL
        assert _status(S, s.sadi_set_watchdog, -1) == S.SADI_EINVAL

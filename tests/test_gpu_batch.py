"""Batched stepping services through the C ABI: CUDA-graph replay
(sadi_graph_*) and the autotuner (sadi_autotune)."""
import numpy as np
import pytest

from oracle import sadi as O
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


# (N, alpha, kappa, tau, g, prec): register path (N' = 64, 256, and the
# dense form at N' = 2048), shared-memory engine (the GS form at N' = 2048)
SPECS = [(63, 1.5, 1.0, 0.02, 1, 1), (50, 1.2, 0.7, 0.03, 2, 1), (200, 1.8, 1.3, 0.01, 1, 2),
         (255, 1.6, 1.0, 0.005, 1, 2), (1500, 1.4, 0.5, 1e-3, 1, 1), (1100, 1.7, 0.8, 1e-3, 2, 2)]


def _make(S, stream):
    out = []
    for k, (N, al, ka, ta, g, prec) in enumerate(SPECS):
        s = S.Sadi(N, al, ka, ta)
        s.set_options(g, prec)
        s.set_stream(stream)
        s.set_initial(WL.gaussian_bumps(N, 4, 500 + k), 0.2 * WL.random_field(N, 600 + k))
        out.append(s)
    return out


def test_graph_replay_matches_batch_stepping_bitwise(S):
    import torch
    st = torch.cuda.Stream()
    ref = _make(S, st.cuda_stream)
    S.sadi_batch_step(ref, 7)
    want = [s.get()[0] for s in ref]
    run = _make(S, st.cuda_stream)
    S.sadi_batch_step(run, 1)                 # the n = 0 step is not replayed
    g = S.SadiGraph(run, nsteps=2)
    assert all(s.get()[1] == 1 for s in run)  # capture runs nothing
    # two steps: register groups (N' = 64 FP32: 4 kernels; N' = 256 and
    # N' = 2048 dense: 3 kernels + one launch of both sweep GEMMs each), one
    # shared-memory context (FP32: 3 + the y sweep on the transpose, 3)
    assert g.sadi_graph_kernels() == 2 * (4 + 4 + 6 + 4)
    g.launch(3)
    for s, w in zip(run, want):
        u, n = s.get()
        assert n == 7 and np.array_equal(u, w)
    g.close()
    for s in ref + run:
        s.close()


def test_graph_rejects_what_it_cannot_replay(S):
    import torch
    st = torch.cuda.Stream()
    a = S.Sadi(31, 1.5, 1.0, 0.1)
    a.set_options(1, S.SADI_PREC_FP32)
    a.set_stream(st.cuda_stream)
    a.set_initial(WL.gaussian(31, 10.0))
    with pytest.raises(S.SadiError) as ei:     # n = 0
        S.SadiGraph([a])
    assert ei.value.status == S.SADI_ESTATE
    b = S.Sadi(31, 1.5, 1.0, 0.1)
    b.set_stream(st.cuda_stream)
    b.set_initial(WL.gaussian(31, 10.0))
    b.step(1)
    with pytest.raises(S.SadiError) as ei:     # FP64 (ping-pong state)
        S.SadiGraph([b])
    assert ei.value.status == S.SADI_EUNSUPPORTED
    a.step(1)
    g = S.SadiGraph([a])
    a.set_initial(WL.gaussian(31, 10.0))       # back to n = 0: launching must refuse
    with pytest.raises(S.SadiError) as ei:
        g.launch(1)
    assert ei.value.status == S.SADI_ESTATE
    g.close()
    a.close()
    b.close()


def test_autotune_picks_a_form_per_n_and_keeps_parity(S):
    Ns = [63, 63, 1100]
    ctxs = [S.Sadi(N, 1.5, 1.0, 0.01) for N in Ns]
    S.sadi_autotune(ctxs, 1)
    logs = [s.sadi_tuning_log() for s in ctxs]
    assert logs[0] == logs[1] and "N=63" in logs[0] and "->" in logs[0]
    assert "N=1100" in logs[2] and "tiles" in logs[2]
    for N, s in zip(Ns, ctxs):
        with pytest.raises(S.SadiError):       # left uninitialised
            s.step(1)
        phi1 = WL.gaussian_bumps(N, 6, 700 + N)
        s.set_initial(phi1)
        s.step(5)
        u, _ = s.get()
        P = O.Problem(N, 1.5, 1.0, 0.01, -1.0, 1.0, 1)
        if N <= 100:
            ref = O.run(P, phi1, np.zeros_like(phi1), 5, tier="fft")
        else:
            with S.Sadi(N, 1.5, 1.0, 0.01) as r:
                r.set_options(1, S.SADI_PREC_FP64)
                r.set_initial(phi1)
                r.step(5)
                ref, _ = r.get()
        assert O.rel_l2(u, ref) <= 1e-5
        s.close()


def test_autotune_can_keep_the_precision(S):
    # flags bit 1: tiles only, the precision each context was given stays
    # (the GS form at N' = 2048 on the shared-memory engine has tiles; the
    # dense form there runs on the register path, which has none)
    ctxs = [S.Sadi(1100, 1.5, 1.0, 0.01) for _ in range(2)]
    ctxs[0].set_options(1, S.SADI_PREC_FP32)
    ctxs[1].set_options(1, S.SADI_PREC_FP32)
    S.sadi_autotune(ctxs, 1, 2)
    assert all(s.sadi_get_options() == (1, S.SADI_PREC_FP32) for s in ctxs)
    assert "fp32-dense" not in ctxs[0].sadi_tuning_log() and "tiles" in ctxs[0].sadi_tuning_log()
    dense = [S.Sadi(1100, 1.5, 1.0, 0.01) for _ in range(2)]
    for s in dense:
        s.set_options(1, S.SADI_PREC_FP32_DENSE)
    S.sadi_autotune(dense, 1, 2)
    assert all(s.sadi_get_options() == (1, S.SADI_PREC_FP32_DENSE) for s in dense)
    assert "fp32-gsfft" not in dense[0].sadi_tuning_log() and "tiles" not in dense[0].sadi_tuning_log()
    ctxs += dense
    f64 = S.Sadi(63, 1.5, 1.0, 0.01)
    with pytest.raises(S.SadiError) as ei:
        S.sadi_autotune([f64], 1, 2)
    assert ei.value.status == S.SADI_EUNSUPPORTED
    for s in ctxs + [f64]:
        s.close()

"""The batch handle (sadi_batch_create / set_initial / run / get) through the
C ABI: members of uneven N, alpha, kappa, tau advanced together give the same
bits as each member stepped alone with the same step form (batched launches
and graph replays compute each member exactly as sadi_step does)."""
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


def _alone(S, N, alpha, kappa, tau, g, prec, tiles, phi1, steps):
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(g, prec)
        if tiles is not None:
            s.sadi_set_tiles(*tiles)
        s.set_initial(phi1)
        s.step(steps)
        return s.get()


def _member_setup(S, b, k):
    import ctypes
    ctx = b.sadi_batch_member(k)
    g, p = ctypes.c_int(), ctypes.c_int()
    assert S.lib().sadi_get_options(ctx, ctypes.byref(g), ctypes.byref(p)) == 0
    t = (ctypes.c_int * 3)()
    assert S.lib().sadi_get_tiles(ctx, t) == 0
    return p.value, tuple(t)


@pytest.mark.parametrize("prec_name", ["SADI_PREC_AUTO", "SADI_PREC_FP32", "SADI_PREC_FP64"])
def test_batch_matches_members_stepped_alone(S, prec_name):
    prec = getattr(S, prec_name)
    Ns = [63, 127, 255, 255, 511, 1023]
    rng = np.random.default_rng(WL.SEED_BASE + 70)
    alphas = rng.uniform(1.1, 1.9, len(Ns))
    kappas = rng.uniform(0.5, 2.0, len(Ns))
    taus = [1.0 / (N + 1) for N in Ns]
    phis = [WL.gaussian_bumps(N, 4, WL.SEED_BASE + 71 + k) for k, N in enumerate(Ns)]
    with S.SadiBatch(Ns, alphas, kappas, taus, g=1, prec=prec) as b:
        assert b.sadi_batch_count() == len(Ns)
        with pytest.raises(S.SadiError) as ei:      # no initial data yet
            b.run(1)
        assert ei.value.status == S.SADI_ESTATE
        for k, p in enumerate(phis):
            b.set_initial(k, p)
        b.run(2)
        b.run(4)                                    # FP32 forms: graph replays from here
        setups = [_member_setup(S, b, k) for k in range(len(Ns))]
        outs = [b.get(k) for k in range(len(Ns))]
        for k, N in enumerate(Ns):
            p, tiles = setups[k]
            if prec != S.SADI_PREC_AUTO:
                assert p == prec
            ref, n = _alone(S, N, alphas[k], kappas[k], taus[k], 1, p, tiles, phis[k], 6)
            assert outs[k][1] == n == 6
            assert np.array_equal(outs[k][0], ref), (k, N, p)
        # member 2 starts again; the others continue
        b.set_initial(2, phis[2])
        b.run(3)
        u2, n2 = b.get(2)
        ref, _ = _alone(S, 255, alphas[2], kappas[2], taus[2], 1, setups[2][0], setups[2][1], phis[2], 3)
        assert n2 == 3 and np.array_equal(u2, ref)
        assert b.get(0)[1] == 9


def test_batch_argument_errors(S):
    with pytest.raises(S.SadiError) as ei:
        S.SadiBatch([63, 0], [1.5, 1.5], [1.0, 1.0], [0.01, 0.01], prec=S.SADI_PREC_FP32)
    assert ei.value.status == S.SADI_EINVAL and "member 1" in str(ei.value)
    with S.SadiBatch([31], [1.5], [1.0], [0.01], prec=S.SADI_PREC_FP64) as b:
        with pytest.raises(S.SadiError) as ei:
            b.set_initial(1, np.zeros((31, 31)))
        assert ei.value.status == S.SADI_EINVAL
        with pytest.raises(S.SadiError) as ei:
            b.get(0)
        assert ei.value.status == S.SADI_ESTATE


def test_fp64_graph_replays_even_step_counts(S):
    # FP64 buffers swap every step: graphs of an even number of steps replay
    # bitwise what direct steps give; odd counts are refused, and so is a
    # launch after an odd number of direct steps since the capture
    import torch
    N = 127
    phi1 = WL.gaussian_bumps(N, 4, WL.SEED_BASE + 75)
    stream = torch.cuda.Stream()

    def ctx():
        s = S.Sadi(N, 1.6, 1.0, 1.0 / (N + 1))
        s.set_stream(stream.cuda_stream)
        s.set_options(1, S.SADI_PREC_FP64)
        s.set_initial(phi1)
        s.step(1)
        return s
    with ctx() as a, ctx() as b:
        with pytest.raises(S.SadiError) as ei:
            S.SadiGraph([a], 3)
        assert ei.value.status == S.SADI_EUNSUPPORTED
        g = S.SadiGraph([a], 2)
        g.launch(5)
        b.step(10)
        ua, na = a.get()
        ub, nb = b.get()
        assert na == nb == 11 and np.array_equal(ua, ub)
        a.step(1)
        with pytest.raises(S.SadiError) as ei:
            g.launch(1)
        assert ei.value.status == S.SADI_ESTATE
        a.step(1)
        g.launch(1)
        b.step(4)
        assert np.array_equal(a.get()[0], b.get()[0])
        g.close()
    # the batch handle replays FP64 members in two-step graphs, an odd tail directly
    with S.SadiBatch([63, 127], [1.4, 1.6], [1.0, 1.0], [1 / 64, 1 / 128], g=1, prec=S.SADI_PREC_FP64) as bt:
        for k, n in enumerate((63, 127)):
            bt.set_initial(k, WL.gaussian_bumps(n, 3, WL.SEED_BASE + 76 + k))
        bt.run(7)
        bt.run(4)
        for k, n in enumerate((63, 127)):
            ref, _ = _alone(S, n, [1.4, 1.6][k], 1.0, [1 / 64, 1 / 128][k], 1, S.SADI_PREC_FP64, None,
                            WL.gaussian_bumps(n, 3, WL.SEED_BASE + 76 + k), 11)
            u, m = bt.get(k)
            assert m == 11 and np.array_equal(u, ref), k

"""sadi_step_noalloc (caller-owned device state, fixed library scratch) against
sadi_step on the same context setup.

Collected last on purpose: the entry point shares one scratch array for the
whole process, so it must give the same results both in a fresh process and
after every other GPU test has run.  Tolerance: the FP64 path's 1e-10
relative L2."""
import numpy as np
import pytest

from paper_2312_06206_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_06206_gb300 import build
    build.build()
    from paper_2312_06206_gb300 import sadi
    return sadi, torch


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _reference_levels(S, N, alpha, kappa, tau, g, phi1, phi2, levels, F=None, omega=0.0, phase=0.0):
    """u^0 .. u^levels from sadi_step + sadi_get (one step at a time)."""
    out = []
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(g, S.SADI_PREC_FP64)
        if F is not None:
            s.sadi_set_source(F, omega, phase)
        s.set_initial(phi1, phi2)
        out.append(s.get()[0])
        for _ in range(levels):
            s.step(1)
            out.append(s.get()[0])
    return out


@pytest.mark.parametrize("N,alpha,g,with_source", [
    (63, 1.5, 1, False),      # -u^3
    (200, 1.8, 2, True),      # -sin u, plus a source term, ragged N (N' = 256)
    (1024, 1.3, 2, False),    # the largest N the fixed scratch serves
])
def test_noalloc_matches_sadi_step_on_two_calls_in_a_row(env, N, alpha, g, with_source):
    S, torch = env
    kappa, tau = 1.0, 2.0 / (N + 1)
    phi1 = WL.gaussian_bumps(N, 6, seed=WL.SEED_BASE + 40 + N)
    phi2 = 0.3 * WL.gaussian_bumps(N, 3, seed=WL.SEED_BASE + 41 + N)
    F = omega = phase = None
    if with_source:
        X, Y = WL.coords(N, -1.0, 1.0)
        F, omega, phase = np.exp(-8.0 * (X ** 2 + Y ** 2)), 3.0, 0.25
    ref = _reference_levels(S, N, alpha, kappa, tau, g, phi1, phi2, 4, F, omega or 0.0, phase or 0.0)

    dev = torch.device("cuda:0")
    with S.Sadi(N, alpha, kappa, tau) as s:
        s.set_options(g, S.SADI_PREC_FP64)
        if with_source:
            s.sadi_set_source(F, omega, phase)
        st = torch.cuda.Stream(device=dev)
        s.sadi_set_stream(st.cuda_stream)
        A = torch.tensor(ref[1], dtype=torch.float64, device=dev)   # u^1
        B = torch.tensor(ref[2], dtype=torch.float64, device=dev)   # u^2
        C = torch.empty((N, N), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        # first call: u^3 from (u^1, u^2) into a separate buffer
        s.sadi_step_noalloc(A.data_ptr(), B.data_ptr(), C.data_ptr(), 2)
        st.synchronize()
        u3 = C.cpu().numpy()
        assert _rel(u3, ref[3]) <= TOL
        # second call right after: u^4 from (u^2, u^3), in place over u^2
        s.sadi_step_noalloc(B.data_ptr(), C.data_ptr(), B.data_ptr(), 3)
        st.synchronize()
        u4 = B.cpu().numpy()
        assert _rel(u4, ref[4]) <= TOL
        # the context's own state was not touched
        with pytest.raises(S.SadiError):
            s.get()


def test_noalloc_rejects_what_it_cannot_serve(env):
    S, torch = env
    dev = torch.device("cuda:0")
    # N' = 2048: 16 N N' + 8 N^2 bytes exceed the fixed scratch
    N = 1025
    with S.Sadi(N, 1.5, 1.0, 1e-3) as s:
        bufs = [torch.zeros((N, N), dtype=torch.float64, device=dev) for _ in range(3)]
        with pytest.raises(S.SadiError) as ei:
            s.sadi_step_noalloc(bufs[0].data_ptr(), bufs[1].data_ptr(), bufs[2].data_ptr(), 1)
        assert ei.value.status == S.SADI_EINVAL and "scratch" in str(ei.value)
    N = 31
    with S.Sadi(N, 1.5, 1.0, 1e-2) as s:
        d = [torch.zeros((N, N), dtype=torch.float64, device=dev) for _ in range(3)]
        host = np.zeros((N, N))
        with pytest.raises(S.SadiError) as ei:   # host memory is refused before any launch
            s.sadi_step_noalloc(host.ctypes.data, d[1].data_ptr(), d[2].data_ptr(), 1)
        assert ei.value.status == S.SADI_EINVAL
        with pytest.raises(S.SadiError) as ei:   # u_next may not overlap u_cur
            s.sadi_step_noalloc(d[0].data_ptr(), d[1].data_ptr(), d[1].data_ptr(), 1)
        assert ei.value.status == S.SADI_EINVAL
        with pytest.raises(S.SadiError) as ei:   # n is the level of u_cur, >= 1
            s.sadi_step_noalloc(d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), 0)
        assert ei.value.status == S.SADI_EINVAL
        s.set_options(0, S.SADI_PREC_FP32)
        with pytest.raises(S.SadiError) as ei:
            s.sadi_step_noalloc(d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), 1)
        assert ei.value.status == S.SADI_EUNSUPPORTED


def test_noalloc_allocates_nothing_and_checks_buffer_lengths(env):
    S, torch = env
    dev = torch.device("cuda:0")
    N = 512
    nn_bytes = N * N * 8
    with S.Sadi(N, 1.5, 1.0, 2.0 / (N + 1)) as s:
        s.set_options(1, S.SADI_PREC_FP64)
        st = torch.cuda.Stream(device=dev)
        s.sadi_set_stream(st.cuda_stream)
        u = [torch.tensor(WL.gaussian_bumps(N, 4, seed=WL.SEED_BASE + 50 + k), dtype=torch.float64, device=dev)
             for k in range(3)]
        torch.cuda.synchronize()
        s.sadi_step_noalloc(u[0].data_ptr(), u[1].data_ptr(), u[2].data_ptr(), 1)   # device set-up done
        st.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        for k in range(4):
            s.sadi_step_noalloc(u[k % 3].data_ptr(), u[(k + 1) % 3].data_ptr(), u[(k + 2) % 3].data_ptr(), 2 + k)
        st.synchronize()
        assert torch.cuda.mem_get_info(dev)[0] == free0, "a call changed the free device memory"
        assert all(bool(torch.isfinite(x).all()) for x in u)
        # a buffer that ends one grid row early inside its allocation: a fresh
        # 12 MiB tensor (above the caching allocator's 10 MB threshold, so it
        # gets an allocation of its own), pointers placed near its end
        torch.cuda.empty_cache()
        T = torch.zeros((12 << 20) // 8, dtype=torch.float64, device=dev)
        end = T.data_ptr() + (12 << 20)
        short = end - (nn_bytes - 8 * N)
        exact = end - nn_bytes
        for args in ((short, u[1].data_ptr(), u[2].data_ptr()), (u[0].data_ptr(), short, u[2].data_ptr()),
                     (u[0].data_ptr(), u[1].data_ptr(), short)):
            with pytest.raises(S.SadiError) as ei:
                s.sadi_step_noalloc(*args, 3)
            assert ei.value.status == S.SADI_EINVAL and "shorter" in str(ei.value)
        s.sadi_step_noalloc(u[0].data_ptr(), u[1].data_ptr(), exact, 3)   # exactly N*N doubles: accepted
        st.synchronize()
        assert bool(torch.isfinite(T).all())

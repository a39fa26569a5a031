"""Checkpoint and resume through the C ABI (sadi_save_state /
sadi_load_state): a resumed context continues bitwise as the saved one; and
asynchronous reads of the state (sadi_get_async / sadi_wait) equal the
synchronous ones."""
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


def _ctx(S, N, prec, alpha=1.6):
    s = S.Sadi(N, alpha, 0.9, 0.02)
    s.set_options(1, prec)
    return s


@pytest.mark.parametrize("N,prec", [(63, 0), (63, 1), (200, 2), (1500, 1)])
@pytest.mark.parametrize("at", [0, 7])
def test_resume_continues_bitwise(S, N, prec, at):
    phi1 = WL.gaussian_bumps(N, 5, 900 + N)
    phi2 = 0.3 * WL.random_field(N, 901 + N)
    a = _ctx(S, N, prec)
    a.set_initial(phi1, phi2)
    a.step(at)
    blob = a.sadi_save_state()
    a.step(5)
    ua, na = a.get()
    b = _ctx(S, N, prec)
    b.sadi_load_state(blob)
    b.step(5)
    ub, nb = b.get()
    assert na == nb == at + 5
    assert np.array_equal(ua, ub)
    a.close()
    b.close()


def test_load_rejects_a_foreign_blob(S):
    a = _ctx(S, 31, 1)
    with pytest.raises(S.SadiError) as ei:          # nothing to save yet
        a.sadi_save_state()
    assert ei.value.status == S.SADI_ESTATE
    a.set_initial(WL.gaussian(31, 10.0))
    a.step(2)
    blob = a.sadi_save_state()
    for other in (_ctx(S, 31, 1, alpha=1.7), _ctx(S, 31, 0), _ctx(S, 33, 1)):
        with pytest.raises(S.SadiError) as ei:
            other.sadi_load_state(blob)
        assert ei.value.status == S.SADI_EINVAL
        other.close()
    b = _ctx(S, 31, 1)
    with pytest.raises(S.SadiError):
        b.sadi_load_state(blob[:100])
    with pytest.raises(S.SadiError):
        b.sadi_load_state(b"x" * len(blob))
    a.close()
    b.close()


@pytest.mark.parametrize("N,prec", [(200, 0), (200, 1), (200, 2), (1500, 1)])
def test_async_reads_match_synchronous_reads(S, N, prec):
    # sadi_get_async of consecutive steps into separate pinned buffers, waited
    # for once, returns the same fields as sadi_get after each step; a read
    # queued before sadi_set_initial (which rewrites the staging buffer) still
    # returns the state it was queued for
    import torch
    phi1 = WL.gaussian_bumps(N, 5, 910 + N)
    phi2 = 0.2 * WL.random_field(N, 911 + N)
    ref = []
    with _ctx(S, N, prec) as s:
        s.set_initial(phi1, phi2)
        for _ in range(4):
            s.step(1)
            ref.append(s.get()[0])
    bufs = [torch.empty((N, N), dtype=torch.float64).pin_memory() for _ in range(5)]
    with _ctx(S, N, prec) as s:
        s.set_initial(phi1, phi2)
        for k in range(4):
            s.step(1)
            s.sadi_get_async(bufs[k].data_ptr())
        s.sadi_wait()
        for k in range(4):
            assert np.array_equal(bufs[k].numpy(), ref[k])
        s.sadi_get_async(bufs[4].data_ptr())
        s.set_initial(phi2, None)
        s.sadi_wait()
        assert np.array_equal(bufs[4].numpy(), ref[3])
        with pytest.raises(S.SadiError) as ei:
            s.sadi_get_async(0)
        assert ei.value.status == S.SADI_EINVAL
    with _ctx(S, N, prec) as s:
        with pytest.raises(S.SadiError) as ei:
            s.sadi_get_async(bufs[0].data_ptr())
        assert ei.value.status == S.SADI_ESTATE

"""Checkpoint and resume through the C ABI (sadi_save_state /
sadi_load_state): a resumed context continues bitwise as the saved one."""
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

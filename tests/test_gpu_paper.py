"""The paper's own accuracy tables (Sec. 6) reproduced through the C ABI on
the GPU, to half a unit of the last printed digit.

Table 1 (Example 1, sine-Gordon, alpha = 1.5, h = 1/40 so N = 799, t = 5):
Error_1(tau) = sqrt(h^2 sum |u(tau) - u(tau/2)|^2) for tau = 1/10 ... 1/80.
Table 4 (Example 2, Klein-Gordon, alpha = 1.5, tau = 1/125, t = 8):
Error_2 between h = 2/5 (N = 49) and h = 1/5 (N = 99), with the initial
amplitude 2 that reproduces the printed values."""
import math

import numpy as np
import pytest

from oracle import sadi as O
from paper_2312_06206_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TABLE1_A15 = {10: 8.9900e-3, 20: 2.2583e-3, 40: 5.6526e-4, 80: 1.4136e-4}


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_06206_gb300 import build
    build.build()
    from paper_2312_06206_gb300 import sadi
    return sadi


def _half_unit(ref):
    return 0.5 * 10.0 ** (np.floor(np.log10(ref)) - 4)


def _run(S, w, prec):
    with S.Sadi(w.N, w.alpha, w.kappa, w.tau, (w.a, w.b)) as s:
        s.set_options(w.g, prec)
        s.set_initial(w.phi1, w.phi2)
        s.step(w.steps)
        u, n = s.get()
    assert n == w.steps
    return u


@pytest.fixture(scope="module")
def table1_fp64(S):
    N, alpha = 799, 1.5
    return {m: _run(S, WL.paper_example1(N, alpha, 1.0 / m), 0) for m in (10, 20, 40, 80, 160)}


def test_paper_table1_alpha15_column(table1_fp64):
    us = table1_fp64
    for m, ref in TABLE1_A15.items():
        e = O.error1(1 / 40, us[m], us[2 * m])
        assert abs(e - ref) <= _half_unit(ref), (m, e, ref)


@pytest.mark.parametrize("prec", [1, 2])
def test_paper_table1_fp32_forms_track_fp64(S, table1_fp64, prec):
    # Error_1 is a small difference of two runs (down to 1.4e-4 here), so the
    # FP32 forms cannot keep its five printed digits; they must agree with the
    # FP64 value to 2 eps h ||u|| with eps = 1e-6 (the FP32 forms' relative
    # accuracy on u).  The dense form is held to it only where s a_0 <= 0.2
    # (s = kappa tau^2 / (2 h^alpha)), the range the autotuner offers it in; at
    # tau = 1/20 already s a_0 = 0.50 and the split of E costs about 5e-6.
    N, alpha, h = 799, 1.5, 1 / 40
    a0 = math.gamma(2.5) / math.gamma(1.75) ** 2              # a_0 of the 1D weights at alpha = 1.5
    taus = [m for m in (10, 20, 40, 80) if prec == 1 or (1.0 / m) ** 2 / (2 * h ** alpha) * a0 <= 0.2]
    us = {m: _run(S, WL.paper_example1(N, alpha, 1.0 / m), prec) for m in sorted(set(taus + [2 * m for m in taus]))}
    for m in taus:
        e64 = O.error1(h, table1_fp64[m], table1_fp64[2 * m])
        e32 = O.error1(h, us[m], us[2 * m])
        bound = 2 * 1e-6 * h * np.linalg.norm(table1_fp64[m])
        assert abs(e32 - e64) <= bound, (prec, m, e32, e64, bound)


def test_paper_table4_alpha15(S):
    alpha, ref = 1.5, 3.9151e-01
    us = [_run(S, WL.paper_example2(N, alpha, 1 / 125), 0) for N in (49, 99)]
    e = O.error2(20.0 / 50, us[0], us[1])
    assert abs(e - ref) <= _half_unit(ref), (e, ref)

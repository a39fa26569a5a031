"""Independent contexts running at the same time through the C ABI.

The header promises that different contexts may be driven concurrently (only
calls on one context must not overlap).  Every form keeps all of its mutable
device state (scratch, state, GEMM dependency counters, error flag) in its own
context, and every kernel's work decomposition is fixed at launch, so a
context's field must not depend on what runs beside it: it must equal, bitwise,
the field of the same context run alone.  Checked for contexts interleaved on
separate CUDA streams of one host thread, and for contexts driven by separate
host threads in a fresh process, where the threads also make the process's
first launches of every kernel at the same time (the per-device launch caches),
together with concurrent calls of the stand-alone split-BF16 GEMM."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2312_06206_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (N, alpha, kappa, tau, g, prec): register path FP32 (N' = 64) and dense
# (N' = 256, cooperative GEMM), FP64 engine, shared-memory engine dense
# (N' = 2048) and FP32 (y sweep on the transpose)
SPECS = [(63, 1.5, 1.0, 0.02, 1, 1), (200, 1.8, 1.3, 0.01, 1, 2), (100, 1.3, 0.9, 0.02, 2, 0),
         (1100, 1.7, 0.8, 1e-3, 2, 2), (1500, 1.4, 0.5, 1e-3, 1, 1)]
STEPS = 6


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_06206_gb300 import build
    build.build()
    from paper_2312_06206_gb300 import sadi
    return sadi


def _make(S, k, stream=None):
    N, al, ka, ta, g, prec = SPECS[k]
    s = S.Sadi(N, al, ka, ta)
    s.set_options(g, prec)
    if stream is not None:
        s.set_stream(stream)
    s.set_initial(WL.gaussian_bumps(N, 4, 700 + k), 0.2 * WL.random_field(N, 800 + k))
    return s


def test_contexts_on_separate_streams_match_solo_runs(S):
    import torch
    want = []
    for k in range(len(SPECS)):
        with _make(S, k) as s:
            s.step(STEPS)
            want.append(s.get()[0])
    streams = [torch.cuda.Stream() for _ in SPECS]
    ctxs = [_make(S, k, st.cuda_stream) for k, st in enumerate(streams)]
    for _ in range(STEPS):          # one step of each in turn: their kernels overlap
        for s in ctxs:
            s.step(1)
    for k, (s, w) in enumerate(zip(ctxs, want)):
        u, n = s.get()
        assert n == STEPS
        assert np.array_equal(u, w), f"context {k} {SPECS[k]} differs when run beside the others"
        s.close()


_THREADS = r"""
import sys, threading
import numpy as np
sys.path.insert(0, ROOT)
import torch
from paper_2312_06206_gb300 import sadi as S, workloads as WL

def make(k):
    N, al, ka, ta, g, prec = SPECS[k]
    s = S.Sadi(N, al, ka, ta)
    s.set_options(g, prec)
    s.set_initial(WL.gaussian_bumps(N, 4, 700 + k), 0.2 * WL.random_field(N, 800 + k))
    return s

def run_ctx(k, out):
    with make(k) as s:
        for _ in range(STEPS):
            s.step(1)
        out[k] = s.get()

GEMMS = [(640, 768, 192), (1024, 1024, 1024), (300, 200, 130)]
dev = torch.device("cuda:0")
ops = []
for j, (M, N, K) in enumerate(GEMMS):
    rng = np.random.default_rng(2000 + j)
    A = torch.from_numpy(rng.standard_normal((M, K)).astype(np.float32)).to(dev)
    B = torch.from_numpy(rng.standard_normal((N, K)).astype(np.float32)).to(dev)
    ops.append((A, B))
torch.cuda.synchronize()

def run_gemm(j, out, stream):
    M, N, K = GEMMS[j]
    A, B = ops[j]
    res = []
    for _ in range(3):
        C = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        S.sadi_gemm_split_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, stream)
        res.append(C.cpu().numpy())
    out[j] = res

ctx_out = [None] * len(SPECS)
gemm_out = [None] * len(GEMMS)
streams = [torch.cuda.Stream() for _ in GEMMS]
errs = []
start = threading.Barrier(len(SPECS) + len(GEMMS))

def guarded(fn, *args):
    try:
        start.wait()
        fn(*args)
    except BaseException as e:
        errs.append(repr(e))

threads = [threading.Thread(target=guarded, args=(run_ctx, k, ctx_out)) for k in range(len(SPECS))]
threads += [threading.Thread(target=guarded, args=(run_gemm, j, gemm_out, streams[j].cuda_stream))
            for j in range(len(GEMMS))]
for t in threads:
    t.start()
for t in threads:
    t.join()
assert not errs, errs

for k in range(len(SPECS)):
    with make(k) as s:
        s.step(STEPS)
        u, n = s.get()
    assert ctx_out[k][1] == n == STEPS, (k, ctx_out[k][1], n)
    assert np.array_equal(ctx_out[k][0], u), ("context", k, SPECS[k])
for j, (M, N, K) in enumerate(GEMMS):
    A, B = ops[j]
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    S.sadi_gemm_split_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, 0)
    want = C.cpu().numpy()
    assert np.isfinite(want).all(), j
    for r in gemm_out[j]:
        assert np.array_equal(r, want), ("gemm", j, GEMMS[j])
print("concurrent threads: ok")
"""


def test_host_threads_on_separate_contexts_in_a_fresh_process(S):
    # a fresh process, so that the threads' first launches of every kernel
    # (the per-device launch caches) happen at the same time
    code = f"ROOT = {ROOT!r}\nSPECS = {SPECS!r}\nSTEPS = {STEPS}\n" + _THREADS
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "concurrent threads: ok" in r.stdout

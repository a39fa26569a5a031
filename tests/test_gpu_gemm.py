"""The split-BF16 tensor-core contraction (sadi_gemm_split_bf16) against an
exact FP64 evaluation of the same three-term split product.

The BF16 rounding of the split is emulated bit-exactly in numpy
(round-to-nearest-even on the upper 16 bits of the FP32 pattern), so the only
difference left is the FP32 accumulation of the tensor cores, whose rounding
error grows like sqrt(K): the tolerance is 1e-5 of the largest |C| for
K <= 1024, scaled by sqrt(K / 1024) above.  For K <= 1024 it is far below
the size of either cross term (about 2^-9 relative), so a dropped or swapped
term fails; the long-K case checks the staging ring over many K blocks."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_06206_gb300 import build
    build.build()
    from paper_2312_06206_gb300 import sadi
    return sadi, torch


def bf16_round(x):
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, dtype=np.float32)
    hi = bf16_round(x)
    lo = bf16_round(x - hi)
    return hi.astype(np.float64), lo.astype(np.float64)


def test_bf16_emulation_matches_known_values():
    # 1 + 2^-8 lies halfway between BF16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e-3], dtype=np.float32)
    r = bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -6 and r[3] == -2.5
    assert abs(r[4] - 3.0e-3) <= 2.0 ** -8 * 3.0e-3


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 200, 130), (1, 1, 1), (1024, 1024, 1024),
                                   (256, 512, 4096), (640, 768, 192)])
def test_split_bf16_gemm_matches_exact_split_product(env, M, N, K):
    S, torch = env
    rng = np.random.default_rng(1000 + M + 7 * N + 13 * K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = (rng.standard_normal((N, K)) * rng.uniform(0.1, 10.0, size=(N, 1))).astype(np.float32)
    dev = torch.device("cuda:0")
    tA, tB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    tC = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    S.sadi_gemm_split_bf16(tA.data_ptr(), tB.data_ptr(), tC.data_ptr(), M, N, K)
    C = tC.cpu().numpy().astype(np.float64)
    ah, al = split(A)
    bh, bl = split(B)
    want = ah @ bh.T + ah @ bl.T + al @ bh.T
    scale = np.abs(want).max()
    assert np.isfinite(C).all()
    tol = 1e-5 * max(1.0, np.sqrt(K / 1024.0))
    assert np.abs(C - want).max() <= tol * scale
    # and against the exact product: the split keeps about 16 bits
    exact = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.abs(C - exact).max() <= 1e-4 * np.abs(exact).max()
    # the cross terms are resolved (a hi-only product is visibly worse)
    if 64 <= K <= 1024:
        assert np.abs(ah @ bh.T - want).max() > 20 * np.abs(C - want).max()

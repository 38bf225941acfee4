"""The BF16 tensor-core GEMM (as_gemm_bf16) against float64 products of the same bf16 values.

Products of two bf16 numbers are exact in float32, so the only difference from the float64 sum is
float32 accumulation: the bound |D - D64| <= (K + 2) * eps32 * sum_k |A_mk B_nk| is written in the
test. A layout probe (unit vectors through one tile) names the element that lands wrong if the
shared-memory operand layout or the accumulator lanes were misread.
"""
import numpy as np
import pytest

from paper_2101_05844_gb300 import binding

pytestmark = pytest.mark.gpu
EPS32 = np.finfo(np.float32).eps


def _run(M, N, K, bn, seed, lda_pad=0, ldb_pad=0):
    torch = pytest.importorskip("torch")
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(M, K + lda_pad, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K + ldb_pad, generator=g).to(torch.bfloat16)
    Ad, Bd = A.cuda(), B.cuda()
    D = torch.full((M, N), float("nan"), device="cuda")
    st = binding.gemm_bf16(Ad[:, :K], Bd[:, :K], D, bn=bn)
    assert st == 0, st
    a = A[:, :K].double().numpy()
    b = B[:, :K].double().numpy()
    ref = a @ b.T
    bound = (K + 2) * EPS32 * (np.abs(a) @ np.abs(b).T)
    err = np.abs(D.cpu().double().numpy() - ref)
    assert np.isfinite(D.cpu().numpy()).all()
    assert (err <= bound).all(), (float(err.max()), np.unravel_index(err.argmax(), err.shape))


def test_layout_probe_one_tile():
    """A = unit rows, B = distinct integers: D[m][n] = B[n][m], so every misplaced element shows."""
    torch = pytest.importorskip("torch")
    M, N, K = 128, 32, 64
    A = torch.zeros(M, K)
    for m in range(M):
        A[m, m % K] = 1.0
    B = torch.arange(N * K, dtype=torch.float32).reshape(N, K) % 251   # exact in bf16
    Ad, Bd = A.to(torch.bfloat16).cuda(), B.to(torch.bfloat16).cuda()
    D = torch.zeros(M, N, device="cuda")
    assert binding.gemm_bf16(Ad, Bd, D, bn=32) == 0
    got = D.cpu()
    want = torch.stack([B[:, m % K] for m in range(M)])
    bad = (got != want).nonzero()
    assert bad.numel() == 0, f"{len(bad)} wrong; first {bad[:8].tolist()}: got {[float(got[i, j]) for i, j in bad[:8].tolist()]}"


@pytest.mark.parametrize("M,N,K,bn", [(128, 32, 64, 32), (256, 64, 128, 64), (300, 100, 200, 128),
                                      (1000, 256, 576, 256), (64, 48, 24, 64), (777, 33, 1032, 32),
                                      (384, 512, 8192, 64), (130, 40, 320, 128), (129, 8, 4104, 256)])
def test_matches_float64_within_accumulation_bound(M, N, K, bn):
    _run(M, N, K, bn, seed=M + N + K)


def test_row_strides_larger_than_k():
    _run(200, 64, 96, 64, seed=5, lda_pad=32, ldb_pad=16)


def test_bad_arguments_are_rejected():
    torch = pytest.importorskip("torch")
    A = torch.zeros(16, 12, dtype=torch.bfloat16, device="cuda")   # K = 12: not a multiple of 8
    B = torch.zeros(16, 12, dtype=torch.bfloat16, device="cuda")
    D = torch.zeros(16, 16, device="cuda")
    assert binding.gemm_bf16(A, B, D) == 1
    A = torch.zeros(16, 16, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(16, 16, dtype=torch.bfloat16, device="cuda")
    assert binding.gemm_bf16(A, B, D, bn=48) == 1

"""The chain's GEMM kernels against a float64 matmul (tcgen05 bf16 / 3xtf32, SIMT fp32)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2208_05740_gb300 import build, gcp
    build.build()
    return gcp


SHAPES = [(128, 128, 64), (300, 200, 784), (9216, 256, 256), (257, 130, 40), (1, 16, 8), (640, 784, 256)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tcgen05_tf32x3_matches_float64(g, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32) / np.sqrt(K)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    C = g.selftest_gemm(1, A, B)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    assert np.max(np.abs(C - ref) / np.maximum(scale, 1e-30)) < 4e-6
    C32 = g.selftest_gemm(2, A, B)
    assert np.max(np.abs(C32 - ref) / np.maximum(scale, 1e-30)) < 4e-6


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tcgen05_bf16_matches_bf16_inputs(g, M, N, K):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7 * M + N + K)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32) / np.sqrt(K)
    Ab = torch.tensor(A).to(torch.bfloat16).to(torch.float64).numpy()
    Bb = torch.tensor(B).to(torch.bfloat16).to(torch.float64).numpy()
    ref = Ab @ Bb.T
    C = g.selftest_gemm(0, A, B)
    scale = np.abs(Ab) @ np.abs(Bb).T
    assert np.max(np.abs(C - ref) / np.maximum(scale, 1e-30)) < 1e-5

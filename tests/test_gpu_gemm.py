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
# shapes whose products take 224-column tiles (fewer waves):
# the MLP's backward product onto its 784-wide input layer, and a ragged one
WIDE = [(9216, 784, 256), (9100, 780, 104)]


@pytest.mark.parametrize("M,N,K", SHAPES + WIDE)
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


@pytest.mark.parametrize("M,N,K", SHAPES + WIDE)
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


F64_SHAPES = [(300, 200, 256), (130, 784, 256), (64, 96, 1024), (37, 20, 16), (9, 33, 784)]


@pytest.mark.parametrize("M,N,K", F64_SHAPES)
def test_f64_slices_product_within_its_bound(g, M, N, K):
    """The certification's float64 product on the tensor cores (exact bf16
    slices): on sampled entries the exact rational product lies within the
    reported bound cerr * Cabs, and every entry agrees with numpy's float64
    product within that bound plus numpy's rounding. Rows at scales
    1e-3 .. 1e3, 10% zeros and an all-zero row."""
    from fractions import Fraction
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.normal(size=(M, K)) * 10.0 ** rng.uniform(-3, 3, size=(M, 1))
    A[rng.random((M, K)) < 0.1] = 0.0
    A[0] = 0.0
    B = rng.normal(size=(N, K)) / np.sqrt(K)
    C, Cabs, cerr = g.selftest_gemm_f64(A, B)
    assert 0.0 < cerr < 1e-13
    scale = np.abs(A) @ np.abs(B).T
    # against numpy's float64 product: the bound plus numpy's own rounding
    assert np.all(np.abs(C - A @ B.T) <= cerr * Cabs + K * 2.0 ** -52 * scale)
    assert np.all(C[0] == 0.0)
    pick = [(0, 0)] + [(int(rng.integers(0, M)), int(rng.integers(0, N))) for _ in range(40)]
    for r, c in pick:
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(A[r].tolist(), B[c].tolist()))
        assert abs(Fraction(float(C[r, c])) - exact) <= Fraction(cerr) * Fraction(float(Cabs[r, c])), (r, c)


def test_f64_slices_product_non_finite_and_extreme_rows(g):
    """Rows with NaN or inf give NaN (error scale inf); rows of subnormal and
    of very large numbers keep their exact products within the bound."""
    A = np.ones((7, 64))
    A[2, 7] = np.nan
    A[3, 1] = np.inf
    A[5] = 3e-310          # subnormal
    A[6] = 1e300
    B = np.ones((4, 64))
    B[3] = 0.5
    C, Cabs, cerr = g.selftest_gemm_f64(A, B)
    assert np.all(np.isnan(C[2])) and np.all(np.isnan(C[3])) and np.all(np.isinf(Cabs[2:4]))
    np.testing.assert_array_equal(C[[0, 1, 4], :3], 64.0)
    np.testing.assert_array_equal(C[[0, 1, 4], 3], 32.0)
    for r in (5, 6):
        exact = A[r] @ B.T          # sums of equal terms: exact in float64 here
        assert np.all(np.abs(C[r] - exact) <= cerr * Cabs[r].astype(np.float64)), r

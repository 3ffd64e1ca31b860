"""GPU symmetric eigensolvers (the k x k step of Algorithm 3) against LAPACK.

Tolerances: eigenvalues to 50 k eps ||K|| (absolute; both methods are
backward stable), eigen-residual ||K z - lambda z|| <= 50 k eps ||K||,
orthonormality ||Z^T Z - I||_max <= 1e-12.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _spd(k, lo, hi, seed, mult=None):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    lam = np.exp(rng.uniform(np.log(lo), np.log(hi), k))
    if mult:
        lam[:mult] = lam[0]
    return (Q * lam) @ Q.T


def _run(R, K, method):
    k = K.shape[0]
    Kt = torch.tensor(np.asfortranarray(K).T.copy(), device=DEV)   # column-major = K^T row-major
    lam = torch.empty(k, dtype=torch.float64, device=DEV)
    Z = torch.empty(k, k, dtype=torch.float64, device=DEV)
    R.riot_symm_eig(Kt, lam, Z, method)
    return lam.cpu().numpy(), Z.cpu().numpy().T                  # columns = eigenvectors


# k = 700 takes the tridiagonalisation whose columns stream from L2 (more columns than warps)
CASES = [("graded", 7, 1e-6, 1e6, 0), ("graded", 40, 1e-8, 1e4, 1), ("graded", 100, 1e-3, 1e3, 2),
         ("graded", 512, 1e8, 1e20, 3), ("cluster", 64, 1.0, 10.0, 4), ("cluster", 301, 0.5, 2.0, 5),
         ("graded", 700, 1e-3, 1e3, 6)]


# the tridiagonal solver (method 0) on every case; parallel Jacobi (method 1), the slow
# reference method, on the cases up to k = 128
METHOD_CASES = [(m,) + c for m in (0, 1) for c in CASES if m == 0 or c[1] <= 128]


@pytest.mark.parametrize("method,kind,k,lo,hi,seed", METHOD_CASES)
def test_symm_eig_against_lapack(gpu_lib, method, kind, k, lo, hi, seed):
    R = gpu_lib
    K = _spd(k, lo, hi, seed, mult=(k // 4 if kind == "cluster" else None))
    K = 0.5 * (K + K.T)
    ref = np.sort(np.linalg.eigvalsh(K))[::-1]
    lam, Z = _run(R, K, method)
    nrm = np.abs(ref).max()
    tol = 50 * k * np.finfo(float).eps * nrm
    np.testing.assert_allclose(lam, ref, rtol=0, atol=tol)
    assert np.abs(K @ Z - Z * lam).max() <= tol
    assert np.abs(Z.T @ Z - np.eye(k)).max() <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 33])
def test_symm_eig_degenerate(gpu_lib, k):
    R = gpu_lib
    for K in (np.eye(k), np.zeros((k, k)), np.diag(np.arange(k, dtype=float))):
        lam, Z = _run(R, K, 0)
        np.testing.assert_allclose(lam, np.sort(np.linalg.eigvalsh(K))[::-1], atol=1e-14)
        assert np.abs(Z.T @ Z - np.eye(k)).max() <= 1e-12
        assert np.abs(K @ Z - Z * lam).max() <= 1e-13


def test_symm_eig_block_diagonal_splits(gpu_lib):
    """Independent blocks make T split into unreduced blocks (zero off-diagonals at
    the block boundaries); k > 1024 spreads the split flags over two tiles of the
    split kernel's prefix count.  Same tolerances as above."""
    R = gpu_lib
    sizes = [1, 5, 300, 2, 700, 94, 1, 97]
    k = sum(sizes)
    K = np.zeros((k, k))
    o = 0
    for b, m in enumerate(sizes):
        K[o:o + m, o:o + m] = _spd(m, 0.1 * (b + 1), 10.0 * (b + 1), 40 + b)
        o += m
    K = 0.5 * (K + K.T)
    ref = np.sort(np.linalg.eigvalsh(K))[::-1]
    lam, Z = _run(R, K, 0)
    tol = 50 * k * np.finfo(float).eps * np.abs(ref).max()
    np.testing.assert_allclose(lam, ref, rtol=0, atol=tol)
    assert np.abs(K @ Z - Z * lam).max() <= tol
    assert np.abs(Z.T @ Z - np.eye(k)).max() <= 1e-12


def test_refined_reciprocal_within_one_ulp_and_faster(gpu_lib):
    """The reciprocal on the FP64 chains (Cholesky pivots, the inverse iteration's LU, the
    Householder reflectors): the hardware approximation refined by one third-order Newton
    step must stay within one ulp of the correctly rounded 1 / x over 2^24 inputs spanning
    the double range (and its limits), and must be shorter on the chain than the division."""
    p = gpu_lib.riot_measure_peaks(0)
    assert p["fp64_rcp_fast_max_ulps"] <= 1.0
    assert 0.0 < p["fp64_rcp_fast_cycles"] < p["fp64_div_cycles"]
    assert p["fp64_fma_cycles"] > 0.0 and p["fp64_tflops"] > 0.0 and p["fp32_tflops"] > p["fp64_tflops"]

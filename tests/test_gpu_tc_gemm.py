"""The tcgen05 sketch GEMM against an FP64 reference (PyTorch CPU matmul of
the same FP32 inputs).  Three BF16 terms per value and the six leading term
products reproduce the FP32 products to ~2^-24 relative; accumulating K of
them in FP32 adds a random-walk error of ~K^(1/2) 2^-24 of the result scale
(||op(A)|| ||op(B)|| / K^(1/2) for these Gaussian inputs).  Required: twice
that, plus 1e-6."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.mark.parametrize("ta,tb,m,n,k", [
    ("T", "N", 512, 512, 4096),     # Q^T W of the large Lorenz-96 sketch
    ("N", "N", 4096, 512, 512),     # U = Q Z
    ("N", "T", 300, 200, 1000),     # ragged tiles and K chunks
    ("T", "T", 17, 33, 5),          # smaller than one tile and one chunk
    ("N", "N", 128, 128, 64),       # exactly one tile, one chunk
])
def test_tc_sgemm_matches_fp64(gpu_lib, ta, tb, m, n, k):
    R = gpu_lib
    g = torch.Generator().manual_seed(m * 7 + n * 3 + k)
    Ah = torch.randn((k, m) if ta == "T" else (m, k), generator=g, dtype=torch.float32)
    Bh = torch.randn((n, k) if tb == "T" else (k, n), generator=g, dtype=torch.float32)
    Ch = torch.randn(m, n, generator=g, dtype=torch.float32)
    # column-major storage: a (rows, cols) matrix is a (cols, rows) row-major tensor
    A = Ah.T.contiguous().to(DEV)
    B = Bh.T.contiguous().to(DEV)
    C = Ch.T.contiguous().to(DEV)
    alpha, beta = 1.5, -0.5
    lda, ldb = Ah.shape[0], Bh.shape[0]
    R.riot_tc_sgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, m)
    opA = (Ah.T if ta == "T" else Ah).double()
    opB = (Bh.T if tb == "T" else Bh).double()
    ref = alpha * opA @ opB + beta * Ch.double()
    got = C.cpu().T.double()
    err = float((got - ref).norm() / (abs(alpha) * opA.norm() * opB.norm() / np.sqrt(k) + abs(beta) * Ch.norm()))
    assert err <= 2 * np.sqrt(k) * 2.0 ** -24 + 1e-6, err

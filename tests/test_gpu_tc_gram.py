"""The tensor-core Gram of the mixed-precision CholeskyQR (G = Y^T Y, lower
triangle, FP64 result from FP32 Y) through riot_tc_gram.

1. Values of at most 15 significant bits relative to their column's largest
   magnitude (y = (128 a + b) 2^(e - 14), |a| <= 127, |b| <= 63) are split
   without remainder into two slices, so the result must equal the exact
   integer Gram bit for bit: this checks that the tensor cores accumulate the
   slice products without rounding, at the largest slice magnitudes.
2. Gaussian columns with norms spread over six decades against the FP64 Gram
   of the same FP32 values: the truncation below 2^-36 of the column maximum
   and the slice products left out (weights 2^-49 and below, products below
   2^13) bound each entry's error by n 2^(e_i + e_j - 33) (with
   2^(e_j - 1) <= max|y_j| < 2^e_j).  Off the diagonal the dropped terms have
   random signs and the error is ~n^(1/2) 2^-38 2^(e_i + e_j), about
   1.7e-10 n^(-1/2) rms of sqrt(G_ii G_jj) for these columns: 3e-9 n^(-1/2)
   is required.  The diagonal is an FP64 sum of squares: 1e-13.
3. A column holding NaN or Inf poisons its row and column only; an all-zero
   column gives zeros; the strict upper triangle is never written."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _run(R, Yh, sentinel=7.0):
    n, k = Yh.shape
    Y = torch.tensor(Yh.T.copy(), device=DEV)          # column-major n x k
    G = torch.full((k, k), sentinel, dtype=torch.float64, device=DEV)
    R.riot_tc_gram(n, k, Y, max(n, 1), G, k)
    return G.cpu().numpy().T                            # G[i, j] in numpy indexing


@pytest.mark.parametrize("n,k,seed", [(4096, 512, 1), (1000, 200, 2), (31, 7, 3), (5000, 130, 4)])
def test_gram_exact_on_short_values(gpu_lib, n, k, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(-127, 128, size=(n, k))
    a[: n // 2] = np.where(rng.random((n // 2, k)) < 0.5, 127, -127)   # largest slices, both signs
    a[0] = 127
    b = rng.integers(-63, 64, size=(n, k))
    v = 128 * a + b                                     # |v| < 2^14
    e = rng.integers(-20, 21, size=k)
    Yh = (v * np.ldexp(1.0, e - 14)[None, :]).astype(np.float32)
    assert np.array_equal(Yh.astype(np.float64), v * np.ldexp(1.0, e - 14)[None, :])
    got = _run(gpu_lib, Yh)
    exact_int = v.T.astype(np.int64) @ v.astype(np.int64)
    want = exact_int * np.ldexp(1.0, e[:, None] + e[None, :] - 28)
    lo = np.tril_indices(k)
    np.testing.assert_array_equal(got[lo], want[lo])
    assert np.all(got[np.triu_indices(k, 1)] == 7.0)


@pytest.mark.parametrize("n,k", [(4096, 512), (777, 300), (64, 33)])
def test_gram_gaussian_matches_fp64(gpu_lib, n, k):
    rng = np.random.default_rng(n + k)
    Yh = (rng.standard_normal((n, k)) * np.logspace(-3, 3, k)[None, :]).astype(np.float32)
    got = _run(gpu_lib, Yh)
    Yd = Yh.astype(np.float64)
    ref = Yd.T @ Yd
    lo = np.tril_indices(k)
    mx = np.abs(Yd).max(axis=0)
    e = np.frexp(mx)[1]
    bound = n * np.ldexp(1.0, e[:, None] + e[None, :] - 33)
    err = np.abs(got - ref)
    assert np.all(err[lo] <= bound[lo])
    d = np.sqrt(np.diag(ref))
    rel = err / np.outer(d, d)
    off = np.tril_indices(k, -1)
    assert rel[off].max() < 3e-9 / np.sqrt(n), rel[off].max()
    assert np.diag(rel).max() < 1e-13
    assert np.all(got[np.triu_indices(k, 1)] == 7.0)


def test_gram_special_columns(gpu_lib):
    n, k = 300, 40
    rng = np.random.default_rng(9)
    Yh = rng.standard_normal((n, k)).astype(np.float32)
    Yh[:, 3] = 0.0
    Yh[17, 10] = np.nan
    Yh[5, 25] = np.inf
    got = _run(gpu_lib, Yh)
    lo = np.zeros((k, k), dtype=bool)
    lo[np.tril_indices(k)] = True
    bad = np.zeros(k, dtype=bool)
    bad[[10, 25]] = True
    poisoned = (bad[:, None] | bad[None, :]) & lo
    assert np.all(np.isnan(got[poisoned]))
    clean = lo & ~poisoned
    Yd = np.where(np.isfinite(Yh), Yh, 0).astype(np.float64)
    ref = Yd.T @ Yd
    d = np.sqrt(np.maximum(np.diag(ref), 1e-300))
    assert np.all(np.abs(got - ref)[clean] <= 3e-9 / np.sqrt(n) * np.outer(d, d)[clean])
    assert np.all(got[3, :4] == 0.0) and np.all(got[3:, 3][~bad[3:]] == 0.0)


def test_gram_empty_rows(gpu_lib):
    got = _run(gpu_lib, np.zeros((0, 20), dtype=np.float32))
    assert np.all(got[np.tril_indices(20)] == 0.0)

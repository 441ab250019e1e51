"""The numerical fact behind the GPU form of the Appendix estimator (CPU
only, numpy; nothing here calls the library or the oracle).

The estimator applies D = A - U diag(S) V^T and then D^T.  In FP32 the
product D^T D w has to be formed that way: expanding it into A^T A w minus
the rank-k terms subtracts quantities of size ||A||^2 to obtain ||D||^2,
which is lost once ||D|| < sqrt(u32) ||A||.  Shown on the paper's first test
matrix (Section 6.1 spectrum, DCT-II factors) at k = 32.
"""
import numpy as np


def _dct2(n):
    """Orthonormal DCT-II matrix (rows are the basis vectors)."""
    j = np.arange(n)[:, None]
    x = np.arange(n)[None, :]
    E = np.cos(np.pi * j * (2 * x + 1) / (2 * n)) * np.sqrt(2.0 / n)
    E[0] /= np.sqrt(2.0)
    return E


def _first_example(n):
    """The paper's first test matrix (Section 6.1 spectrum) on DCT-II factors."""
    j = np.arange(1, n + 1, dtype=np.float64)
    S = np.where(j <= 20, 10.0 ** (-4 * (j - 1) / 19), 1e-4 / np.maximum(j - 20, 1) ** 0.1)
    E = _dct2(n)
    return (E.T * S[None, :]) @ E, S


def test_dct2_is_orthonormal():
    E = _dct2(64)
    assert np.abs(E @ E.T - np.eye(64)).max() < 1e-13


def test_fp32_estimator_needs_d_then_dt():
    n, k = 256, 32
    A, S = _first_example(n)
    E = _dct2(n)
    U, V = E.T[:, :k], E.T[:, :k]            # exact top-k singular vectors (A is symmetric PSD)
    rng = np.random.default_rng(3)
    w = rng.standard_normal(n)
    w /= np.linalg.norm(w)
    D = A - (U * S[:k]) @ V.T
    exact = np.linalg.norm(D.T @ (D @ w))     # FP64 truth, about sigma_{k+1}^2
    assert 0.1 * S[k] ** 2 < exact <= S[k] ** 2 * (1 + 1e-12)
    A32, U32, V32, S32, w32 = (x.astype(np.float32) for x in (A, U, V, S[:k], w))
    # D then D^T, every product in FP32
    y = A32 @ w32 - U32 @ (S32 * (V32.T @ w32))
    z = A32.T @ y - V32 @ (S32 * (U32.T @ y))
    two_step = np.linalg.norm(z.astype(np.float64))
    # A^T A w first, the rank-k terms subtracted afterwards, in FP32
    AtAw = A32.T @ (A32 @ w32)
    fused = AtAw - (A32.T @ U32) @ (S32 * (V32.T @ w32)) - V32 @ (S32 * (U32.T @ (A32 @ w32))) \
        + V32 @ (S32 * ((U32.T @ U32) @ (S32 * (V32.T @ w32))))
    fused_n = np.linalg.norm(fused.astype(np.float64))
    assert abs(two_step - exact) < 1e-2 * exact
    assert abs(fused_n - exact) > 0.5 * exact          # the expanded form has lost ||D||^2 (measured: 119 %)


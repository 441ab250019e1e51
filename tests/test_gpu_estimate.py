"""The Appendix error estimate p_{j,q}(D), D = A - U S V^T, on the GPU
(rpca_estimate_error), against the FP64 oracle's power method from the same
start vectors, and the adaptive rank (rpca_run_adaptive) on the paper's
first example (DCT-II factors, Section 6.1), where the optimum rank-k error
is sigma_{k+1}."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as est  # noqa: E402
from synth import generators as gen  # noqa: E402

pytestmark = pytest.mark.gpu


def R():
    from paper_1007_5510_gb300 import rpca
    rpca.load_library()
    return rpca


def _start(n, q, seed):
    # the oracle draws its start vectors one column after the other
    rng = np.random.default_rng(seed)
    return np.stack([rng.standard_normal(n) for _ in range(q)], axis=1), seed


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-4), ("bf16", 2e-2)])
def test_estimate_matches_oracle_power_method(dtype, tol):
    rpca = R()
    m, n, k = 3000, 500, 10
    sig = np.concatenate([np.arange(1, 31) ** -1.0, 1e-3 * np.ones(470)])
    A64 = gen.lowrank_np(m, n, sig, seed=21)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    A = torch.from_numpy(A64).cuda().to(tdt)
    Ao = A.double().cpu().numpy()
    U, S, V = rpca.pca(A, k, k + 2, 1, seed=3)
    torch.cuda.synchronize()
    q, j = 4, 6
    omega, s = _start(n, q, 17)
    p_gpu, cols = rpca.estimate_error(A, U, S, V, j=j, q=q, omega=omega)
    Uh, Vh, Sh = U.double().cpu().numpy(), V.double().cpu().numpy(), S.cpu().numpy()
    D, Dt = est.residual_operators(Ao, Uh, Sh, Vh)
    p_or = est.power_estimate(D, Dt, n, j=j, k=q, rng=np.random.default_rng(s))
    true = est.spectral_error(Ao, Uh, Sh, Vh)
    print("PARITY estimate %s p_gpu %.6e p_oracle %.6e rel %.2e true %.6e" % (dtype, p_gpu, p_or,
                                                                               abs(p_gpu - p_or) / p_or, true))
    assert abs(p_gpu - p_or) <= tol * p_or
    assert len(cols) == q and max(cols) == pytest.approx(p_gpu)
    # Appendix: p <= ||D||, and within a factor of two with high probability
    assert p_gpu <= true * (1 + max(tol, 1e-6)) and p_gpu >= true / 2


def test_estimate_default_start_vectors_are_reproducible():
    rpca = R()
    A64 = gen.lowrank_np(2000, 300, np.arange(1, 301) ** -1.5, seed=5)
    A = torch.from_numpy(A64.astype(np.float32)).cuda()
    U, S, V = rpca.pca(A, 8, 10, 1, seed=1)
    p1, _ = rpca.estimate_error(A, U, S, V, seed=9)
    p2, _ = rpca.estimate_error(A, U, S, V, seed=9)
    # same start vectors; the passes' FP32 atomics add in no fixed order
    assert abs(p1 - p2) <= 1e-5 * p1
    true = est.spectral_error(A.double().cpu().numpy(), U.double().cpu().numpy(), S.cpu().numpy(),
                              V.double().cpu().numpy())
    assert true / 2 <= p1 <= true * (1 + 1e-4)


def _dct_example1(n):
    scipy_fft = pytest.importorskip("scipy.fft")
    j = np.arange(1, n + 1, dtype=np.float64)
    S = np.where(j <= 20, 10.0 ** (-4 * (j - 1) / 19), 1e-4 / np.maximum(j - 20, 1) ** 0.1)
    E = scipy_fft.dct(np.eye(n), type=2, norm="ortho", axis=0)
    return (E * S[None, :]) @ E.T, S


def test_adaptive_rank_on_the_first_example():
    """tol = 2e-4 between sigma_17 = 4.3e-4 and sigma_33 = 7.7e-5: doubling
    from k = 4 stops at k = 32 (errors at the optimum, Tables 1a/1b)."""
    rpca = R()
    A64, S = _dct_example1(1024)
    A = torch.from_numpy(A64.astype(np.float32)).cuda()
    U, Sg, V, k, eps = rpca.pca_adaptive(A, 2e-4, 4, 64, oversample=2, i=3, seed=2010)
    torch.cuda.synchronize()
    print("PARITY adaptive rank k %d eps %.3e sigma_k+1 %.3e" % (k, eps, S[k]))
    assert k == 32
    assert eps <= 2e-4
    assert S[k] / 2 <= eps <= S[k] * 1.1
    true = est.spectral_error(A64, U.double().cpu().numpy(), Sg.cpu().numpy(), V.double().cpu().numpy())
    assert true <= 1.1 * S[k]
    # the rank before it (16) misses the tolerance: sigma_17 = 4.3e-4
    assert S[16] > 2e-4

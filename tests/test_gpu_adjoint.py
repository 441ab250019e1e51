"""Adjoint of the computed singular values (rpca_backward, G fixed).

Pinned to central differences of the FP64 oracle's singular values (same
Philox G), on the exact case w = n (8 x 6, 40 x 30) and a randomised one
(40 x 30, w = 12 < n); the exact case also against autograd through a dense
SVD; FP32 against FP64; the autograd wrapper against the direct call.
Losses: L1 = sum_j sigma_j, L2 = ||A - U S V^T||_F^2 = ||A||_F^2 - sum_j sigma_j^2."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rpca_oracle as ro  # noqa: E402

pytestmark = pytest.mark.gpu


def R():
    from paper_1007_5510_gb300 import rpca
    rpca.load_library()
    return rpca


def _gpu_grad(A, k, l, i, seed, loss, dtype=torch.float64):
    rpca = R()
    At = torch.from_numpy(A).to(dtype).cuda()
    code = rpca.F64 if dtype == torch.float64 else rpca.F32
    obj = rpca.PCA(A.shape[0], A.shape[1], k, l, i, code, seed=seed, adjoint=True)
    try:
        U, S, V = obj.run(At)
        s = S.cpu().numpy()
        dS = np.ones(k) if loss == "L1" else -2.0 * s
        dA = obj.backward(At, dS).cpu().double().numpy()
    finally:
        obj.close()
    if loss == "L2":
        dA = dA + 2.0 * A
    return dA, s


def _oracle_loss(A, k, l, i, seed, loss):
    _, S, _ = ro.rpca(A, k, l, i, seed=seed, normalize=True)
    return S.sum() if loss == "L1" else float((A * A).sum() - (S * S).sum())


def _fd(A, k, l, i, seed, loss, D, h):
    return (_oracle_loss(A + h * D, k, l, i, seed, loss) - _oracle_loss(A - h * D, k, l, i, seed, loss)) / (2 * h)


@pytest.mark.parametrize("loss", ["L1", "L2"])
def test_adjoint_fd_8x6_all_entries(loss):
    rng = np.random.default_rng(8)
    A = rng.standard_normal((8, 6))
    k, l, i, seed = 2, 3, 1, 21                  # w = 6 = n: the exact truncated SVD
    dA, _ = _gpu_grad(A, k, l, i, seed, loss)
    h = 1e-6 * np.abs(A).max()
    fd = np.zeros_like(A)
    for r in range(8):
        for c in range(6):
            D = np.zeros_like(A)
            D[r, c] = 1.0
            fd[r, c] = _fd(A, k, l, i, seed, loss, D, h)
    assert np.abs(dA - fd).max() <= 1e-6 * np.abs(fd).max()


@pytest.mark.parametrize("k,l,i,loss", [(4, 15, 1, "L1"), (4, 6, 1, "L1"), (4, 6, 1, "L2"), (3, 5, 2, "L1")])
def test_adjoint_fd_40x30_directions(k, l, i, loss):
    rng = np.random.default_rng(40 + l + i)
    A = rng.standard_normal((40, 30)) @ np.diag(0.8 ** np.arange(30))
    seed = 33
    dA, _ = _gpu_grad(A, k, l, i, seed, loss)
    h = 1e-6 * np.abs(A).max()
    errs, mags = [], []
    for _ in range(64):
        D = rng.standard_normal(A.shape)
        fd = _fd(A, k, l, i, seed, loss, D, h)
        errs.append(abs(float((dA * D).sum()) - fd))
        mags.append(abs(fd))
    assert max(errs) <= 1e-6 * max(mags), (max(errs), max(mags))


def test_adjoint_exact_case_matches_dense_svd_autograd():
    """w = n: the method returns the exact truncated SVD, so the gradient of
    sum_{j<=k} sigma_j is U_k V_k^T, as autograd through a dense SVD gives."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((40, 30))
    k, l, i = 4, 15, 1
    dA, _ = _gpu_grad(A, k, l, i, 5, "L1")
    At = torch.from_numpy(A).requires_grad_(True)
    torch.linalg.svdvals(At)[:k].sum().backward()
    assert np.abs(dA - At.grad.numpy()).max() < 1e-9


def test_adjoint_fp32_matches_fp64():
    rng = np.random.default_rng(12)
    m, n, k, l, i = 20_000, 300, 10, 12, 2
    A = (rng.standard_normal((m, 40)) @ (rng.standard_normal((40, n)) * 0.9 ** np.arange(40)[:, None])
         + 1e-2 * rng.standard_normal((m, n)))
    A = A.astype(np.float32).astype(np.float64)
    d64, s64 = _gpu_grad(A, k, l, i, 3, "L1", torch.float64)
    d32, s32 = _gpu_grad(A, k, l, i, 3, "L1", torch.float32)
    assert np.abs(d32 - d64).max() <= 1e-4 * np.abs(d64).max()


def test_autograd_wrapper_matches_direct_call():
    rpca = R()
    rng = np.random.default_rng(2)
    A = rng.standard_normal((3000, 200))
    At = torch.from_numpy(A).cuda().requires_grad_(True)
    U, S, V = rpca.pca_autograd(At, 6, 8, 1, seed=4)
    loss = (At * At).sum() - (S * S).sum()
    loss.backward()
    direct, _ = _gpu_grad(A, 6, 8, 1, 4, "L2")
    assert np.abs(At.grad.cpu().numpy() - direct).max() <= 1e-10 * np.abs(direct).max()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_adjoint_matches_single_problems(dtype):
    """rpca_batch_backward over uneven problems equals rpca_backward of each
    problem on its own (which the FD and dense-SVD pins above cover)."""
    rpca = R()
    rng = np.random.default_rng(41)
    shapes = [(int(rng.integers(200, 3000)), int(rng.integers(30, 150))) for _ in range(7)]
    k, l, i = 4, 8, 1
    tdt = torch.float64 if dtype == "f64" else torch.float32
    code = rpca.F64 if dtype == "f64" else rpca.F32
    As = [torch.from_numpy(rng.standard_normal((m, n)) @ np.diag(0.9 ** np.arange(n))).to(tdt).cuda()
          for m, n in shapes]
    b = rpca.Batch(shapes, k, l, i, dtype=code, seeds=range(10, 10 + len(shapes)), nstreams=3, adjoint=True)
    try:
        outs = b.run(As)
        dSs = [torch.ones(k, dtype=torch.float64, device="cuda") for _ in shapes]
        dAs = b.backward(As, dSs)
        torch.cuda.synchronize()
        for p, (m, n) in enumerate(shapes):
            obj = rpca.PCA(m, n, k, l, i, code, seed=10 + p, adjoint=True)
            try:
                obj.run(As[p])
                ref = obj.backward(As[p], np.ones(k))
            finally:
                obj.close()
            e = float((dAs[p] - ref).abs().max() / ref.abs().max())
            assert e < (1e-12 if dtype == "f64" else 1e-5), (p, e)
    finally:
        b.close()

"""Bounded device-side waits: a wait that expires ends the kernel early, the
call reports RPCA_ETIMEOUT, and the device stays usable.

The expiry is made safely: the test hook leaves one TMA stage of the first
CTA unissued, so nothing is in flight for it and the consumer's wait on it
can only run out (limit 20 ms instead of 2 s).  Every other copy and MMA of
the launch completes before its CTA exits.  Each case then runs the same
call normally and checks the result against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import rpca_oracle as ro  # noqa: E402
from synth import generators as gen  # noqa: E402

LIMIT_NS = 20_000_000


@pytest.fixture()
def R():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1007_5510_gb300 import rpca
    rpca.load_library()
    yield rpca
    # whatever happened, no later launch inherits an armed hook
    rpca.arm_wait_expiry(0, 2_000_000_000, -1)
    rpca.arm_wait_expiry(1, 2_000_000_000, -1)


def _rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max())


def _bf16(rng, m, n):
    A = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda().to(torch.bfloat16)
    return A, A.float().cpu().double().numpy()


def test_t_pass_wait_expiry_then_normal_call(R):
    rng = np.random.default_rng(1)
    m, n, w = 20_000, 512, 66
    A, Ao = _bf16(rng, m, n)
    Q = torch.from_numpy(np.linalg.qr(rng.standard_normal((m, w)))[0].astype(np.float32)).cuda()
    R.arm_wait_expiry(1, LIMIT_NS, 1)
    with pytest.raises(R.RpcaError) as e:
        R.t_pass(A, Q, kernel=2)
    assert e.value.status == -6                       # RPCA_ETIMEOUT
    T = R.t_pass(A, Q, kernel=2)                      # the device is still usable
    torch.cuda.synchronize()
    To = ro.t_pass_product(Ao, gen.round_bf16_np(Q.cpu().numpy()).astype(np.float64))
    assert _rel(T.cpu().numpy(), To) < 2e-5


def test_fused_pass_noalloc_wait_expiry_then_normal_call(R):
    rng = np.random.default_rng(2)
    m, n, p = 9_001, 4096, 60
    A, Ao = _bf16(rng, m, n)
    X = torch.from_numpy(rng.standard_normal((n, p)).astype(np.float32)).cuda()
    R.arm_wait_expiry(0, LIMIT_NS, 3)
    with pytest.raises(R.RpcaError) as e:
        R.fused_pass_noalloc(A, X)
    assert e.value.status == -6
    H, F = R.fused_pass_noalloc(A, X)
    torch.cuda.synchronize()
    Ho, _ = ro.fused_pass_products(Ao, gen.round_bf16_np(X.cpu().numpy()).astype(np.float64))
    assert _rel(H.cpu().numpy(), Ho) < 2e-5
    Fo = ro.t_pass_product(Ao, gen.round_bf16_np(H.cpu().numpy()).astype(np.float64))
    assert _rel(F.cpu().numpy(), Fo) < 2e-5


def test_whole_pca_wait_expiry_then_normal_run(R):
    """The T pass of a whole BF16 PCA times out: rpca_run returns
    RPCA_ETIMEOUT; the next run on the same device matches the oracle."""
    m, n, k, l, i = 20_000, 512, 8, 20, 1
    A = gen.lowrank_np(m, n, 0.8 ** np.arange(n), seed=4) + 1e-3 * np.random.default_rng(4).standard_normal((m, n))
    Ab = torch.from_numpy(A.astype(np.float32)).cuda().to(torch.bfloat16)
    R.arm_wait_expiry(1, LIMIT_NS, 2)
    with pytest.raises(R.RpcaError) as e:
        R.pca(Ab, k, l, i, seed=3)
    assert e.value.status == -6
    U, S, V = R.pca(Ab, k, l, i, seed=3)
    Uo, So, Vo = ro.rpca(Ab.float().cpu().double().numpy(), k, l, i, seed=3, reorth=True)
    assert np.max(np.abs(S.cpu().numpy() - So) / So) < 1e-3

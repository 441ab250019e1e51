"""Parity at the full workload sizes, in the configuration bench.py times.

fp32_center (200,000 x 2,000, centred) runs against the FP64 oracle.  The
precision workload (1,000,000 x 4,096, k=50 l=60 i=2) runs against the FP64
oracle too (two oracle runs of a few minutes each on the host cores, one on
the FP32 values and one on the BF16 values, streamed by row blocks as in
Section 4.2), and in addition through relations that hold exactly at any
size:
  * A^T U = V Sigma (Section 3: T = A^T Q = V~ Sigma~ W^T and U = Q W, so
    A^T Q W = V~ Sigma~ column by column), on sampled columns of A;
  * U^T U = I and V^T V = I;
  * the spectral error of the BF16 path within 1.05x of the FP32 path's."""
import concurrent.futures as cf

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rpca_oracle as ro, estimator as est  # noqa: E402
from synth import generators as gen  # noqa: E402

pytestmark = pytest.mark.gpu


def R():
    from paper_1007_5510_gb300 import rpca
    rpca.load_library()
    return rpca


def test_fp32_center_full_size_matches_oracle():
    cfg = gen.CONFIGS["fp32_center"]
    m, n, k, l, i = cfg["m"], cfg["n"], cfg["k"], cfg["l"], cfg["i"]
    A = gen.workload_np("fp32_center").astype(np.float32)
    U, S, V = R().pca(torch.from_numpy(A).cuda(), k, l, i, seed=1007, center=True)
    A64 = A.astype(np.float64)
    Uo, So, Vo = ro.rpca(A64, k, l, i, seed=1007, center=True, reorth=True)
    s = S.cpu().numpy()
    rel = np.max(np.abs(s - So) / So)
    au = est.max_principal_angle(U.cpu().double().numpy(), Uo)
    av = est.max_principal_angle(V.cpu().double().numpy(), Vo)
    print("PARITY fp32_center full size sigma_rel %.3e angle_U %.3e angle_V %.3e" % (rel, au, av))
    assert rel <= 1e-4 and au <= 1e-3 and av <= 1e-3, (rel, au, av)


def _spectral_error(A, U, S, V, iters=30, nvec=4):
    g = torch.Generator(device=A.device)
    g.manual_seed(5)
    x = torch.randn(A.shape[1], nvec, generator=g, device=A.device)
    Sf = S.float()
    est_ = 0.0
    for _ in range(iters):
        y = A @ x - U @ (Sf[:, None] * (V.T @ x))
        z = A.T @ y - V @ (Sf[:, None] * (U.T @ y))
        nz = torch.linalg.norm(z, dim=0)
        est_ = float(torch.sqrt(nz.max() / torch.linalg.norm(x, dim=0)[nz.argmax()]))
        x = torch.linalg.qr(z.cpu())[0].to(z.device)
    return est_


@pytest.fixture(scope="module")
def precision_runs():
    cfg = gen.CONFIGS["precision"]
    m, n, k, l, i = cfg["m"], cfg["n"], cfg["k"], cfg["l"], cfg["i"]
    dev = torch.device("cuda")
    A32 = gen.workload_torch("precision", dev, m=m, n=n, seed=1007, rank_cap=1024)
    A16 = A32.to(torch.bfloat16)
    out = {}
    for name, A in (("bf16", A16), ("f32", A32)):
        out[name] = R().pca(A, k, l, i, seed=1007)
    torch.cuda.synchronize()
    yield cfg, A32, A16, out
    del A32, A16


@pytest.mark.parametrize("name", ["bf16", "f32"])
def test_precision_full_size_identities(precision_runs, name):
    cfg, A32, A16, out = precision_runs
    A = A16 if name == "bf16" else A32
    U, S, V = out[name]
    Uh = U.cpu().double().numpy()
    Vh = V.cpu().double().numpy()
    s = S.cpu().numpy()
    k = cfg["k"]
    assert np.all(np.diff(s) <= 0) and s[-1] > 0
    assert np.abs(Uh.T @ Uh - np.eye(k)).max() < 1e-5
    assert np.abs(Vh.T @ Vh - np.eye(k)).max() < 1e-5
    cols = np.random.default_rng(3).choice(A.shape[1], 24, replace=False)
    Ac = A[:, torch.as_tensor(cols, device=A.device)].float().cpu().double().numpy()   # m x 24
    lhs = Ac.T @ Uh                     # rows c of A^T U
    rhs = Vh[cols] * s[None, :]         # rows c of V Sigma
    rel = np.abs(lhs - rhs).max() / np.abs(rhs).max()
    # BF16: T is formed from the BF16-rounded Q (relative 2^-9 per entry,
    # averaging over 1e6 rows); FP32: FP32 storage of U and V
    assert rel < (2e-3 if name == "bf16" else 1e-4), rel


def test_precision_full_size_bf16_error_within_5pct_of_fp32(precision_runs):
    cfg, A32, A16, out = precision_runs
    e16 = _spectral_error(A32, *out["bf16"])
    e32 = _spectral_error(A32, *out["f32"])
    assert e16 <= 1.05 * e32, (e16, e32)


# BF16 storage against the oracle on the same BF16 values (the tensor cores
# see X, H and Q rounded to BF16)
BF16_ANGLE = 1e-2


def test_precision_full_size_matches_oracle(precision_runs):
    """FP32 path against the FP64 oracle on the FP32 values (sigma 1e-4,
    angles 1e-3 rad); BF16 path against the FP64 oracle on the BF16 values.
    Also prints each path's error against the FP64 result on the FP32
    matrix (the unquantised input)."""
    cfg, A32, A16, out = precision_runs
    m, n, k, l, i = cfg["m"], cfg["n"], cfg["k"], cfg["l"], cfg["i"]
    A32h = A32.cpu()
    A16h = A16.cpu()

    def rows32(r0, r1):
        return A32h[r0:r1].numpy()

    def rows16(r0, r1):
        return A16h[r0:r1].float().numpy()

    # the two oracle runs overlap on the host cores (NumPy releases the GIL)
    with cf.ThreadPoolExecutor(2) as ex:
        f32 = ex.submit(ro.rpca, rows32, k, l, i, seed=1007, reorth=True, m=m, n=n, return_parts=True)
        f16 = ex.submit(ro.rpca, rows16, k, l, i, seed=1007, reorth=True, m=m, n=n)
        o32, o16 = f32.result(), f16.result()
    res = {}
    for name, ref, lab in (("f32", o32, "vs oracle(FP32 values)"), ("bf16", o16, "vs oracle(BF16 values)"),
                           ("bf16", o32, "vs oracle(FP32 values)")):
        U, S, V = out[name]
        s = S.cpu().numpy()
        rel = float(np.max(np.abs(s - ref[1]) / ref[1]))
        au = est.max_principal_angle(U.cpu().double().numpy(), ref[0])
        av = est.max_principal_angle(V.cpu().double().numpy(), ref[2])
        print("PARITY precision full size %s %s sigma_rel %.3e angle_U %.3e angle_V %.3e"
              % (name, lab, rel, au, av))
        res[(name, lab)] = (rel, au, av)
    rel, au, av = res[("f32", "vs oracle(FP32 values)")]
    assert rel <= 1e-4 and au <= 1e-3 and av <= 1e-3, (rel, au, av)
    # BF16: the singular values are asserted; the subspace angles are only
    # reported here, because this workload's sigma_50 sits at the edge of the
    # noise bulk (the Ritz gap below), where rounding X, H and Q to BF16 on
    # the tensor cores rotates the 50th direction into its neighbours.  The
    # BF16 path's criterion is its spectral error, within 1.05x of FP32's
    # (test_precision_full_size_bf16_error_within_5pct_of_fp32).
    St = o32[3]["S_all"] if len(o32) > 3 else None
    if St is not None:
        print("PARITY precision full size Ritz gap sigma_%d - sigma_%d = %.3e" % (k, k + 1, St[k - 1] - St[k]))
    rel, au, av = res[("bf16", "vs oracle(BF16 values)")]
    assert rel <= 1e-3, (rel, au, av)

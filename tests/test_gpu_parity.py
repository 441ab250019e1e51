"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances.  FP32 workloads: relative singular-value error <= 1e-4 and
largest principal angle <= 1e-3 rad.  FP64 workload: 1e-10 and 1e-8 rad
(rounding of the normalised FP64 iteration: span errors of the Cholesky QR
basis ~ u kappa(H^(0)) ~ 1e-11, amplified by sigma_1 / (sigma_10 - sigma_11)
~ 2e4 for the singular vectors).  BF16 storage, against the oracle on the
same BF16 values: sigma <= 1e-3 and angles <= BF16_ANGLE, where the tensor
cores see Q rounded to BF16 (2^-9 relative per entry).  Single passes:
elementwise relative to the largest entry, 2e-5 (FP32 accumulation over <= a
few thousand terms).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import rpca_oracle as ro, estimator as est  # noqa: E402
from synth import generators as gen  # noqa: E402

# BF16 whole-method angle bound (see the module docstring)
BF16_ANGLE = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1007_5510_gb300 import rpca
    rpca.load_library()


def R():
    from paper_1007_5510_gb300 import rpca
    return rpca


def _tt(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _stored(A, dtype):
    """Values the library sees for storage dtype (FP64 copy for the oracle)."""
    if dtype == "f64":
        return _tt(A, torch.float64), A
    if dtype == "f32":
        return _tt(A, torch.float32), A.astype(np.float32).astype(np.float64)
    if dtype == "bf16":
        t = _tt(A, torch.float32).to(torch.bfloat16)
        return t, t.float().cpu().double().numpy()
    raise ValueError(dtype)


# --------------------------------------------------------------- single pass
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,p", [(1000, 300, 12), (2345, 517, 22), (777, 1000, 60)])
def test_fused_pass_matches_oracle(dtype, m, n, p):
    rng = np.random.default_rng(m + n + p)
    A = rng.standard_normal((m, n))
    X = rng.standard_normal((n, p))
    At, Ao = _stored(A, dtype)
    cdt = torch.float64 if dtype == "f64" else torch.float32
    H, F = R().fused_pass(At, _tt(X, cdt), kernel=1)
    torch.cuda.synchronize()
    Xo = X if dtype == "f64" else X.astype(np.float32).astype(np.float64)
    Ho, Fo = ro.fused_pass_products(Ao, Xo)
    tol = 1e-12 if dtype == "f64" else 2e-5
    assert _rel(H.cpu().numpy(), Ho) < tol
    assert _rel(F.cpu().numpy(), Fo) < tol * 5


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_fused_pass_shift_and_scale(dtype):
    rng = np.random.default_rng(5)
    m, n, p = 1500, 333, 20
    A = rng.standard_normal((m, n)) + 3.0
    X = rng.standard_normal((n, p))
    s = (A[:128].mean(axis=0)).astype(np.float32)
    c = rng.uniform(0.5, 2.0, n).astype(np.float32)
    At, Ao = _stored(A, dtype)
    H, F = R().fused_pass(At, _tt(X), shift=_tt(s), col_scale=_tt(c), kernel=1)
    torch.cuda.synchronize()
    Ho, Fo = ro.fused_pass_products(Ao, X.astype(np.float32).astype(np.float64), shift=s.astype(np.float64),
                                    col_scale=c.astype(np.float64))
    assert _rel(H.cpu().numpy(), Ho) < 5e-5
    assert _rel(F.cpu().numpy(), Fo) < 2e-4


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_t_pass_matches_oracle(dtype):
    rng = np.random.default_rng(11)
    m, n, w = 3001, 257, 66
    A = rng.standard_normal((m, n))
    Q = np.linalg.qr(rng.standard_normal((m, w)))[0]
    At, Ao = _stored(A, dtype)
    cdt = torch.float64 if dtype == "f64" else torch.float32
    T = R().t_pass(At, _tt(Q, cdt), kernel=1)
    torch.cuda.synchronize()
    Qo = Q if dtype == "f64" else Q.astype(np.float32).astype(np.float64)
    To = ro.t_pass_product(Ao, Qo)
    assert _rel(T.cpu().numpy(), To) < (1e-12 if dtype == "f64" else 5e-5)


# ------------------------------------------------------------------ Step 2
@pytest.mark.parametrize("f64,m", [(True, 5000), (False, 5000), (False, 50_000)])
def test_block_qr(f64, m):
    """Step 2 on CUDA cores (m = 5000) and on tensor cores (m = 50,000, TF32 x3)."""
    rng = np.random.default_rng(3)
    l, nblk = 20, 3
    H = rng.standard_normal((m, nblk * l)) @ np.diag(0.9 ** np.arange(nblk * l))
    Ht = _tt(H, torch.float64 if f64 else torch.float32)
    R().qr_inplace(Ht, nblk, l)
    torch.cuda.synchronize()
    Q = Ht.cpu().double().numpy()
    orth = np.abs(Q.T @ Q - np.eye(nblk * l)).max()
    assert orth < (1e-13 if f64 else 1e-5)
    Qo, _, _ = ro.pivoted_qr(H)
    assert est.max_principal_angle(Q, Qo) < (1e-10 if f64 else 1e-4)


@pytest.mark.parametrize("f64,l,nblk", [(False, 20, 2), (True, 20, 2), (False, 60, 1), (True, 7, 3)])
def test_block_qr_shifted_cholesky(f64, l, nblk):
    """A block with two nearly equal columns makes the first Cholesky pivot
    fail; the shifted Cholesky QR (Section 3's Step 2 with a diagonal shift,
    then up to two more passes) must still return an orthonormal Q whose span
    contains H's columns."""
    rng = np.random.default_rng(l + nblk)
    m, w = 6000, nblk * l
    H = rng.standard_normal((m, w))
    j = w - 3
    H[:, j] = H[:, j - 1] + (1e-13 if f64 else 1e-7) * rng.standard_normal(m)
    Ht = _tt(H, torch.float64 if f64 else torch.float32)
    R().qr_inplace(Ht, nblk, l)
    torch.cuda.synchronize()
    Q = Ht.cpu().double().numpy()
    Hc = H if f64 else H.astype(np.float32).astype(np.float64)
    assert np.abs(Q.T @ Q - np.eye(w)).max() < (1e-12 if f64 else 1e-5)
    res = np.linalg.norm(Hc - Q @ (Q.T @ Hc)) / np.linalg.norm(Hc)
    assert res < (1e-12 if f64 else 1e-5)


@pytest.mark.parametrize("m,l,nblk,decay", [(100_000, 60, 3, 0.97), (30_001, 48, 2, 0.9), (20_000, 64, 3, 0.95)])
def test_block_qr_sliced_tensor_cores(m, l, nblk, decay):
    """Step 2 with H held in three BF16 slices on tensor cores (blocks of
    40..64 columns padded to 64): orthonormal to FP32 level and spanning the
    pivoted-QR basis of the oracle."""
    rng = np.random.default_rng(m + l)
    w = nblk * l
    H = rng.standard_normal((m, w)) @ np.diag(decay ** np.arange(w))
    H32 = H.astype(np.float32)
    Ht = _tt(H32)
    R().qr_inplace(Ht, nblk, l)
    torch.cuda.synchronize()
    Q = Ht.cpu().double().numpy()
    assert np.abs(Q.T @ Q - np.eye(w)).max() < 1e-5
    Qo, _, _ = ro.pivoted_qr(H32.astype(np.float64))
    assert est.max_principal_angle(Q, Qo) < 1e-4


# ------------------------------------------------------------------ Step 4
@pytest.mark.parametrize("f64,w", [(True, 24), (False, 66), (False, 180)])
def test_small_svd(f64, w):
    rng = np.random.default_rng(w)
    n = 700
    sig = np.exp(-np.arange(w) / 15.0)
    T = gen.lowrank_np(n, w, sig, seed=w)
    Tt = _tt(T, torch.float64 if f64 else torch.float32)
    S, Vt, W = R().small_svd(Tt)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    Se = np.linalg.svd(Tt.cpu().double().numpy(), compute_uv=False)
    # FP32: the QR of T is normwise stable, so values far below sigma_1 are
    # accurate to ~1e-7 sigma_1 absolutely; the leading ones relatively.
    big = Se >= 1e-2 * Se[0]
    assert np.max(np.abs(S - Se)[big] / Se[big]) < (1e-12 if f64 else 1e-5)
    assert np.max(np.abs(S - Se)) < (1e-14 if f64 else 2e-6) * Se[0]
    Vt = Vt.cpu().double().numpy()
    W = W.cpu().numpy()
    recon = (Vt * S[None, :]) @ W.T
    assert _rel(recon, Tt.cpu().double().numpy()) < (1e-12 if f64 else 2e-5)


# ------------------------------------------------------------- whole method
def _compare(U, S, V, Uo, So, Vo, s_tol, a_tol, label=""):
    """Relative singular-value error and the largest principal angles of U
    and V against the oracle's (printed, then asserted)."""
    S = S.cpu().numpy()
    rel = np.max(np.abs(S - So) / So)
    au = est.max_principal_angle(U.cpu().double().numpy(), Uo)
    av = est.max_principal_angle(V.cpu().double().numpy(), Vo)
    print("PARITY %s sigma_rel %.3e angle_U %.3e angle_V %.3e (bounds %.0e, %.0e)" % (label, rel, au, av, s_tol, a_tol))
    assert rel <= s_tol and au <= a_tol and av <= a_tol, (rel, au, av)
    return rel, au, av


def test_pca_fp64_small_workload():
    """fp64_small at full size (2000 x 1000, k=10 l=12 i=1)."""
    cfg = gen.CONFIGS["fp64_small"]
    A = gen.workload_np("fp64_small")
    U, S, V = R().pca(_tt(A, torch.float64), cfg["k"], cfg["l"], cfg["i"], seed=1007)
    Uo, So, Vo = ro.rpca(A, cfg["k"], cfg["l"], cfg["i"], seed=1007, reorth=True)
    _compare(U, S, V, Uo, So, Vo, 1e-10, 1e-8, "fp64_small")


@pytest.mark.parametrize("m,n,k,l,i", [(5000, 300, 10, 12, 2), (4099, 1031, 20, 22, 1), (1000, 64, 16, 20, 1)])
def test_pca_fp32_matches_oracle(m, n, k, l, i):
    A = gen.lowrank_np(m, n, np.arange(1, n + 1) ** -1.0, seed=m) + 1e-4 * np.random.default_rng(1).standard_normal((m, n))
    A32 = A.astype(np.float32)
    U, S, V = R().pca(_tt(A32), k, l, i, seed=99)
    Uo, So, Vo = ro.rpca(A32.astype(np.float64), k, l, i, seed=99, reorth=True)
    _compare(U, S, V, Uo, So, Vo, 1e-4, 1e-3, "fp32 %dx%d" % (m, n))


@pytest.mark.parametrize("dtype,m,n,k,l,i,r", [("f32", 3000, 400, 5, 10, 2, 8), ("f64", 2000, 300, 4, 9, 2, 7),
                                               ("bf16", 20_000, 512, 8, 48, 1, 16)])
def test_pca_exactly_low_rank(dtype, m, n, k, l, i, r):
    """rank(A) = r < (i+1) l: the later Krylov blocks are rounding noise, so H
    is numerically rank deficient and their Cholesky passes need the shift.
    The top k singular values still match the oracle (pivoted QR) on the same
    matrix, and U, V stay orthonormal."""
    sig = np.linspace(1.0, 0.3, r)
    A = gen.lowrank_np(m, n, sig, seed=r)
    if dtype == "f64":
        At = _tt(A, torch.float64)
    else:
        At = torch.from_numpy(A.astype(np.float32)).cuda()
        if dtype == "bf16":
            At = At.to(torch.bfloat16)
    U, S, V = R().pca(At, k, l, i, seed=5)
    Aref = At.double().cpu().numpy()
    Uo, So, Vo = ro.rpca(Aref, k, l, i, seed=5, reorth=True)
    tol = {"f64": 1e-10, "f32": 1e-4, "bf16": 1e-3}[dtype]
    assert np.max(np.abs(S.cpu().numpy() - So) / So) < tol
    Ud, Vd = U.cpu().double().numpy(), V.cpu().double().numpy()
    otol = 1e-12 if dtype == "f64" else 1e-4
    assert np.abs(Ud.T @ Ud - np.eye(k)).max() < otol
    assert np.abs(Vd.T @ Vd - np.eye(k)).max() < otol


def test_pca_centered_fp32_reduced():
    """fp32_center construction at reduced size (m=20,000, n=500), centred,
    against the normalised FP64 oracle at the FP32 bounds."""
    A = gen.workload_np("fp32_center", m=20_000, n=500).astype(np.float32)
    U, S, V = R().pca(_tt(A), 20, 22, 2, seed=7, center=True)
    Uo, So, Vo = ro.rpca(A.astype(np.float64), 20, 22, 2, seed=7, center=True, reorth=True)
    _compare(U, S, V, Uo, So, Vo, 1e-4, 1e-3, "fp32_center 20000x500")


def test_pca_centered_fp64_reduced():
    """The centring corrections (shift in registers, rank-one terms) in FP64
    reproduce the oracle's explicit centring at the FP64 bounds."""
    A = gen.workload_np("fp32_center", m=20_000, n=500)
    U, S, V = R().pca(_tt(A, torch.float64), 20, 22, 2, seed=7, center=True)
    Uo, So, Vo = ro.rpca(A, 20, 22, 2, seed=7, center=True, reorth=True)
    _compare(U, S, V, Uo, So, Vo, 1e-10, 1e-8, "fp64_center 20000x500")


def test_pca_transposed():
    """n > m: the library runs on A^T (Section 3) and swaps the factors."""
    rng = np.random.default_rng(2)
    A = gen.lowrank_np(300, 900, 0.9 ** np.arange(300), seed=3) + 1e-5 * rng.standard_normal((300, 900))
    A32 = A.astype(np.float32)
    U, S, V = R().pca(_tt(A32), 6, 8, 1, seed=5)
    assert U.shape == (300, 6) and V.shape == (900, 6)
    Uo, So, Vo = ro.rpca(A32.astype(np.float64), 6, 8, 1, seed=5, reorth=True)
    _compare(U, S, V, Uo, So, Vo, 1e-4, 1e-3, "transposed")


def test_explicit_G_equals_seed():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((800, 120)).astype(np.float32)
    from oracle import philox
    G = philox.gaussian_matrix(123, 120, 9)
    U1, S1, V1 = R().pca(_tt(A), 7, 9, 1, seed=123)
    U2, S2, V2 = R().pca(_tt(A), 7, 9, 1, G=G)
    # the two Philox/Box-Muller implementations agree to a few ulp
    assert torch.allclose(S1, S2, rtol=1e-5)


def test_host_streamed_tiles_match_device():
    """Out-of-core form: A in pinned host memory, tiles of 700 rows (ragged)."""
    rng = np.random.default_rng(8)
    m, n = 5000, 256
    A = (gen.lowrank_np(m, n, 0.8 ** np.arange(n), seed=1) + 1e-4 * rng.standard_normal((m, n))).astype(np.float32)
    Ah = torch.from_numpy(A).pin_memory()
    ctx = R().PCA(m, n, 10, 12, 2, R().F32, seed=3, host_a=True, tile_rows=700)
    try:
        U, S, V = ctx.run(Ah)
    finally:
        ctx.close()
    U2, S2, V2 = R().pca(_tt(A), 10, 12, 2, seed=3)
    assert torch.allclose(S, S2, rtol=1e-5)
    Uo, So, Vo = ro.rpca(A.astype(np.float64), 10, 12, 2, seed=3, reorth=True)
    _compare(U, S, V, Uo, So, Vo, 1e-4, 1e-3, "host tiles")


@pytest.mark.parametrize("dtype,m,n", [("f32", 5000, 256), ("bf16", 20_003, 1024)])
def test_host_resident_matches_device(dtype, m, n):
    """A in pinned host memory copied once per run (ragged tiles, the first
    pass on each tile as it lands), the later passes on the device copy; a
    second run with another matrix must see the new values."""
    rng = np.random.default_rng(12)
    A = (gen.lowrank_np(m, n, 0.8 ** np.arange(n), seed=2) + 1e-4 * rng.standard_normal((m, n))).astype(np.float32)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    code = R().BF16 if dtype == "bf16" else R().F32
    Ad = torch.from_numpy(A).cuda().to(tdt)
    Ah = Ad.cpu().pin_memory()
    Bh = (Ad * 4).cpu().pin_memory()                   # exact in BF16 too
    k, l, i = 10, 12, 2
    ctx = R().PCA(m, n, k, l, i, code, seed=3, host_a=True, host_resident=True, tile_rows=1700)
    try:
        _, S, _ = ctx.run(Ah)
        S = S.clone()
        _, S3, _ = ctx.run(Bh)
        S3 = S3.clone()
    finally:
        ctx.close()
    _, S2, _ = R().pca(Ad, k, l, i, seed=3)
    assert torch.allclose(S, S2, rtol=1e-5 if dtype == "f32" else 1e-4)
    assert torch.allclose(S3, 4 * S2, rtol=1e-5 if dtype == "f32" else 1e-4)


def test_rerun_reuses_context():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((1200, 200)).astype(np.float32)
    B = (A * 2.0).astype(np.float32)
    ctx = R().PCA(1200, 200, 5, 7, 1, R().F32, seed=1)
    try:
        _, S1, _ = ctx.run(_tt(A))
        _, S2, _ = ctx.run(_tt(B))
    finally:
        ctx.close()
    assert torch.allclose(S2, 2 * S1, rtol=1e-5)


# ------------------------------------------------- tensor-core T pass (BF16)
@pytest.mark.parametrize("m,n,w", [(3001, 512, 66), (5000, 520, 180), (20000, 4096, 180), (777, 256, 24)])
def test_t_pass_tensor_cores_bf16(m, n, w):
    """tcgen05 T pass: BF16 A and BF16-rounded Q, FP32 accumulation."""
    rng = np.random.default_rng(m + w)
    A = rng.standard_normal((m, n))
    Q = np.linalg.qr(rng.standard_normal((m, w)))[0]
    At, Ao = _stored(A, "bf16")
    T = R().t_pass(At, _tt(Q), kernel=2)
    torch.cuda.synchronize()
    Qo = gen.round_bf16_np(Q).astype(np.float64)
    To = ro.t_pass_product(Ao, Qo)
    assert _rel(T.cpu().numpy(), To) < 2e-5


# ------------------------------------------- tensor-core fused pass (BF16)
@pytest.mark.parametrize("m,n,l", [(1000, 512, 12), (5000, 4096, 60), (777, 1000, 22),
                                   (3001, 2000, 30), (300, 64, 20),
                                   (8000, 4104, 40),       # 16-CTA clusters, 7 empty column slabs
                                   (40_001, 2600, 63)])    # 6 slabs rounded up to 8, ~20 panels per cluster
@pytest.mark.parametrize("with_f", [True, False])
def test_fused_pass_tensor_cores_bf16(m, n, l, with_f):
    """Cluster-split tcgen05 pass: H = A bf16(X) and F = A^T bf16(H) (the
    kernel feeds BF16 operands to the tensor cores, FP32 accumulation)."""
    rng = np.random.default_rng(m + n + l)
    A = rng.standard_normal((m, n))
    X = rng.standard_normal((n, l))
    At, Ao = _stored(A, "bf16")
    H, F = R().fused_pass(At, _tt(X), with_f=with_f, kernel=2)
    torch.cuda.synchronize()
    Xo = gen.round_bf16_np(X).astype(np.float64)
    Ho, _ = ro.fused_pass_products(Ao, Xo)
    assert _rel(H.cpu().numpy(), Ho) < 2e-5
    if with_f:
        Fg = F.cpu().numpy()
        Hb = gen.round_bf16_np(H.cpu().numpy()).astype(np.float64)
        Fo = ro.t_pass_product(Ao, Hb)
        assert _rel(Fg, Fo) < 2e-5
        # independent of the GPU's own H: against A^T H_o with the oracle's
        # unrounded H_o.  The kernel multiplies by bf16(H), |bf16(H) - H| <=
        # 2^-9 |H| per entry, and |H - H_o| <= 2e-5 max|H_o| (asserted above),
        # so |F - A^T H_o| <= |A|^T (2^-9 |H_o| + 2e-5 max|H_o|) plus the FP32
        # accumulation (2e-5 of max|F|).
        Fo2 = ro.t_pass_product(Ao, Ho)
        absA = np.abs(Ao)
        bound = absA.T @ (2.0 ** -9 * np.abs(Ho) + 2e-5 * np.abs(Ho).max()) + 2e-5 * np.abs(Fo2).max()
        assert np.all(np.abs(Fg - Fo2) <= bound)


# ---------------------------- tensor-core passes over FP32 A (converters)
@pytest.mark.parametrize("m,n,l", [(1000, 512, 12), (5000, 4096, 60), (777, 1000, 22), (3001, 2000, 30),
                                   (300, 64, 20), (40_001, 2600, 63)])
@pytest.mark.parametrize("with_f", [True, False])
def test_fused_pass_tensor_cores_f32(m, n, l, with_f):
    """FP32 A on the tensor cores: converter warps split A and X into BF16
    hi/lo slices (hi*hi + lo*hi + hi*lo, FP32 accumulation), then F from
    the hi/lo slices of H.  Against the oracle on the FP32 values."""
    rng = np.random.default_rng(m + n + l + 1)
    A = rng.standard_normal((m, n))
    X = rng.standard_normal((n, l))
    At, Ao = _stored(A, "f32")
    H, F = R().fused_pass(At, _tt(X), with_f=with_f, kernel=2)
    torch.cuda.synchronize()
    Ho, Fo = ro.fused_pass_products(Ao, X.astype(np.float32).astype(np.float64))
    eh = _rel(H.cpu().numpy(), Ho)
    print("PARITY fused f32 tc %dx%d l=%d H %.2e" % (m, n, l, eh), end="")
    assert eh < 3e-5
    if with_f:
        ef = _rel(F.cpu().numpy(), Fo)
        print(" F %.2e" % ef, end="")
        assert ef < 5e-5
    print()


@pytest.mark.parametrize("m,n,l", [(20_000, 500, 22), (4099, 1028, 20)])
def test_fused_pass_tensor_cores_f32_shift_and_scale(m, n, l):
    """The centring shift and a per-column scale applied by the converter:
    A_c = A diag(c) - 1 s^T in FP32 before the split."""
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, n)) * 0.01 + 3.0
    X = rng.standard_normal((n, l))
    c = rng.uniform(0.5, 2.0, n).astype(np.float32)
    A32 = A.astype(np.float32)
    s = (A32[:128].astype(np.float64) * c).mean(axis=0).astype(np.float32)
    H, F = R().fused_pass(_tt(A32), _tt(X), shift=_tt(s), col_scale=_tt(c), kernel=2)
    torch.cuda.synchronize()
    Ho, Fo = ro.fused_pass_products(A32.astype(np.float64), X.astype(np.float32).astype(np.float64),
                                    shift=s.astype(np.float64), col_scale=c.astype(np.float64))
    eh, ef = _rel(H.cpu().numpy(), Ho), _rel(F.cpu().numpy(), Fo)
    print("PARITY fused f32 tc shift+scale %dx%d H %.2e F %.2e" % (m, n, eh, ef))
    assert eh < 5e-5 and ef < 1e-4


@pytest.mark.parametrize("m,n,w", [(3001, 512, 66), (5000, 520, 180), (20000, 4096, 180), (777, 256, 24)])
def test_t_pass_tensor_cores_f32(m, n, w):
    """T = A^T Q for FP32 A on the tensor cores (A and Q as BF16 hi/lo)."""
    rng = np.random.default_rng(m + w + 1)
    A = rng.standard_normal((m, n))
    Q = np.linalg.qr(rng.standard_normal((m, w)))[0]
    At, Ao = _stored(A, "f32")
    T = R().t_pass(At, _tt(Q), kernel=2)
    torch.cuda.synchronize()
    To = ro.t_pass_product(Ao, Q.astype(np.float32).astype(np.float64))
    e = _rel(T.cpu().numpy(), To)
    print("PARITY t pass f32 tc %dx%d w=%d %.2e" % (m, n, w, e))
    assert e < 5e-5


@pytest.mark.parametrize("m,n,l", [(1000, 512, 12), (5000, 4096, 60), (3001, 2000, 30), (40_001, 2608, 63)])
def test_fused_pass_tensor_cores_fp8(m, n, l):
    """FP8-e4m3 bytes widened exactly to BF16 by the converters, the
    per-column scales folded into X (H = A8 diag(s) X) and into F's rows,
    X and H as BF16 hi/lo slices.  Against the oracle on the dequantised
    values."""
    rng = np.random.default_rng(m + l + 7)
    A = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
    q, sc = gen.quantize_fp8_torch(A)
    X = rng.standard_normal((n, l))
    H, F = R().fused_pass(q, _tt(X), col_scale=sc, kernel=2)
    torch.cuda.synchronize()
    Adq = (q.view(torch.float8_e4m3fn).float() * sc[None, :]).double().cpu().numpy()
    Ho, Fo = ro.fused_pass_products(Adq, X.astype(np.float32).astype(np.float64))
    eh, ef = _rel(H.cpu().numpy(), Ho), _rel(F.cpu().numpy(), Fo)
    print("PARITY fused fp8 tc %dx%d l=%d H %.2e F %.2e" % (m, n, l, eh, ef))
    assert eh < 3e-5 and ef < 5e-5


@pytest.mark.parametrize("m,n,w", [(3001, 512, 66), (20000, 4096, 180)])
def test_t_pass_tensor_cores_fp8(m, n, w):
    rng = np.random.default_rng(m + w + 3)
    A = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
    q, sc = gen.quantize_fp8_torch(A)
    Q = np.linalg.qr(rng.standard_normal((m, w)))[0]
    T = R().t_pass(q, _tt(Q), col_scale=sc, kernel=2)
    torch.cuda.synchronize()
    Adq = (q.view(torch.float8_e4m3fn).float() * sc[None, :]).double().cpu().numpy()
    To = ro.t_pass_product(Adq, Q.astype(np.float32).astype(np.float64))
    e = _rel(T.cpu().numpy(), To)
    print("PARITY t pass fp8 tc %dx%d w=%d %.2e" % (m, n, w, e))
    assert e < 5e-5


def test_fused_pass_tensor_cores_bf16_shifted():
    """BF16 storage with a centring shift: the converters form a - s in FP32
    and split it, so the shift costs no precision."""
    rng = np.random.default_rng(31)
    m, n, l = 20_000, 1024, 40
    A = rng.standard_normal((m, n)) * 0.01 + 5.0
    At, Ao = _stored(A, "bf16")
    s = Ao[:128].mean(axis=0).astype(np.float32)
    X = rng.standard_normal((n, l))
    H, F = R().fused_pass(At, _tt(X), shift=_tt(s), kernel=2)
    torch.cuda.synchronize()
    Ho, Fo = ro.fused_pass_products(Ao, X.astype(np.float32).astype(np.float64), shift=s.astype(np.float64))
    eh, ef = _rel(H.cpu().numpy(), Ho), _rel(F.cpu().numpy(), Fo)
    print("PARITY fused bf16 shifted tc H %.2e F %.2e" % (eh, ef))
    assert eh < 5e-5 and ef < 1e-4


@pytest.mark.parametrize("dtype", ["f32", "fp8"])
def test_pca_t_from_f_blocks_matches_t_pass(dtype):
    """Step 3 without its pass over A: T = [F^(0) .. F^(i)] R^-1 from the F
    blocks of the fused passes (Q = H R^-1 in Step 2).  Same results as the
    run with its own T pass, and the oracle's at the FP32 bounds; the
    context reports i+1 passes over A instead of i+2."""
    m, n, k, l, i = 60_000, 1024, 20, 48, 2
    A = gen.lowrank_np(m, n, np.exp(-np.arange(1, n + 1) / 25.0), seed=13) + \
        1e-3 * np.random.default_rng(13).standard_normal((m, n))
    At = torch.from_numpy(A.astype(np.float32)).cuda()
    sc = None
    code = R().F32
    if dtype == "fp8":
        At, sc = gen.quantize_fp8_torch(At)
        code = R().FP8E4M3
    outs = {}
    for keep in (False, True):
        ctx = R().PCA(m, n, k, l, i, code, seed=21, keep_t_pass=keep)
        try:
            U, S, V = ctx.run(At, col_scale=sc)
            outs[keep] = (U.clone(), S.clone(), V.clone(), ctx.passes_last_run())
        finally:
            ctx.close()
    assert outs[False][3] == i + 1 and outs[True][3] == i + 2, (outs[False][3], outs[True][3])
    s0, s1 = outs[False][1].cpu().numpy(), outs[True][1].cpu().numpy()
    assert np.max(np.abs(s0 - s1) / s1) < 2e-5
    Ao = At.double().cpu().numpy() if dtype == "f32" else \
        (At.view(torch.float8_e4m3fn).float() * sc[None, :]).double().cpu().numpy()
    Uo, So, Vo = ro.rpca(Ao, k, l, i, seed=21, reorth=True)
    _compare(outs[False][0], outs[False][1], outs[False][2], Uo, So, Vo, 1e-4, 1e-3, "T from F blocks %s" % dtype)


def test_pca_bf16_tensor_cores_vs_fp32():
    """Whole method on BF16 storage (tensor-core passes) against the oracle on
    the same BF16 values, and its spectral error against the FP32 path's."""
    m, n, k, l, i = 20_000, 1024, 16, 20, 2
    A = gen.lowrank_np(m, n, np.exp(-np.arange(1, n + 1) / 10.0), seed=3) + \
        1e-3 * np.random.default_rng(3).standard_normal((m, n))
    A32 = A.astype(np.float32)
    Ab = torch.from_numpy(A32).cuda().to(torch.bfloat16)
    U, S, V = R().pca(Ab, k, l, i, seed=11)
    U2, S2, V2 = R().pca(_tt(A32), k, l, i, seed=11)
    Aob = Ab.float().cpu().double().numpy()
    Uo, So, Vo = ro.rpca(Aob, k, l, i, seed=11, reorth=True)
    _compare(U, S, V, Uo, So, Vo, 1e-3, BF16_ANGLE, "bf16 whole method")
    e16 = est.spectral_error(A32.astype(np.float64), U.cpu().double().numpy(), S.cpu().numpy(), V.cpu().double().numpy())
    e32 = est.spectral_error(A32.astype(np.float64), U2.cpu().double().numpy(), S2.cpu().numpy(), V2.cpu().double().numpy())
    assert e16 <= 1.05 * e32, (e16, e32)


def test_pca_fp32_tensor_core_qr():
    """m above the tensor-core threshold: Step 2, Steps 5-6 on TF32 x3 tensor
    cores; results against the oracle."""
    m, n, k, l, i = 40_000, 256, 10, 12, 2
    A = gen.lowrank_np(m, n, 0.9 ** np.arange(n), seed=21) + 1e-4 * np.random.default_rng(21).standard_normal((m, n))
    A32 = A.astype(np.float32)
    U, S, V = R().pca(_tt(A32), k, l, i, seed=5)
    Uo, So, Vo = ro.rpca(A32.astype(np.float64), k, l, i, seed=5, reorth=True)
    _compare(U, S, V, Uo, So, Vo, 1e-4, 1e-3, "fp32 tensor-core QR")


# --------------------------------------- TF32 x3 tensor-core tall products
@pytest.mark.parametrize("m,p,q,same", [(50_000, 20, 20, True), (50_000, 60, 60, True), (30_000, 180, 180, True),
                                        (40_000, 120, 60, False), (9000, 40, 20, False)])
def test_gram_tensor_cores(m, p, q, same):
    rng = np.random.default_rng(m + p)
    X = rng.standard_normal((m, p)).astype(np.float32)
    Y = X if same else rng.standard_normal((m, q)).astype(np.float32)
    Xt = _tt(X)
    Yt = Xt if same else _tt(Y)
    C = R().gram(Xt, Yt, kernel=2).cpu().numpy()
    Co = X.astype(np.float64).T @ Y.astype(np.float64)
    # BF16 slices give exact products; the tensor cores' FP32 accumulation
    # leaves ~3e-6 relative
    assert _rel(C, Co) < 1e-5


@pytest.mark.parametrize("p", [60, 180])
def test_gram_tensor_cores_long_same_sign_sums(p):
    """Two million rows: every diagonal entry of X^T X is a sum of positive
    products, where an accumulator that rounds relative to its own size
    drifts.  Each diagonal entry must hold to 2e-6 of itself (the orthogonality
    of Q is read from this Gram)."""
    m = 2_000_000
    rng = np.random.default_rng(p)
    X = (rng.standard_normal((m, p)) / np.sqrt(m)).astype(np.float32)
    C = R().gram(_tt(X), kernel=2).cpu().numpy()
    X64 = X.astype(np.float64)
    d = np.einsum("ij,ij->j", X64, X64)
    assert np.max(np.abs(np.diag(C) - d) / d) < 2e-6
    Co = X64.T @ X64
    assert _rel(C, Co) < 2e-6


@pytest.mark.parametrize("m,p,q", [(20_000, 20, 20), (20_000, 60, 60), (30_001, 180, 50), (9000, 120, 60)])
@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_apply_tensor_cores(m, p, q, beta):
    rng = np.random.default_rng(m + p + q)
    X = rng.standard_normal((m, p)).astype(np.float32)
    M = rng.standard_normal((p, q))
    Y0 = rng.standard_normal((m, q)).astype(np.float32)
    Yt = _tt(Y0)
    R().apply(_tt(X), _tt(M, torch.float64), Y=Yt, alpha=-0.5, beta=beta, kernel=2)
    Yo = beta * Y0.astype(np.float64) - 0.5 * X.astype(np.float64) @ M
    assert _rel(Yt.cpu().numpy(), Yo) < 1e-5


@pytest.mark.parametrize("m,p", [(20_000, 66), (20_000, 22), (9000, 130)])
def test_gram_tensor_cores_odd_widths(m, p):
    rng = np.random.default_rng(p)
    X = rng.standard_normal((m, p)).astype(np.float32)
    C = R().gram(_tt(X), kernel=2).cpu().numpy()
    Co = X.astype(np.float64).T @ X.astype(np.float64)
    assert _rel(C, Co) < 1e-5


def test_block_qr_tensor_cores_unaligned_blocks():
    """l = 22: block offsets are not 16-byte aligned (mixed tensor-core and
    CUDA-core products inside one QR)."""
    rng = np.random.default_rng(8)
    m, l, nblk = 20_000, 22, 3
    H = rng.standard_normal((m, nblk * l)) @ np.diag(0.95 ** np.arange(nblk * l))
    Ht = _tt(H)
    R().qr_inplace(Ht, nblk, l)
    Q = Ht.cpu().double().numpy()
    assert np.abs(Q.T @ Q - np.eye(nblk * l)).max() < 1e-5
    Qo, _, _ = ro.pivoted_qr(H)
    assert est.max_principal_angle(Q, Qo) < 1e-4


def test_pca_ordered_after_callers_default_stream_work():
    """A context built on the caller's default stream must run after work the
    caller queued there: A arrives by an asynchronous pinned copy issued just
    before the PCA (a library-private stream would read a half-copied A)."""
    m, n, k, l, i = 200_000, 512, 8, 10, 1
    rng = np.random.default_rng(17)
    A = gen.lowrank_np(2000, n, 0.8 ** np.arange(n), seed=4)
    A = np.tile(A, (m // 2000, 1)).astype(np.float32) + 1e-4 * rng.standard_normal((m, n)).astype(np.float32)
    Ah = torch.from_numpy(A).pin_memory()
    ref = R().pca(_tt(A), k, l, i, seed=3)
    Ad = torch.zeros(m, n, device="cuda")
    torch.cuda.synchronize()
    Ad.copy_(Ah, non_blocking=True)
    U, S, V = R().pca(Ad, k, l, i, seed=3)
    torch.cuda.synchronize()
    assert np.max(np.abs(S.cpu().numpy() - ref[1].cpu().numpy()) / ref[1].cpu().numpy()) < 1e-5


@pytest.mark.parametrize("m,n", [(20_000, 512), (9_001, 333)])
def test_pca_fp8_column_scaled_matches_oracle(m, n):
    """FP8-e4m3 storage with per-column FP32 scales: the PCA of the stored
    matrix diag-scaled (A~ = A8 diag(s)), against the oracle on the same
    dequantised values; FP32 arithmetic, so the FP32 tolerances apply."""
    rng = np.random.default_rng(m + n)
    A = gen.lowrank_np(m, n, np.exp(-np.arange(1, n + 1) / 20.0), seed=8) + 1e-3 * rng.standard_normal((m, n))
    At = torch.from_numpy(A.astype(np.float32)).cuda()
    q, s = gen.quantize_fp8_torch(At)
    k, l, i = 10, 12, 2
    U, S, V = R().pca(q, k, l, i, seed=5, col_scale=s)
    Adq = (q.view(torch.float8_e4m3fn).float() * s[None, :]).double().cpu().numpy()
    Uo, So, Vo = ro.rpca(Adq, k, l, i, seed=5, reorth=True)
    _compare(U, S, V, Uo, So, Vo, 1e-4, 1e-3, "fp8 dequantised %dx%d" % (m, n))

"""Seeded synthetic test matrices (shared by tests, bench and oracle).

No arithmetic of the PCA method lives here: only constructions of inputs
A = U0 diag(sigma) V0^T (+ 1 c^T) (+ noise), where U0 and V0 are the Q
factors (positive-diagonal R) of seeded standard-Gaussian matrices, and the
rounding of A to its storage precision.

Workloads (shapes, spectra, parameters k, l, i):
  fp64_small    m=2,000   n=1,000  sigma_j = 10^(-5(j-1)/11) (j<=11),
                1e-5*11/j (j>11); k=10 l=12 i=1; FP64; no centring
  fp32_center   m=200,000 n=2,000  sigma_j = j^-2, plus 1 c^T with
                c_j ~ N(0,1); FP32; centred; k=20 l=22 i=2
  precision     m=1,000,000 n=4,096 sigma_j = exp(-j/40) plus i.i.d.
                N(0, 1e-6) noise (variance); FP32 / BF16 / FP8-e4m3 with
                per-column scales; k=50 l=60 i=2
  out_of_core   m=6,000,000 n=8,192 rank 64, sigma_j = 0.9^j, plus
                N(0, 1e-4) noise (variance); FP32; k=40 l=48 i=2
  batched       512 problems, m ~ U[1000, 50000], n ~ U[64, 1024],
                sigma_j = j^-1.5; BF16; k=16 l=20 i=1

Spectra whose tail sits far below the storage rounding floor are truncated
at rank ``rank_cap`` (1024 by default): for fp32_center sigma_1025 ~ 9.5e-7
is below the FP32 rounding of an O(1) entry summed over the matrix; for
precision sigma_1025 ~ 7.6e-12 is far below the noise.
"""
import numpy as np

CONFIGS = {
    "fp64_small": dict(m=2000, n=1000, k=10, l=12, i=1, dtype="f64", center=False),
    "fp32_center": dict(m=200_000, n=2000, k=20, l=22, i=2, dtype="f32", center=True),
    "precision": dict(m=1_000_000, n=4096, k=50, l=60, i=2, dtype="f32", center=False),
    "out_of_core": dict(m=6_000_000, n=8192, k=40, l=48, i=2, dtype="f32", center=False),
    "batched": dict(count=512, m_range=(1000, 50000), n_range=(64, 1024), k=16, l=20,
                    i=1, dtype="bf16", center=False),
}

NOISE_STD = {"precision": 1e-3, "out_of_core": 1e-2}


def spectrum(name, r):
    """First r prescribed singular values of workload ``name`` (FP64)."""
    j = np.arange(1, r + 1, dtype=np.float64)
    if name == "fp64_small":
        return np.where(j <= 11, 10.0 ** (-5.0 * (j - 1) / 11.0), 1e-5 * 11.0 / j)
    if name == "fp32_center":
        return j ** -2.0
    if name == "precision":
        return np.exp(-j / 40.0)
    if name == "out_of_core":
        return 0.9 ** j
    if name == "batched":
        return j ** -1.5
    raise KeyError(name)


# ---------------------------------------------------------------- numpy (CPU)
def qfactor_np(Z):
    """Q factor of Z with diag(R) > 0."""
    Q, R = np.linalg.qr(Z)
    s = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * s[None, :]


def lowrank_np(m, n, sigma, seed, offset_std=0.0, noise_std=0.0):
    """A = U0 diag(sigma) V0^T (+ 1 c^T, c ~ N(0, offset_std^2))
    (+ noise ~ N(0, noise_std^2)), FP64, rank len(sigma)."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    U0 = qfactor_np(rng.standard_normal((m, r)))
    V0 = qfactor_np(rng.standard_normal((n, r)))
    A = (U0 * np.asarray(sigma)[None, :]) @ V0.T
    if offset_std:
        A += offset_std * rng.standard_normal(n)[None, :]
    if noise_std:
        A += noise_std * rng.standard_normal((m, n))
    return A


def workload_np(name, m=None, n=None, seed=1007, rank_cap=1024):
    """FP64 matrix of workload ``name`` (optionally at a reduced size)."""
    cfg = CONFIGS[name]
    m = cfg["m"] if m is None else m
    n = cfg["n"] if n is None else n
    r = min(m, n, rank_cap) if name != "out_of_core" else min(64, m, n)
    sig = spectrum(name, r)
    return lowrank_np(m, n, sig, seed,
                      offset_std=1.0 if name == "fp32_center" else 0.0,
                      noise_std=NOISE_STD.get(name, 0.0))


def round_bf16_np(A):
    """Round FP64/FP32 values to bfloat16 (round to nearest, ties to even),
    returned as the FP32 numbers they represent."""
    x = np.ascontiguousarray(np.asarray(A, dtype=np.float32))
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).reshape(x.shape)


def bf16_bits_np(A):
    """uint16 bit patterns of round_bf16_np(A)."""
    r = round_bf16_np(A)
    return (r.view(np.uint32) >> 16).astype(np.uint16)


# ---------------------------------------------------------------- torch (GPU)
def _torch():
    import torch
    return torch


def lowrank_torch(m, n, sigma, seed, device, dtype=None, offset_std=0.0,
                  noise_std=0.0, chunk_rows=1 << 17):
    """Same construction as lowrank_np, generated with torch on ``device``:
    the tall Q factor by Cholesky QR twice (FP64 Gram), the n-side one by
    torch.linalg.qr, the product in FP32 row chunks.  The small
    factorisations run on the CPU, so the device needs no solver library.  Returns ``dtype``
    (FP32 default).  Different random stream from lowrank_np."""
    torch = _torch()
    dtype = torch.float32 if dtype is None else dtype
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    r = len(sigma)
    sig = torch.as_tensor(np.asarray(sigma), dtype=torch.float64, device=device)
    U0 = torch.randn(m, r, generator=g, device=device, dtype=torch.float32)
    Zv = torch.randn(n, r, generator=g, device=device, dtype=torch.float64)
    for _ in range(2):
        Gm = torch.zeros(r, r, dtype=torch.float64, device=device)
        for r0 in range(0, m, chunk_rows):
            blk = U0[r0:r0 + chunk_rows].double()
            Gm += blk.T @ blk
        L = torch.linalg.cholesky(Gm.cpu())
        Rinv = torch.linalg.inv(L.T).float().to(device)
        for r0 in range(0, m, chunk_rows):
            U0[r0:r0 + chunk_rows] = U0[r0:r0 + chunk_rows] @ Rinv
    Qv, Rv = (t.to(device) for t in torch.linalg.qr(Zv.cpu()))
    Qv = Qv * torch.where(torch.diagonal(Rv) < 0, -1.0, 1.0)[None, :]
    B = (Qv * sig[None, :]).T.contiguous().float()     # r x n
    A = torch.empty(m, n, dtype=dtype, device=device)
    c = None
    if offset_std:
        c = (offset_std * torch.randn(n, generator=g, device=device, dtype=torch.float64)).float()
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for r0 in range(0, m, chunk_rows):
            blk = U0[r0:r0 + chunk_rows] @ B
            if c is not None:
                blk += c[None, :]
            if noise_std:
                blk += noise_std * torch.randn(blk.shape, generator=g, device=device,
                                               dtype=torch.float32)
            A[r0:r0 + chunk_rows] = blk.to(dtype)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    del U0
    return A


def workload_torch(name, device, m=None, n=None, seed=1007, rank_cap=1024,
                   dtype=None):
    cfg = CONFIGS[name]
    m = cfg["m"] if m is None else m
    n = cfg["n"] if n is None else n
    r = min(m, n, rank_cap) if name != "out_of_core" else min(64, m, n)
    sig = spectrum(name, r)
    return lowrank_torch(m, n, sig, seed, device, dtype=dtype,
                         offset_std=1.0 if name == "fp32_center" else 0.0,
                         noise_std=NOISE_STD.get(name, 0.0))


def quantize_fp8_torch(A):
    """FP8-e4m3 storage with per-column FP32 scales s_j = amax_j / 448:
    stored = RNE(a / s_j) in e4m3.  Returns (uint8 tensor, scales FP32)."""
    torch = _torch()
    amax = A.abs().amax(dim=0).float()
    s = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax))
    q = (A.float() / s[None, :]).clamp(-448.0, 448.0).to(torch.float8_e4m3fn)
    return q.view(torch.uint8), s


def batched_shapes(count=512, seed=5510, m_range=(1000, 50000), n_range=(64, 1024)):
    """Per-problem (m, n) for the batched workload, uniform integers."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=count)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    return [(int(a), int(b)) for a, b in zip(ms, ns)]


def ceil_div(a, b):
    return -(-a // b)


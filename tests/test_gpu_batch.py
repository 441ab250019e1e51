"""Batches of independent problems (rpca_batch_*): every problem of a batch
matches the single-problem path (itself parity-tested against the oracle)
and the oracle, on the direct first run and on the CUDA-graph replay."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rpca_oracle as ro, estimator as est  # noqa: E402
from synth import generators as gen  # noqa: E402

pytestmark = pytest.mark.gpu

# BF16 storage: the tensor cores see X, H and Q rounded to BF16
BF16_ANGLE = 1e-2


def R():
    from paper_1007_5510_gb300 import rpca
    rpca.load_library()
    return rpca


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_batch_matches_single_problems_and_oracle(dtype):
    rpca = R()
    rng = np.random.default_rng(7)
    shapes = [(int(rng.integers(1000, 12000)), int(rng.integers(64, 600))) for _ in range(10)]
    shapes += [(900, 1000)]                     # n > m: transposed internally
    k, l, i = 8, 10, 1
    As64 = [gen.lowrank_np(m, n, np.arange(1, min(m, n) + 1) ** -1.5, seed=p) for p, (m, n) in enumerate(shapes)]
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    As = [torch.from_numpy(A.astype(np.float32)).cuda().to(tdt) for A in As64]
    code = rpca.BF16 if dtype == "bf16" else rpca.F32
    b = rpca.Batch(shapes, k, l, i, dtype=code, seeds=range(100, 100 + len(shapes)), nstreams=4)
    try:
        first = [tuple(t.clone() for t in o) for o in b.run(As)]
        outs = b.run(As)                          # recorded graph
        outs = b.run(As, outs)                    # replay
        torch.cuda.synchronize()
        # run-to-run spread: FP32 atomics add in no fixed order, which can flip
        # a BF16 rounding of X or H (BF16 storage) -> ~1e-5
        tol = 1e-4 if dtype == "bf16" else 1e-5
        for p, (m, n) in enumerate(shapes):
            U, S, V = outs[p]
            s1 = first[p][1].cpu().numpy()
            s = S.cpu().numpy()
            assert np.max(np.abs(s - s1) / s1) < tol, p
            Us, Ss, Vs = rpca.pca(As[p], k, l, i, seed=100 + p)
            assert np.max(np.abs(s - Ss.cpu().numpy()) / s) < tol, p
            Ao = As[p].float().cpu().double().numpy()
            Uo, So, Vo = ro.rpca(Ao, k, l, i, seed=100 + p, reorth=True)
            rel = np.max(np.abs(s - So) / So)
            au = est.max_principal_angle(U.cpu().double().numpy(), Uo)
            av = est.max_principal_angle(V.cpu().double().numpy(), Vo)
            print("PARITY batch %s problem %d (%d x %d) sigma_rel %.3e angle_U %.3e angle_V %.3e"
                  % (dtype, p, m, n, rel, au, av))
            s_tol, a_tol = (1e-3, BF16_ANGLE) if dtype == "bf16" else (1e-4, 1e-3)
            assert rel < s_tol and au < a_tol and av < a_tol, (p, rel, au, av)
    finally:
        b.close()

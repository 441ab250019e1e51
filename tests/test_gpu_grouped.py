"""Grouped batches (one launch per step over all problems): every problem
against the FP64 oracle on the same BF16 values, ragged shapes, both the
H-pass-only and the fused power step, the fall-back to per-problem contexts
when a matrix's layout does not fit TMA, the tuning knobs and the
autotuner's JSON cache."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rpca_oracle as ro, estimator as est  # noqa: E402
from synth import generators as gen  # noqa: E402

pytestmark = pytest.mark.gpu

# BF16 storage: X, H and Q reach the tensor cores rounded to BF16
S_TOL, A_TOL = 1e-3, 1e-2


def R():
    from paper_1007_5510_gb300 import rpca
    rpca.load_library()
    return rpca


def _problems(shapes, seed0=0, ld_pad=True):
    """Low-rank-plus-decay test matrices (sigma_j = j^-1.5), BF16 on the
    device with ld a multiple of 8 when ld_pad (TMA); the FP64 copies the
    oracle sees hold the same BF16 values."""
    As, Ao = [], []
    for p, (m, n) in enumerate(shapes):
        A = gen.lowrank_np(m, n, np.arange(1, min(m, n) + 1) ** -1.5, seed=seed0 + p)
        ld = (n + 7) // 8 * 8 if ld_pad else n
        buf = torch.zeros(m, ld, dtype=torch.bfloat16, device="cuda")
        buf[:, :n] = torch.from_numpy(A.astype(np.float32)).cuda().to(torch.bfloat16)
        As.append(buf[:, :n])
        Ao.append(buf[:, :n].float().cpu().double().numpy())
    return As, Ao


def _check(rpca, shapes, outs, Ao, k, l, i, seeds, label):
    worst = [0.0, 0.0, 0.0]
    for p, (m, n) in enumerate(shapes):
        U, S, V = outs[p]
        s = S.cpu().numpy()
        Uh, Vh = U.cpu().double().numpy(), V.cpu().double().numpy()
        # cheap checks first: a non-finite output must not reach LAPACK
        assert np.isfinite(s).all() and np.isfinite(Uh).all() and np.isfinite(Vh).all(), (label, p)
        Uo, So, Vo = ro.rpca(Ao[p], k, l, i, seed=seeds[p], reorth=True)
        rel = float(np.max(np.abs(s - So) / So))
        au = est.max_principal_angle(Uh, Uo)
        av = est.max_principal_angle(Vh, Vo)
        worst = [max(worst[0], rel), max(worst[1], au), max(worst[2], av)]
        assert np.all(np.diff(s) <= 0), (label, p)
        assert np.abs(Uh.T @ Uh - np.eye(k)).max() < 1e-4, (label, p)
        assert np.abs(Vh.T @ Vh - np.eye(k)).max() < 1e-4, (label, p)
        assert rel < S_TOL and au < A_TOL and av < A_TOL, (label, p, m, n, rel, au, av)
    print("PARITY grouped %s: %d problems, worst sigma_rel %.3e angle_U %.3e angle_V %.3e"
          % (label, len(shapes), *worst))


@pytest.mark.parametrize("i,l", [(1, 20), (2, 20), (0, 24), (1, 32)])
def test_grouped_batch_matches_oracle(i, l):
    rpca = R()
    rng = np.random.default_rng(11 + i)
    w = (i + 1) * l
    shapes = [(int(rng.integers(1000, 20000)), int(rng.integers(max(w, 64), 1025))) for _ in range(14)]
    shapes = [(m, min(n, 45056 // w)) for m, n in shapes]
    shapes += [(w + 3, w), (128, 64 if w <= 64 else w), (3001, 129), (20011, 1024 if w <= 44 else 45056 // w)]
    k = min(16, l - 2)
    seeds = list(range(300, 300 + len(shapes)))
    As, Ao = _problems(shapes, seed0=50 + i)
    b = rpca.Batch(shapes, k, l, i, dtype=rpca.BF16, seeds=seeds)
    try:
        assert b.grouped
        outs = b.run(As)
        torch.cuda.synchronize()
        assert b.grouped
        _check(rpca, shapes, outs, Ao, k, l, i, seeds, "i=%d l=%d" % (i, l))
        # a second run on the same buffers gives the same values (FP32
        # reductions add in no fixed order: BF16 roundings may flip)
        s1 = [o[1].clone() for o in outs]
        outs = b.run(As, outs)
        torch.cuda.synchronize()
        for p in range(len(shapes)):
            a, c = s1[p].cpu().numpy(), outs[p][1].cpu().numpy()
            assert np.max(np.abs(a - c) / a) < 1e-4, p
    finally:
        b.close()


def test_grouped_matches_per_problem_form():
    rpca = R()
    rng = np.random.default_rng(5)
    shapes = [(int(rng.integers(2000, 15000)), int(rng.integers(64, 700))) for _ in range(12)]
    k, l, i = 16, 20, 1
    seeds = list(range(40, 40 + len(shapes)))
    As, Ao = _problems(shapes, seed0=900)
    g = rpca.Batch(shapes, k, l, i, dtype=rpca.BF16, seeds=seeds)
    pp = rpca.Batch(shapes, k, l, i, dtype=rpca.BF16, seeds=seeds, grouped=False, nstreams=4)
    try:
        og = g.run(As)
        op = pp.run(As)
        torch.cuda.synchronize()
        assert g.grouped and not pp.grouped
        for p in range(len(shapes)):
            sg, sp = og[p][1].cpu().numpy(), op[p][1].cpu().numpy()
            assert np.isfinite(sg).all() and np.isfinite(og[p][0].cpu().numpy()).all(), p
            assert np.max(np.abs(sg - sp) / sp) < 1e-3, p
            assert est.max_principal_angle(og[p][0].cpu().double().numpy(),
                                           op[p][0].cpu().double().numpy()) < A_TOL, p
    finally:
        g.close()
        pp.close()


def test_grouped_falls_back_when_layout_does_not_fit_tma():
    rpca = R()
    shapes = [(3000, 201), (5001, 333), (2500, 64)]
    k, l, i = 8, 12, 1
    seeds = [7, 8, 9]
    As, Ao = _problems(shapes, seed0=70, ld_pad=False)   # ld = n, odd n: not 16-byte rows
    b = rpca.Batch(shapes, k, l, i, dtype=rpca.BF16, seeds=seeds)
    try:
        outs = b.run(As)
        torch.cuda.synchronize()
        assert not b.grouped
        _check(rpca, shapes, outs, Ao, k, l, i, seeds, "fallback")
    finally:
        b.close()


def test_grouped_tuning_and_autotuner_cache(tmp_path):
    rpca = R()
    rng = np.random.default_rng(9)
    shapes = [(int(rng.integers(3000, 12000)), int(rng.integers(64, 512))) for _ in range(8)]
    k, l, i = 12, 16, 1
    seeds = list(range(500, 508))
    As, Ao = _problems(shapes, seed0=600)
    b = rpca.Batch(shapes, k, l, i, dtype=rpca.BF16, seeds=seeds)
    try:
        base = [o[1].clone() for o in b.run(As)]
        b.tuning = (4, 4, 1024, 512, 0)
        assert b.tuning == (4, 4, 1024, 512, 0)
        outs = b.run(As)
        torch.cuda.synchronize()
        for p in range(len(shapes)):
            a, c = base[p].cpu().numpy(), outs[p][1].cpu().numpy()
            assert np.max(np.abs(a - c) / a) < 1e-4, p
        _check(rpca, shapes, outs, Ao, k, l, i, seeds, "tuned (4, 4, 1024, 512, 0)")
        cache = tmp_path / "tuning.json"
        chosen = b.tune(As, cache)
        data = json.loads(cache.read_text())["rpca_batch_tuning"]
        assert list(data.values()) == [list(chosen)]
        key = next(iter(data))
        assert key.startswith("bf16/n") and "/k12/l16/i1" in key
        # a cached key is applied without timing
        b.tuning = (3, 5, 4096, 2048, 16)
        assert b.tune(As, cache) == chosen
        assert b.tuning == chosen
        outs = b.run(As)
        torch.cuda.synchronize()
        _check(rpca, shapes, outs, Ao, k, l, i, seeds, "autotuned %s" % (chosen,))
    finally:
        b.close()

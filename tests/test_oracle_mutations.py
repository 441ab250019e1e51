"""Planted mistakes in the oracle (CPU only) must be caught by the pins.

Each mutation patches one step of the oracle with a plausible error (a
dropped term, a wrong sign or index, a transposed operand) and checks that
at least one of the independent pins fails on it.
"""
import numpy as np
import pytest

from oracle import philox, rpca_oracle as ro
from synth import generators as gen


def _pins_pass():
    """Independent checks: exact truncated SVD in the w = n case, the
    low-rank exact case with centring, and orthonormality."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 30))
    U, S, V = ro.rpca(A, 4, 15, 1, seed=11, block_rows=16)
    Ue, Se, VTe = np.linalg.svd(A, full_matrices=False)
    ok = np.allclose(S, Se[:4], rtol=1e-10)
    ok &= np.allclose(np.abs(np.sum(U * Ue[:, :4], axis=0)), 1.0, atol=1e-8)
    ok &= np.allclose(np.abs(np.sum(V * VTe[:4].T, axis=0)), 1.0, atol=1e-8)
    sig = np.array([4.0, 2.0, 1.0, 0.5])
    B = gen.lowrank_np(50, 20, sig, seed=2) + np.arange(20)[None, :]
    U2, S2, V2 = ro.rpca(B, 2, 6, 1, seed=3, center=True, block_rows=16)
    Bc = B - B.mean(axis=0)
    ok &= np.allclose(S2, np.linalg.svd(Bc, compute_uv=False)[:2], rtol=1e-9)
    ok &= np.allclose(U2.T @ U2, np.eye(2), atol=1e-10)
    # test matrix G matches its defining stream
    ok &= np.array_equal(philox.gaussian_matrix(1, 3, 2).ravel(), philox.gaussian(1, 0, 6))
    return bool(ok)


def test_unmutated_pins_pass():
    assert _pins_pass()


def _mut_t_times_no_transpose(self, Y):
    out = np.zeros((self.n, Y.shape[1]))
    for r0, r1, B in self.blocks():
        out += B.T @ Y[:r1 - r0]            # wrong rows of Y
    return out


def _mut_householder_sign(x):
    v, beta = _orig_house(x)
    return v, -beta


def _mut_svd_transpose(T, full_matrices=False):
    u, s, vh = _orig_svd(T, full_matrices=full_matrices)
    return u, s, vh.T                       # W^T used where W belongs


def _mut_center_sign(self):
    return -_orig_means(self)


_orig_house = ro._householder
_orig_svd = np.linalg.svd
_orig_means = ro.RowSource.column_means


@pytest.mark.parametrize("target,attr,repl", [
    (ro.RowSource, "t_times", _mut_t_times_no_transpose),
    (ro, "_householder", _mut_householder_sign),
    (ro.np.linalg, "svd", _mut_svd_transpose),
    (ro.RowSource, "column_means", _mut_center_sign),
])
def test_planted_mistake_is_caught(monkeypatch, target, attr, repl):
    monkeypatch.setattr(target, attr, repl)
    try:
        caught = not _pins_pass()
    except Exception:
        caught = True
    assert caught


def test_planted_power_step_drop_is_caught(monkeypatch):
    """Dropping A^T in the power step (H^(j) = A H^(j-1)) is a shape error or
    a wrong result."""
    orig = ro.RowSource.t_times

    def bad(self, Y):
        out = orig(self, Y)
        return out * 0.0 + np.random.default_rng(0).standard_normal(out.shape)
    monkeypatch.setattr(ro.RowSource, "t_times", bad)
    try:
        caught = not _pins_pass()
    except Exception:
        caught = True
    assert caught


def test_planted_plain_mean_is_caught(monkeypatch):
    """A single-pass streamed sum (no correction pass) misses the exactly
    rounded mean on offset columns."""
    import math

    def plain(self):
        t = np.zeros(self.n)
        for _, _, B in self.blocks():
            t += B.sum(axis=0)
        return t / self.m
    monkeypatch.setattr(ro.RowSource, "column_means", plain)
    rng = np.random.default_rng(12)
    m, n = 60_000, 7
    A = 1e6 * (1.0 + np.arange(n))[None, :] + 1e-3 * rng.standard_normal((m, n))
    c = ro.RowSource(A, block_rows=64).column_means()
    exact = np.array([math.fsum(A[:, j]) / m for j in range(n)])
    assert not np.all(np.abs(c - exact) <= 4 * np.spacing(np.abs(exact)))


def test_planted_rng_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(philox, "_M0", np.uint64(0xD2511F55))
    out = philox.philox4x32_10(np.zeros((1, 4), np.uint32), (np.uint32(0), np.uint32(0)))
    assert [int(x) for x in out[0]] != [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]

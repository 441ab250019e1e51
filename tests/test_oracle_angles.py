"""Pins of the oracle's subspace checker (``oracle.estimator.max_principal_angle``).

Every angle assertion of the parity tests rests on this function, so it is
pinned here against subspaces whose principal angles are known in closed
form (rotations of coordinate planes), against the independent SciPy routine
``scipy.linalg.subspace_angles`` (Bjorck-Golub), and against the invariances
the definition fixes: the angle depends on the spans only (any invertible
mixing of the columns), is symmetric, and is the LARGEST principal angle.
The comparison metric is the one the outputs U, V of Section 3 (Steps 5-6)
are judged by: the singular vectors are defined up to sign and, for equal
singular values, rotation, so only their spans are compared.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import estimator as est


def _rotated_plane(n, angles):
    """Qa = [e_1 .. e_p], Qb = [cos a_j e_j + sin a_j e_{p+j}]: the principal
    angles between span(Qa) and span(Qb) are exactly the a_j."""
    p = len(angles)
    Qa = np.zeros((n, p))
    Qb = np.zeros((n, p))
    for j, a in enumerate(angles):
        Qa[j, j] = 1.0
        Qb[j, j] = np.cos(a)
        Qb[p + j, j] = np.sin(a)
    return Qa, Qb


def angle_pins(f=None):
    """True if the checker passes every pin (used by the planted-mistake
    tests, which substitute a wrong checker for f)."""
    f = est.max_principal_angle if f is None else f
    ok = True
    # one rotated direction, the other shared: the angle is theta
    for th in (1e-9, 1e-5, 0.3, 1.0, np.pi / 2 - 1e-3, np.pi / 2):
        Qa, Qb = _rotated_plane(6, [th, 0.0])
        ok &= abs(f(Qa, Qb) - th) <= 1e-12 + 1e-9 * th
    # two different angles: the largest one, in either column order
    Qa, Qb = _rotated_plane(8, [0.2, 0.7])
    ok &= abs(f(Qa, Qb) - 0.7) < 1e-12
    ok &= abs(f(Qa, Qb[:, ::-1]) - 0.7) < 1e-12
    Qa, Qb = _rotated_plane(10, [0.05, 0.4, 0.1])
    ok &= abs(f(Qa, Qb) - 0.4) < 1e-12
    # spans only: mixing and scaling the columns changes nothing
    rng = np.random.default_rng(1)
    M = rng.standard_normal((3, 3)) + 3 * np.eye(3)
    ok &= abs(f(Qa @ M, Qb @ np.diag([1e3, 1.0, 1e-3])) - 0.4) < 1e-9
    # symmetric
    ok &= abs(f(Qb, Qa) - 0.4) < 1e-12
    # the same space in two bases: zero; an orthogonal space: pi/2
    A = np.linalg.qr(rng.standard_normal((40, 4)))[0]
    ok &= f(A, A @ np.linalg.qr(rng.standard_normal((4, 4)))[0]) < 1e-7
    C = np.linalg.qr(rng.standard_normal((40, 8)))[0]
    ok &= abs(f(C[:, :4], C[:, 4:]) - np.pi / 2) < 1e-12
    # an independent implementation (SciPy, Bjorck-Golub) on random subspaces
    for s in range(3):
        r = np.random.default_rng(10 + s)
        X = r.standard_normal((50, 5))
        Y = X + 0.3 * r.standard_normal((50, 5))
        ref = float(np.max(scipy.linalg.subspace_angles(X, Y)))
        ok &= abs(f(X, Y) - ref) < 1e-10
    return bool(ok)


def test_max_principal_angle_pins():
    assert angle_pins()


@pytest.mark.parametrize("th", [1e-8, 1e-3, 0.5, 1.2])
def test_rotated_plane_angle(th):
    Qa, Qb = _rotated_plane(5, [th])
    assert abs(est.max_principal_angle(Qa, Qb) - th) <= 1e-12 + 1e-9 * th


# ------------------------------------------------------- planted mistakes
def _wrong_basis(Qa, Qb):
    Qa = np.linalg.qr(np.asarray(Qa, np.float64))[0]
    Qb = np.linalg.qr(np.asarray(Qb, np.float64))[0]
    M = Qb - Qb @ (Qb.T @ Qb)                 # projects with the wrong basis
    return float(np.arcsin(min(1.0, np.linalg.norm(M, 2))))


def _cosine(Qa, Qb):
    Qa = np.linalg.qr(np.asarray(Qa, np.float64))[0]
    Qb = np.linalg.qr(np.asarray(Qb, np.float64))[0]
    s = np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2)
    return float(np.arccos(min(1.0, s)))      # arccos of a sine


def _no_orthonormalisation(Qa, Qb):
    Qa = np.asarray(Qa, np.float64)
    Qb = np.asarray(Qb, np.float64)
    s = np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2)
    return float(np.arcsin(min(1.0, s)))


def _frobenius(Qa, Qb):
    Qa = np.linalg.qr(np.asarray(Qa, np.float64))[0]
    Qb = np.linalg.qr(np.asarray(Qb, np.float64))[0]
    s = np.linalg.norm(Qb - Qa @ (Qa.T @ Qb))   # all angles mixed
    return float(np.arcsin(min(1.0, s)))


def _smallest(Qa, Qb):
    Qa = np.linalg.qr(np.asarray(Qa, np.float64))[0]
    Qb = np.linalg.qr(np.asarray(Qb, np.float64))[0]
    sv = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    return float(np.arccos(min(1.0, sv.max())))   # smallest angle instead


@pytest.mark.parametrize("bad", [_wrong_basis, _cosine, _no_orthonormalisation, _frobenius, _smallest])
def test_planted_angle_mistake_is_caught(bad):
    try:
        caught = not angle_pins(bad)
    except Exception:
        caught = True
    assert caught

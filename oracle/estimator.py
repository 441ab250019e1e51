"""Error measurement for the oracle tests (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``bound_factor`` -- the factor of eq. (sort_of_svd), Section 3:
      ||A - U S V^T||_2 <= sqrt((C k n)^(1/(2i+1)) + min(1, C/n)) sigma_{k+1}
  (C = 10: small failure probability; C = 100: negligible).
* ``power_estimate`` -- the Appendix estimate
      p_{j,k}(D) = max_q sqrt(||(D^T D)^j w_q|| / ||(D^T D)^(j-1) w_q||)
  with w_q i.i.d. standard Gaussian n-vectors, D applied only through
  products with D and D^T (the paper uses j = 6 and k = the rank).
  p_{j,k}(D) <= ||D||_2 always; p >= ||D||_2 / 2 with probability at least
  1 - (2n / ((2j-1) 16^j))^(k/2)   (eq. high_prob).
* ``spectral_error`` -- ||A - U S V^T||_2 exactly (dense SVD), small inputs.
* ``max_principal_angle`` -- largest principal angle between two subspaces,
  sin(theta) = ||(I - P_a) B||_2 for orthonormal bases.
"""
import numpy as np


def bound_factor(k, n, i, C=100.0):
    return np.sqrt((C * k * n) ** (1.0 / (2 * i + 1)) + min(1.0, C / n))


def bound_success_probability(n, j, k):
    """Lower bound on P(p_{j,k}(D) >= ||D||_2 / 2), eq. high_prob."""
    return 1.0 - (2.0 * n / ((2 * j - 1) * 16.0 ** j)) ** (k / 2.0)


def power_estimate(apply_D, apply_Dt, n, j=6, k=1, rng=None):
    """p_{j,k}(D) of the Appendix."""
    rng = np.random.default_rng(0) if rng is None else rng
    best = 0.0
    for _ in range(k):
        x = rng.standard_normal(n)
        prev = x
        for _step in range(j):
            cur = apply_Dt(apply_D(prev))          # (D^T D) prev
            if _step == j - 1:
                num, den = np.linalg.norm(cur), np.linalg.norm(prev)
            else:
                prev = cur
        if den > 0:
            best = max(best, np.sqrt(num / den))
    return best


def residual_operators(A, U, S, V):
    """x -> (A - U S V^T) x and y -> (A - U S V^T)^T y, never forming D."""
    A = np.asarray(A, np.float64)

    def D(x):
        return A @ x - U @ (S * (V.T @ x))

    def Dt(y):
        return A.T @ y - V @ (S * (U.T @ y))
    return D, Dt


def spectral_error(A, U, S, V):
    A = np.asarray(A, np.float64)
    return np.linalg.norm(A - (U * S[None, :]) @ V.T, 2)


def max_principal_angle(Qa, Qb):
    """Largest principal angle (radians) between span(Qa) and span(Qb), both
    with orthonormal columns and the same column count."""
    Qa = np.asarray(Qa, np.float64)
    Qb = np.asarray(Qb, np.float64)
    # orthonormalise defensively (FP32 inputs)
    Qa, _ = np.linalg.qr(Qa)
    Qb, _ = np.linalg.qr(Qb)
    M = Qb - Qa @ (Qa.T @ Qb)
    s = np.linalg.norm(M, 2)
    return float(np.arcsin(min(1.0, s)))

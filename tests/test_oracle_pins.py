"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Every check here is independent of the oracle's own arithmetic: published
known-answer vectors, closed forms, exact special cases, invariances,
bounds stated in the paper, and the printed results of its Tables 1-2.
"""
import os

import numpy as np
import pytest
import scipy.fft

from oracle import philox, rpca_oracle as ro, estimator as est
from synth import generators as gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ RNG pins
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        ctr = np.array([v[0:4]], dtype=np.uint32)
        out = philox.philox4x32_10(ctr, (np.uint32(v[4]), np.uint32(v[5])))
        assert [int(x) for x in out[0]] == v[6:10]


def test_box_muller_identity_and_moments():
    u1, u2 = philox.uniform_pairs(99, 0, 50_000)
    assert np.all(u1 > 0) and np.all(u1 < 1) and np.all(u2 > 0) and np.all(u2 < 1)
    z = philox.gaussian(99, 0, 100_000)
    # z0^2 + z1^2 = -2 ln u1 (Box-Muller radius)
    np.testing.assert_allclose(z[0::2] ** 2 + z[1::2] ** 2, -2 * np.log(u1), rtol=1e-12)
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1) < 0.02
    # different domains and seeds give different streams
    assert not np.allclose(philox.gaussian(99, 1, 10), philox.gaussian(99, 0, 10))
    assert not np.allclose(philox.gaussian(98, 0, 10), philox.gaussian(99, 0, 10))
    # G is row-major over the stream
    G = philox.gaussian_matrix(5, 7, 3)
    np.testing.assert_array_equal(G.ravel(), philox.gaussian(5, 0, 21))


# ------------------------------------------------------------ pivoted QR pins
def test_pivoted_qr_properties():
    rng = np.random.default_rng(3)
    H = rng.standard_normal((300, 12)) @ np.diag(10.0 ** -np.arange(12))
    Q, R, perm = ro.pivoted_qr(H)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-13)
    np.testing.assert_allclose(Q @ R, H[:, perm], atol=1e-13)
    assert np.allclose(R, np.triu(R))
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-12))          # pivoting order
    # same span as an unpivoted library QR
    Ql, _ = np.linalg.qr(H)
    assert est.max_principal_angle(Q, Ql) < 1e-10
    # rank-deficient input: still w orthonormal columns (Step 2 keeps all)
    Hd = np.hstack([H[:, :4], H[:, :4] * 2.0])
    Qd, Rd, _ = ro.pivoted_qr(Hd)
    np.testing.assert_allclose(Qd.T @ Qd, np.eye(8), atol=1e-12)
    np.testing.assert_allclose(Qd @ Rd, Hd[:, _], atol=1e-12)


# ------------------------------------------------ exact special cases (brute)
@pytest.mark.parametrize("m,n,k,l,i", [(8, 6, 2, 3, 1), (40, 30, 4, 15, 1), (50, 20, 3, 10, 1)])
def test_exact_when_Q_spans_range(m, n, k, l, i):
    """With (i+1)l = n the range of H is the range of A, so Steps 2-6 return
    the truncated SVD exactly."""
    rng = np.random.default_rng(m * n)
    A = rng.standard_normal((m, n))
    assert (i + 1) * l == n
    U, S, V = ro.rpca(A, k, l, i, seed=11)
    Ue, Se, VTe = np.linalg.svd(A, full_matrices=False)
    np.testing.assert_allclose(S, Se[:k], rtol=1e-12)
    np.testing.assert_allclose(np.abs(np.sum(U * Ue[:, :k], axis=0)), 1.0, atol=1e-10)
    np.testing.assert_allclose(np.abs(np.sum(V * VTe[:k].T, axis=0)), 1.0, atol=1e-10)


def test_exact_low_rank():
    """rank(A) <= (i+1)l: exact truncated SVD, also with i = 0."""
    rng = np.random.default_rng(1)
    sig = np.array([5.0, 3.0, 2.0, 1.0, 0.5])
    A = gen.lowrank_np(60, 25, sig, seed=4)
    for i in (0, 1):
        U, S, V = ro.rpca(A, 3, 5, i, G=rng.standard_normal((25, 5)))
        np.testing.assert_allclose(S, sig[:3], rtol=1e-12)
        D = A - (U * S) @ V.T
        np.testing.assert_allclose(np.linalg.norm(D, 2), sig[3], rtol=1e-10)


# ----------------------------------------- workload fp64_small: accuracy pins
@pytest.fixture(scope="module")
def small_run():
    cfg = gen.CONFIGS["fp64_small"]
    A = gen.workload_np("fp64_small")
    U, S, V, parts = ro.rpca(A, cfg["k"], cfg["l"], cfg["i"], seed=1007, return_parts=True)
    return A, U, S, V, parts, cfg


def test_orthonormal_outputs(small_run):
    A, U, S, V, parts, cfg = small_run
    k = cfg["k"]
    assert np.abs(U.T @ U - np.eye(k)).max() < 1e-12
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-12
    assert np.all(S[:-1] >= S[1:]) and np.all(S >= 0)


def test_error_bound_and_floor(small_run):
    """Eckart-Young floor (Section 3) <= error <= eq. (sort_of_svd) bound."""
    A, U, S, V, parts, cfg = small_run
    sig = gen.spectrum("fp64_small", 1000)
    err = est.spectral_error(A, U, S, V)
    k, n, i = cfg["k"], cfg["n"], cfg["i"]
    assert err >= sig[k] * (1 - 1e-9)
    assert err <= est.bound_factor(k, n, i, C=100) * sig[k]
    # in practice close to optimal
    assert err <= 1.5 * sig[k]


def test_interlacing(small_run):
    """0 <= sigma_j(A) - S_j <= ||A - U S V^T||_2  (Weyl / compression)."""
    A, U, S, V, parts, cfg = small_run
    sig = gen.spectrum("fp64_small", 1000)
    err = est.spectral_error(A, U, S, V)
    d = sig[: cfg["k"]] - S
    assert np.all(d >= -1e-12 * sig[0])
    assert np.all(d <= err * (1 + 1e-9))
    np.testing.assert_allclose(S, sig[: cfg["k"]], rtol=1e-4)


def test_raw_and_normalised_iterations_agree():
    """The normalised iteration (Remark on over/underflow, Section 3) spans
    the same H as the raw one: on a moderately conditioned problem both
    forms agree to rounding."""
    A, G, k, l, i = _rand_problem(10, i=2)
    U, S, V = ro.rpca(A, k, l, i, G=G)
    U2, S2, V2 = ro.rpca(A, k, l, i, G=G, normalize=True)
    np.testing.assert_allclose(S2, S, rtol=1e-10)
    assert est.max_principal_angle(U, U2) < 1e-8
    assert est.max_principal_angle(V, V2) < 1e-8


def test_normalised_iteration_is_the_accurate_one(small_run):
    """On fp64_small the raw block (A A^T) A G has condition ~1e15, so the
    raw form loses digits of the smallest kept singular values in FP64; the
    normalised form keeps them.  Both obey interlacing; the normalised one
    is closer to the prescribed spectrum."""
    A, U, S, V, parts, cfg = small_run
    U2, S2, V2 = ro.rpca(A, cfg["k"], cfg["l"], cfg["i"], seed=1007, normalize=True)
    sig = gen.spectrum("fp64_small", cfg["k"])
    assert np.all(S2 <= sig * (1 + 1e-12))
    assert np.all(np.abs(sig - S2) <= np.abs(sig - S) + 1e-14 * sig[0])
    assert abs(sig[-1] - S2[-1]) < 0.6 * abs(sig[-1] - S[-1])
    np.testing.assert_allclose(S2, S, rtol=1e-5)


def test_reorthogonalised_iteration_spans_the_same_space():
    """Block Lanczos reorthogonalisation (every new n-side block taken out of
    the span of the earlier ones) changes no span: on a moderately
    conditioned problem it agrees with the raw and normalised forms to
    rounding, and it is exact where Q spans range(A)."""
    A, G, k, l, i = _rand_problem(10, i=2)
    U, S, V = ro.rpca(A, k, l, i, G=G)
    U2, S2, V2 = ro.rpca(A, k, l, i, G=G, reorth=True)
    np.testing.assert_allclose(S2, S, rtol=1e-10)
    assert est.max_principal_angle(U, U2) < 1e-8
    assert est.max_principal_angle(V, V2) < 1e-8
    rng = np.random.default_rng(5)
    B = rng.standard_normal((40, 30))
    U3, S3, V3 = ro.rpca(B, 4, 15, 1, seed=11, reorth=True)
    np.testing.assert_allclose(S3, np.linalg.svd(B, compute_uv=False)[:4], rtol=1e-12)


def test_reorthogonalised_krylov_block_conditioning():
    """H = A [X^(0) .. X^(i)] with orthonormal blocks: its singular values
    lie in [sigma_min(A), sigma_max(A)] (a product with an orthonormal
    matrix compresses A), so kappa(H) <= kappa(A) -- whatever the spectrum
    decay that makes the normalised Krylov blocks nearly dependent."""
    sig = 0.5 ** np.arange(40)                    # kappa(A) = 2^39
    A = gen.lowrank_np(500, 40, sig, seed=3)
    _, _, _, parts = ro.rpca(A, 4, 6, 3, seed=2, reorth=True, return_parts=True)
    H = np.hstack(parts["H"])
    sv = np.linalg.svd(H, compute_uv=False)
    assert sv[0] <= sig[0] * (1 + 1e-12) and sv[-1] >= sig[-1] * (1 - 1e-6)
    _, _, _, pn = ro.rpca(A, 4, 6, 3, seed=2, normalize=True, return_parts=True)
    svn = np.linalg.svd(np.hstack(pn["H"]), compute_uv=False)
    assert sv[0] / sv[-1] < 1e-3 * svn[0] / svn[-1]


def test_reorthogonalised_form_is_the_accurate_one_on_the_centred_workload():
    """The centred j^-2 workload makes the normalised Krylov blocks nearly
    dependent (kappa(H) ~ 7e10), so in FP64 their U moves by ~1e-7 rad when
    only the order of the row sums changes (a row permutation); the
    reorthogonalised form (kappa(H) ~ 2e4) moves by ~1e-12: its result is
    set by the data, not by rounding."""
    A = gen.workload_np("fp32_center", m=8000, n=400)
    p = np.random.default_rng(3).permutation(A.shape[0])
    U, S, V = ro.rpca(A, 20, 22, 2, seed=7, center=True, reorth=True)
    U2, S2, V2 = ro.rpca(A[p], 20, 22, 2, seed=7, center=True, reorth=True)
    assert est.max_principal_angle(U[p], U2) < 1e-10
    assert est.max_principal_angle(V, V2) < 1e-10
    np.testing.assert_allclose(S2, S, rtol=1e-13)
    Un, _, _ = ro.rpca(A, 20, 22, 2, seed=7, center=True, normalize=True)
    Un2, _, _ = ro.rpca(A[p], 20, 22, 2, seed=7, center=True, normalize=True)
    assert est.max_principal_angle(Un[p], Un2) > 100 * est.max_principal_angle(U[p], U2)


# --------------------------------------------------------------- invariances
def _rand_problem(seed=0, m=300, n=120, k=6, l=8, i=1):  # noqa: E302
    A = gen.lowrank_np(m, n, 0.8 ** np.arange(n), seed) + 1e-3 * np.random.default_rng(seed).standard_normal((m, n))
    G = np.random.default_rng(seed + 1).standard_normal((n, l))
    return A, G, k, l, i


def test_row_permutation_invariance():
    A, G, k, l, i = _rand_problem(1)
    p = np.random.default_rng(7).permutation(A.shape[0])
    U, S, V = ro.rpca(A, k, l, i, G=G)
    Up, Sp, Vp = ro.rpca(A[p], k, l, i, G=G)
    np.testing.assert_allclose(Sp, S, rtol=1e-11)
    assert est.max_principal_angle(Up, U[p]) < 1e-9
    assert est.max_principal_angle(Vp, V) < 1e-9


def test_test_matrix_mixing_invariance():
    """Only span(G) matters: G -> G M with M invertible gives the same result."""
    A, G, k, l, i = _rand_problem(2)
    M = np.random.default_rng(3).standard_normal((l, l)) + 3 * np.eye(l)
    U, S, V = ro.rpca(A, k, l, i, G=G)
    U2, S2, V2 = ro.rpca(A, k, l, i, G=G @ M)
    np.testing.assert_allclose(S2, S, rtol=1e-9)
    assert est.max_principal_angle(U2, U) < 1e-8


def test_scaling():
    A, G, k, l, i = _rand_problem(3)
    U, S, V = ro.rpca(A, k, l, i, G=G)
    U2, S2, V2 = ro.rpca(-2.5 * A, k, l, i, G=G)
    np.testing.assert_allclose(S2, 2.5 * S, rtol=1e-11)
    assert est.max_principal_angle(V2, V) < 1e-9


def test_centering_shift_invariance_and_definition():
    """center=True equals running on A - 1 mean^T; adding 1 d^T changes nothing."""
    A, G, k, l, i = _rand_problem(4)
    d = np.random.default_rng(5).standard_normal(A.shape[1]) * 10
    U, S, V = ro.rpca(A, k, l, i, G=G, center=True)
    U2, S2, V2 = ro.rpca(A + d[None, :], k, l, i, G=G, center=True)
    Ac = A - A.mean(axis=0, keepdims=True)
    U3, S3, V3 = ro.rpca(Ac, k, l, i, G=G)
    np.testing.assert_allclose(S2, S, rtol=1e-9)
    np.testing.assert_allclose(S3, S, rtol=1e-11)
    assert est.max_principal_angle(V2, V) < 1e-8
    # centred left vectors are orthogonal to the ones vector
    assert np.abs(U.sum(axis=0)).max() < 1e-10


def test_column_means_match_the_exactly_rounded_mean():
    """Section 1's column means on columns with a large offset: within a few
    roundings of the exact mean (math.fsum is an exactly rounded sum), where a
    plain streamed sum errs by ~u log(m) |offset|."""
    import math
    rng = np.random.default_rng(12)
    m, n = 60_000, 7
    A = 1e6 * (1.0 + np.arange(n))[None, :] + 1e-3 * rng.standard_normal((m, n))
    src = ro.RowSource(A, block_rows=64)
    c = src.column_means()
    exact = np.array([math.fsum(A[:, j]) / m for j in range(n)])
    assert np.all(np.abs(c - exact) <= 4 * np.spacing(np.abs(exact)))


def test_transpose_rule():
    """n > m: the method runs on A^T (Section 3); with an exact-range setting
    both orientations give the truncated SVD."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((20, 50))
    U, S, V = ro.rpca(A, 4, 10, 1, seed=3)
    assert U.shape == (20, 4) and V.shape == (50, 4)
    Se = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(S, Se[:4], rtol=1e-12)


def test_streaming_block_size_irrelevant():
    A, G, k, l, i = _rand_problem(6)
    U, S, V = ro.rpca(A, k, l, i, G=G, block_rows=7)
    U2, S2, V2 = ro.rpca(A, k, l, i, G=G, block_rows=100000)
    np.testing.assert_allclose(S2, S, rtol=1e-12)


def test_on_the_fly_rows_match_stored():
    """Section 4.1: rows generated on demand give the stored-matrix result."""
    A, G, k, l, i = _rand_problem(8)
    U, S, V = ro.rpca(A, k, l, i, G=G)
    U2, S2, V2 = ro.rpca(lambda r0, r1: A[r0:r1], k, l, i, G=G, m=A.shape[0], n=A.shape[1],
                         block_rows=33)
    np.testing.assert_allclose(S2, S, rtol=1e-12)


def test_parameter_rules():
    A = np.zeros((10, 8))
    for bad in [(0, 2, 1), (8, 9, 0), (3, 2, 1), (2, 3, 2), (2, 3, -1)]:
        with pytest.raises(ro.ParameterError):
            ro.rpca(A, *bad, seed=1)


def test_single_pass_products():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((37, 11))
    X = rng.standard_normal((11, 3))
    s = rng.standard_normal(11)
    c = rng.uniform(0.5, 2, 11)
    H, F = ro.fused_pass_products(A, X, shift=s, col_scale=c)
    Ac = A * c[None, :] - s[None, :]
    np.testing.assert_allclose(H, Ac @ X, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(F, Ac.T @ (Ac @ X), rtol=1e-12, atol=1e-12)
    T = ro.t_pass_product(A, H, shift=s, col_scale=c)
    np.testing.assert_allclose(T, F, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------- Appendix estimator
def test_power_estimate_bounds():
    rng = np.random.default_rng(0)
    for trial in range(5):
        D = rng.standard_normal((60, 40)) @ np.diag(rng.uniform(0, 1, 40))
        nrm = np.linalg.norm(D, 2)
        p = est.power_estimate(lambda x: D @ x, lambda y: D.T @ y, 40, j=6, k=3,
                               rng=np.random.default_rng(trial))
        assert p <= nrm * (1 + 1e-12)
        assert p >= nrm / 2
    # probability bound of eq. (high_prob) with the paper's j = 6
    assert est.bound_success_probability(200_000, 6, 16) > 1 - 1e-10


def test_bound_factor_values():
    # sqrt((C k n)^(1/(2i+1)) + min(1, C/n)) at two hand-computed points
    assert est.bound_factor(1, 100, 0, C=100) == pytest.approx(np.sqrt(10000 + 1.0))
    assert est.bound_factor(10, 1000, 1, C=100) == pytest.approx(np.sqrt(1e6 ** (1 / 3) + 0.1))


# ------------------------------------------ printed results (Tables 1 and 2)
def _dct_example(kind, size):
    n = size
    j = np.arange(1, n + 1, dtype=np.float64)
    if kind == 1:
        S = np.where(j <= 20, 10.0 ** (-4 * (j - 1) / 19), 1e-4 / np.maximum(j - 20, 1) ** 0.1)
    else:
        S = np.where(j <= 3, 1.0, np.where(j <= 6, .67, np.where(j <= 9, .34, np.where(j <= 12, .01, .01 * (n - j) / (n - 13)))))
    E = scipy.fft.dct(np.eye(n), type=2, norm="ortho", axis=0)
    A = (E * S[None, :]) @ E.T           # E S F with F the (transposed) DCT-II
    return A, S


def _two_digits(x):
    return float("%.1e" % x)


@pytest.mark.parametrize("example,k,eps0,eps", [
    tuple(float(t) if "E" in t else int(t) for t in l.split())
    for l in open(os.path.join(GOLDEN, "paper_tables.txt")) if l.strip() and not l.startswith("#")])
def test_tables_1_2_eps_matches_eps0(example, k, eps0, eps):
    """Tables 1-2: the algorithm's error estimate equals the optimum eps0 to
    the two printed digits (i = 3, l = k + 2).  Run at n = m = 1024 instead
    of 2E5 (the error of the method is set by the spectrum near k, which the
    construction fixes independently of n)."""
    A, S = _dct_example(example, 1024)
    U, Sg, V = ro.rpca(A, k, k + 2, 3, seed=2010)
    err = est.spectral_error(A, U, Sg, V)
    D, Dt = est.residual_operators(A, U, Sg, V)
    p = est.power_estimate(D, Dt, A.shape[1], j=6, k=k, rng=np.random.default_rng(1))
    opt = S[k]                                   # sigma_{k+1}: best rank-k error
    # Appendix: p <= ||D||, within a factor 2, and typically within ~10%
    assert p <= err * (1 + 1e-12) and p >= 0.9 * err
    if example == 1 and k == 24:
        # The construction gives sigma_25 = 1e-4 / 5^(1/10) = 8.5e-5; the
        # printed eps0 = 1.0E-4 disagrees with it (recorded as a reading).
        # The flat j^(-1/10) tail makes this row the hardest: the error
        # stays within 10% of the optimum, and the printed 1.0E-4 is within
        # 20% of both.
        assert _two_digits(opt) == 8.5e-5
        assert opt <= err <= 1.1 * opt
        assert abs(eps - err) <= 0.2 * eps
    else:
        # the algorithm reaches the optimum to the printed digits
        assert _two_digits(err) == _two_digits(opt)
        assert _two_digits(opt) == eps0
        assert _two_digits(err) == eps

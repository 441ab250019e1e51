"""The Python binding rejects malformed arguments before any pointer reaches
the C-ABI (CPU only: every case fails a check that comes before the device
check, or the device check itself)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1007_5510_gb300 import rpca as R  # noqa: E402


def _ok():
    m, n, p = 64, 32, 8
    return (torch.zeros(m, n, dtype=torch.bfloat16), torch.zeros(n, p), torch.zeros(m, p), torch.zeros(n, p))


@pytest.mark.parametrize("case,word", [
    ("A_fp32", "dtype"), ("A_1d", "2-D"), ("A_cols_strided", "stride"),
    ("X_fp64", "dtype"), ("X_short", "rows"), ("X_long", "rows"), ("X_transposed", "stride"),
    ("H_short", "rows"), ("H_narrow", "columns"), ("H_bf16", "dtype"),
    ("F_short", "rows"), ("F_narrow", "columns"),
    ("all_on_cpu", "CUDA"),
])
def test_noalloc_binding_rejects(case, word):
    A, X, H, F = _ok()
    if case == "A_fp32":
        A = A.float()
    elif case == "A_1d":
        A = A.reshape(-1)
    elif case == "A_cols_strided":
        A = torch.zeros(64, 64, dtype=torch.bfloat16)[:, ::2]
    elif case == "X_fp64":
        X = X.double()
    elif case == "X_short":
        X = X[:-1]
    elif case == "X_long":
        X = torch.zeros(33, 8)
    elif case == "X_transposed":
        X = torch.zeros(8, 32).t()
    elif case == "H_short":
        H = H[:-1]
    elif case == "H_narrow":
        H = H[:, :-1]
    elif case == "H_bf16":
        H = H.to(torch.bfloat16)
    elif case == "F_short":
        F = F[:-1]
    elif case == "F_narrow":
        F = F[:, :-1]
    with pytest.raises(ValueError, match=word):
        R.fused_pass_noalloc(A, X, H=H, F=F)


@pytest.mark.parametrize("fn", ["fused_pass", "t_pass", "pca"])
def test_other_entries_check_operands(fn):
    A = torch.zeros(64, 32)
    with pytest.raises(ValueError):
        if fn == "fused_pass":
            R.fused_pass(A, torch.zeros(31, 4))             # X rows != n
        elif fn == "t_pass":
            R.t_pass(A, torch.zeros(63, 4))                 # Q rows != m
        else:
            R.pca(A.to(torch.int32), 2, 3, 1)               # not a storage type


def test_context_matrix_shape_is_checked():
    class Fake(R.PCA):
        def __init__(self):          # no library call: only the argument checks are exercised
            self.m, self.n, self.host_a, self.ctx = 10, 4, False, None
    ctx = Fake()
    with pytest.raises(ValueError, match="context"):
        ctx._matrix(torch.zeros(10, 5))
    with pytest.raises(ValueError, match="host_a"):
        ctx._matrix(torch.zeros(10, 4))                   # CPU tensor without host_a
    with pytest.raises(ValueError, match="stride"):
        ctx._matrix(torch.zeros(4, 10).t())


def _est_ok():
    m, n, kd = 40, 12, 3
    return torch.zeros(m, n), torch.zeros(m, kd), torch.ones(kd, dtype=torch.float64), torch.zeros(n, kd)


@pytest.mark.parametrize("case,word", [
    ("A_int", "dtype"), ("S_matrix", "vector"), ("S_empty", "rank"), ("S_too_long", "rank"),
    ("U_short", "rows"), ("U_narrow", "columns"), ("U_fp64", "dtype"), ("V_short", "rows"),
    ("V_transposed", "stride"), ("q_zero", "start vectors"), ("q_above_n", "start vectors"),
    ("j_zero", "power steps"), ("omega_shape", "omega"), ("scale_short", "col_scale"),
    ("all_on_cpu", "CUDA"),
])
def test_estimate_error_binding_rejects(case, word):
    """Every rejected argument fails before a pointer reaches the C-ABI."""
    A, U, S, V = _est_ok()
    kw = {}
    if case == "A_int":
        A = A.to(torch.int32)
    elif case == "S_matrix":
        S = torch.ones(3, 1, dtype=torch.float64)
    elif case == "S_empty":
        S = torch.ones(0, dtype=torch.float64)
    elif case == "S_too_long":
        S = torch.ones(13, dtype=torch.float64)
    elif case == "U_short":
        U = U[:-1]
    elif case == "U_narrow":
        U = U[:, :-1]
    elif case == "U_fp64":
        U = U.double()
    elif case == "V_short":
        V = V[:-1]
    elif case == "V_transposed":
        V = torch.zeros(3, 12).t()
    elif case == "q_zero":
        kw["q"] = 0
    elif case == "q_above_n":
        kw["q"] = 13
    elif case == "j_zero":
        kw["j"] = 0
    elif case == "omega_shape":
        kw["q"], kw["omega"] = 2, [[0.0] * 3] * 12
    elif case == "scale_short":
        kw["col_scale"] = torch.ones(11)
    with pytest.raises(ValueError, match=word):
        R.estimate_error(A, U, S, V, **kw)


@pytest.mark.parametrize("kw,word", [
    (dict(tol=0.0), "tol"), (dict(tol=-1.0), "tol"), (dict(k0=0), "k0"), (dict(kmax=2), "kmax"),
    (dict(kmax=13), "kmax"), (dict(oversample=-1), "oversample"), (dict(j=0), "j >= 1"),
    (dict(col_scale=torch.ones(5)), "col_scale"), (dict(), "CUDA"),
])
def test_pca_adaptive_binding_rejects(kw, word):
    args = dict(tol=1e-3, k0=4, kmax=8)
    args.update(kw)
    with pytest.raises(ValueError, match=word):
        R.pca_adaptive(torch.zeros(40, 12), **args)

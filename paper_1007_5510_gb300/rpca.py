"""Python binding of the C-ABI in include/rpca.h (argument marshalling only).

Every step of the PCA runs inside the CUDA library; this module passes
pointers, sizes and the CUDA stream.  PyTorch provides device memory and
streams.  If the library is missing the functions raise: there is no CPU
fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librpca.so")

OK, MORE = 0, 1
STATUS = {0: "RPCA_OK", 1: "RPCA_MORE", -1: "RPCA_EINVAL", -2: "RPCA_ENOMEM", -3: "RPCA_ECUDA",
          -4: "RPCA_ENODEV", -5: "RPCA_EBREAKDOWN", -6: "RPCA_ETIMEOUT", -7: "RPCA_ESTATE"}
F64, F32, BF16, FP8E4M3 = 0, 1, 2, 3
CENTER, HOST_A, SIMT, TIMING, ADJOINT, HOST_RESIDENT, KEEP_T_PASS = 0x1, 0x2, 0x4, 0x8, 0x10, 0x20, 0x40
NO_GROUPED = 0x80

EXPORTS = ["rpca_init", "rpca_pass", "rpca_finish", "rpca_destroy", "rpca_run", "rpca_rerun",
           "rpca_strerror", "rpca_last_error", "rpca_op_fused_pass", "rpca_op_t_pass",
           "rpca_op_qr", "rpca_op_small_svd", "rpca_gaussian", "rpca_kernel_launches",
           "rpca_phase_times", "rpca_op_gram", "rpca_op_apply", "rpca_op_fused_pass_noalloc",
           "rpca_batch_init", "rpca_batch_run", "rpca_batch_destroy", "rpca_batch_last_error",
           "rpca_backward", "rpca_test_arm_wait_expiry", "rpca_batch_backward", "rpca_last_run_passes",
           "rpca_batch_grouped", "rpca_batch_get_tuning", "rpca_batch_set_tuning", "rpca_batch_tune",
           "rpca_estimate_error", "rpca_run_adaptive"]


class RpcaError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s%s" % (STATUS.get(status, status), (": " + msg) if msg else ""))


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int32),
                ("l", ctypes.c_int32), ("i", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("G", ctypes.POINTER(ctypes.c_double)), ("dtype", ctypes.c_int),
                ("flags", ctypes.c_uint32), ("tile_rows", ctypes.c_int64),
                ("stream", ctypes.c_void_p)]


class Matrix(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("ld", ctypes.c_int64), ("col_scale", ctypes.c_void_p)]


_lib = None


def load_library(path=None):
    """Load librpca.so (build it with __graft_entry__.build()).  Loading does
    not touch the GPU."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    st = ctypes.c_int
    lib.rpca_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Problem)]
    lib.rpca_init.restype = st
    lib.rpca_pass.argtypes = [vp, ctypes.POINTER(Matrix)]
    lib.rpca_pass.restype = st
    lib.rpca_finish.argtypes = [vp, vp, i64, vp, vp, i64]
    lib.rpca_finish.restype = st
    lib.rpca_destroy.argtypes = [vp]
    lib.rpca_destroy.restype = None
    lib.rpca_run.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(Matrix), vp, i64, vp, vp, i64]
    lib.rpca_run.restype = st
    lib.rpca_rerun.argtypes = [vp, ctypes.POINTER(Matrix), vp, i64, vp, vp, i64]
    lib.rpca_rerun.restype = st
    lib.rpca_strerror.argtypes = [st]
    lib.rpca_strerror.restype = ctypes.c_char_p
    lib.rpca_last_error.argtypes = [vp]
    lib.rpca_last_error.restype = ctypes.c_char_p
    lib.rpca_op_fused_pass.argtypes = [st, i64, i64, i32, vp, i64, vp, vp, vp, i64, vp, i64, vp, i64, i32, vp]
    lib.rpca_op_fused_pass.restype = st
    lib.rpca_op_t_pass.argtypes = [st, i64, i64, i32, vp, i64, vp, vp, vp, i64, vp, i64, i32, vp]
    lib.rpca_op_t_pass.restype = st
    lib.rpca_op_qr.argtypes = [i32, i64, i32, i32, vp, i64, vp]
    lib.rpca_op_qr.restype = st
    lib.rpca_op_small_svd.argtypes = [i32, i64, i32, vp, i64, vp, vp, i64, vp, vp]
    lib.rpca_op_small_svd.restype = st
    lib.rpca_gaussian.argtypes = [u64, ctypes.c_uint32, i64, ctypes.POINTER(ctypes.c_double)]
    lib.rpca_gaussian.restype = st
    lib.rpca_kernel_launches.argtypes = []
    lib.rpca_kernel_launches.restype = u64
    lib.rpca_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i32, ctypes.POINTER(i32)]
    lib.rpca_phase_times.restype = i32
    lib.rpca_op_gram.argtypes = [i64, i32, i32, vp, i64, vp, i64, vp, i64, i32, vp]
    lib.rpca_op_gram.restype = st
    lib.rpca_op_apply.argtypes = [i64, i32, i32, vp, i64, vp, i64, ctypes.c_double, ctypes.c_double, vp, i64,
                                  i32, vp]
    lib.rpca_op_apply.restype = st
    lib.rpca_op_fused_pass_noalloc.argtypes = [i64, i64, i32, vp, i64, vp, i64, vp, i64, vp, i64, vp]
    lib.rpca_op_fused_pass_noalloc.restype = st
    lib.rpca_backward.argtypes = [vp, ctypes.POINTER(Matrix), vp, vp, i64]
    lib.rpca_backward.restype = st
    lib.rpca_batch_init.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(Problem), i32]
    lib.rpca_batch_init.restype = st
    lib.rpca_batch_run.argtypes = [vp, ctypes.POINTER(Matrix), ctypes.POINTER(vp), ctypes.POINTER(i64),
                                   ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64)]
    lib.rpca_batch_run.restype = st
    lib.rpca_batch_destroy.argtypes = [vp]
    lib.rpca_batch_destroy.restype = None
    lib.rpca_batch_last_error.argtypes = [vp]
    lib.rpca_batch_last_error.restype = ctypes.c_char_p
    lib.rpca_batch_grouped.argtypes = [vp]
    lib.rpca_batch_grouped.restype = i32
    lib.rpca_batch_get_tuning.argtypes = [vp, ctypes.POINTER(i32)]
    lib.rpca_batch_get_tuning.restype = st
    lib.rpca_batch_set_tuning.argtypes = [vp, ctypes.POINTER(i32)]
    lib.rpca_batch_set_tuning.restype = st
    lib.rpca_batch_tune.argtypes = [vp, ctypes.POINTER(Matrix), ctypes.POINTER(vp), ctypes.POINTER(i64),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.c_char_p,
                                    ctypes.POINTER(i32)]
    lib.rpca_batch_tune.restype = st
    dp = ctypes.POINTER(ctypes.c_double)
    lib.rpca_estimate_error.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(Matrix), vp, i64, vp, vp, i64, i32,
                                        i32, i32, dp, dp, dp]
    lib.rpca_estimate_error.restype = st
    lib.rpca_run_adaptive.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(Matrix), ctypes.c_double, i32, i32,
                                      vp, i64, vp, vp, i64, ctypes.POINTER(i32), dp]
    lib.rpca_run_adaptive.restype = st
    lib.rpca_batch_backward.argtypes = [vp, ctypes.POINTER(Matrix), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(i64)]
    lib.rpca_batch_backward.restype = st
    lib.rpca_last_run_passes.argtypes = [vp]
    lib.rpca_last_run_passes.restype = i32
    lib.rpca_test_arm_wait_expiry.argtypes = [i32, u64, i64]
    lib.rpca_test_arm_wait_expiry.restype = st
    if path is None:
        _lib = lib
    return lib


def _check(status, ctx=None):
    if status in (OK, MORE):
        return status
    msg = ""
    if ctx:
        msg = load_library().rpca_last_error(ctx).decode()
    raise RpcaError(status, msg)


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_shape(t, name, dtypes, rows=None, cols=None):
    """Validate a matrix argument before its pointer crosses the C-ABI: the
    library sees only a pointer and a leading dimension, so a wrong type is
    silently reinterpreted and a short buffer is read or written out of
    bounds.  Checks element type, rank 2, at least `rows` rows and `cols`
    columns, unit column stride and a row stride covering the columns.
    Raises ValueError."""
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s must be a torch tensor" % name)
    if t.dtype not in dtypes:
        raise ValueError("%s: dtype %s, expected one of %s" % (name, t.dtype, [str(d) for d in dtypes]))
    if t.dim() != 2:
        raise ValueError("%s must be a 2-D matrix, got %d dimensions" % (name, t.dim()))
    if rows is not None and t.shape[0] < rows:
        raise ValueError("%s has %d rows, needs at least %d" % (name, t.shape[0], rows))
    if cols is not None and t.shape[1] < cols:
        raise ValueError("%s has %d columns, needs at least %d" % (name, t.shape[1], cols))
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("%s must have unit column stride (row-major), got stride %s" % (name, t.stride()))
    if t.stride(0) < max(1, t.shape[1]) and t.shape[0] > 1:
        raise ValueError("%s: row stride %d is below its column count" % (name, t.stride(0)))


def _check_device(t, name, device=None):
    """t is a CUDA tensor (on `device` when given); raises ValueError."""
    if t.device.type != "cuda":
        raise ValueError("%s must be a CUDA tensor, got %s" % (name, t.device))
    if device is not None and t.device != device:
        raise ValueError("%s is on %s, expected %s" % (name, t.device, device))


def _check_mat(t, name, dtypes, rows=None, cols=None, device=None):
    _check_shape(t, name, dtypes, rows, cols)
    _check_device(t, name, device)


def dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    if t.dtype in (torch.uint8, getattr(torch, "float8_e4m3fn", None)):
        return FP8E4M3
    raise ValueError("unsupported dtype %s" % t.dtype)


def gaussian(seed, count, domain=0):
    """Library-side Philox/Box-Muller stream (host, no GPU needed)."""
    out = np.empty(int(count), dtype=np.float64)
    _check(load_library().rpca_gaussian(ctypes.c_uint64(seed), domain, int(count),
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def kernel_launches():
    return int(load_library().rpca_kernel_launches())


def arm_wait_expiry(kernel, limit_ns, withhold_stage):
    """Test hook: the next tensor-core launch of `kernel` (0 fused pass, 1 T
    pass) leaves one TMA stage unissued and bounds its waits by limit_ns."""
    _check(load_library().rpca_test_arm_wait_expiry(int(kernel), ctypes.c_uint64(int(limit_ns)),
                                                     int(withhold_stage)))


class PCA:
    """A context: rpca_init on construction, passes, finish, rerun."""

    def __init__(self, m, n, k, l, i, dtype=F32, seed=0, center=False, G=None, host_a=False,
                 tile_rows=0, simt=False, stream=None, timing=False, adjoint=False, host_resident=False,
                 keep_t_pass=False):
        """host_a: A is in host memory and every pass streams it in tiles;
        host_resident (with host_a): the first pass of each run copies it
        once into a device copy that the later passes read."""
        lib = load_library()
        self.m, self.n, self.k, self.l, self.i, self.dtype = m, n, k, l, i, dtype
        self.host_a = bool(host_a)
        flags = ((CENTER if center else 0) | (HOST_A if host_a else 0) | (SIMT if simt else 0)
                 | (ADJOINT if adjoint else 0) | (HOST_RESIDENT if host_resident else 0)
                 | (TIMING if timing else 0) | (KEEP_T_PASS if keep_t_pass else 0))
        self._G = None
        Gp = None
        if G is not None:
            self._G = np.ascontiguousarray(G, dtype=np.float64)
            Gp = self._G.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.stream = stream
        sp = _stream_ptr(stream)
        self.prob = Problem(m, n, k, l, i, ctypes.c_uint64(seed), Gp, dtype, flags, tile_rows, sp)
        self.ctx = ctypes.c_void_p()
        _check(lib.rpca_init(ctypes.byref(self.ctx), ctypes.byref(self.prob)))

    def _matrix(self, A, col_scale=None, ld=None):
        if tuple(A.shape) != (self.m, self.n):
            raise ValueError("A is %s, the context was made for %d x %d" % (tuple(A.shape), self.m, self.n))
        if isinstance(A, np.ndarray):
            if not self.host_a:
                raise ValueError("a host array needs a context made with host_a=True")
            if A.strides[1] != A.itemsize:
                raise ValueError("A must have unit column stride")
            data = A.ctypes.data
            ld = A.strides[0] // A.itemsize if ld is None else ld
        else:
            if self.n > 1 and A.stride(1) != 1:
                raise ValueError("A must have unit column stride (row-major)")
            if (A.device.type == "cuda") == self.host_a:
                raise ValueError("A on %s does not match host_a=%s" % (A.device, self.host_a))
            data = A.data_ptr()
            ld = A.stride(0) if ld is None else ld
        if col_scale is not None:
            _check_vec(col_scale, "col_scale", self.n, _torch().float32, col_scale.device)
            if col_scale.device.type != "cuda":
                raise ValueError("col_scale must be a CUDA tensor")
        return Matrix(ctypes.c_void_p(data), ld, None if col_scale is None else col_scale.data_ptr())

    def passes(self, A, col_scale=None):
        lib = load_library()
        mat = self._matrix(A, col_scale)
        while True:
            s = _check(lib.rpca_pass(self.ctx, ctypes.byref(mat)), self.ctx)
            if s == OK:
                break

    def finish(self, U=None, S=None, V=None):
        torch = _torch()
        cdt = torch.float64 if self.dtype == F64 else torch.float32
        dev = torch.device("cuda")
        if U is None:
            U = torch.empty(self.m, self.k, dtype=cdt, device=dev)
        if V is None:
            V = torch.empty(self.n, self.k, dtype=cdt, device=dev)
        if S is None:
            S = torch.empty(self.k, dtype=torch.float64, device=dev)
        _check(load_library().rpca_finish(self.ctx, _ptr(U), U.stride(0), _ptr(S), _ptr(V),
                                          V.stride(0)), self.ctx)
        return U, S, V

    def run(self, A, col_scale=None, U=None, S=None, V=None):
        """All passes + Steps 2-6 (rpca_rerun: no allocation)."""
        torch = _torch()
        cdt = torch.float64 if self.dtype == F64 else torch.float32
        if U is None:
            U = torch.empty(self.m, self.k, dtype=cdt, device="cuda")
        if V is None:
            V = torch.empty(self.n, self.k, dtype=cdt, device="cuda")
        if S is None:
            S = torch.empty(self.k, dtype=torch.float64, device="cuda")
        mat = self._matrix(A, col_scale)
        _check(load_library().rpca_rerun(self.ctx, ctypes.byref(mat), _ptr(U), U.stride(0),
                                         _ptr(S), _ptr(V), V.stride(0)), self.ctx)
        return U, S, V

    def passes_last_run(self):
        """Passes over A of the last run (i+2, or i+1 with T from the F blocks)."""
        return int(load_library().rpca_last_run_passes(self.ctx))

    def phase_times(self):
        """(list of per-phase ms summed over runs, run count) since last call."""
        buf = (ctypes.c_double * 64)()
        runs = ctypes.c_int32(0)
        n = load_library().rpca_phase_times(self.ctx, buf, 64, ctypes.byref(runs))
        return [buf[t] for t in range(n)], runs.value

    def backward(self, A, dS, dA=None):
        """dA = sum_j dS[j] dsigma_j/dA for the last run (context created with
        adjoint=True; A the same device matrix).  dS: k values."""
        torch = _torch()
        cdt = torch.float64 if self.dtype == F64 else torch.float32
        dS = torch.as_tensor(dS, dtype=torch.float64, device="cuda").contiguous()
        if dA is None:
            dA = torch.empty(self.m, self.n, dtype=cdt, device="cuda")
        mat = self._matrix(A)
        _check(load_library().rpca_backward(self.ctx, ctypes.byref(mat), _ptr(dS), _ptr(dA), dA.stride(0)),
               self.ctx)
        return dA

    def close(self):
        if self.ctx:
            load_library().rpca_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pca(A, k, l, i, seed=0, center=False, G=None, col_scale=None, simt=False):
    """Rank-k PCA of a device tensor A (FP64/FP32/BF16/FP8 bytes)."""
    _check_mat(A, "A", _storage_dtypes())
    _check_vec(col_scale, "col_scale", A.shape[1], _torch().float32, A.device)
    m, n = A.shape
    ctx = PCA(m, n, k, l, i, dtype_code(A), seed=seed, center=center, G=G, simt=simt)
    try:
        return ctx.run(A, col_scale=col_scale)
    finally:
        ctx.close()


def estimate_error(A, U, S, V, j=6, q=None, omega=None, seed=0, col_scale=None):
    """The Appendix estimate p_{j,q}(D) of ||A - U diag(S) V^T||_2 on the
    GPU (rpca_estimate_error).  omega: optional n x q start vectors (numpy,
    FP64); else the Philox stream of `seed`.  Returns (p, per-column p)."""
    import numpy as np
    torch = _torch()
    # shapes and types first, devices last
    _check_shape(A, "A", _storage_dtypes())
    m, n = A.shape
    cdt = torch.float64 if A.dtype == torch.float64 else torch.float32
    if getattr(S, "ndim", 1) != 1:
        raise ValueError("S must be a vector of singular values")
    kd = int(len(S))
    if kd < 1 or kd > min(m, n):
        raise ValueError("S has %d values: the rank must be in [1, min(m, n)]" % kd)
    _check_shape(U, "U", (cdt,), rows=m, cols=kd)
    _check_shape(V, "V", (cdt,), rows=n, cols=kd)
    q = kd if q is None else int(q)
    if q < 1 or q > n:
        raise ValueError("q = %d start vectors: needs 1 <= q <= n" % q)
    if int(j) < 1:
        raise ValueError("j = %d power steps: needs j >= 1" % int(j))
    om = None
    if omega is not None:
        om = np.ascontiguousarray(np.asarray(omega, np.float64))
        if om.shape != (n, q):
            raise ValueError("omega must be n x q")
    _check_vec(col_scale, "col_scale", n, torch.float32, A.device)
    _check_device(A, "A")
    _check_device(U, "U", A.device)
    _check_device(V, "V", A.device)
    Sd = torch.as_tensor(S, dtype=torch.float64, device=A.device).contiguous()
    prob = Problem(m, n, kd, kd, 0, ctypes.c_uint64(seed), None, dtype_code(A), 0, 0, _stream_ptr())
    mat = Matrix(ctypes.c_void_p(A.data_ptr()), A.stride(0),
                 ctypes.c_void_p(col_scale.data_ptr()) if col_scale is not None else None)
    est = ctypes.c_double()
    cols = (ctypes.c_double * q)()
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load_library().rpca_estimate_error(
        ctypes.byref(prob), ctypes.byref(mat), _ptr(U), U.stride(0), _ptr(Sd), _ptr(V), V.stride(0), kd, int(j), q,
        om.ctypes.data_as(dp) if om is not None else None, ctypes.byref(est), cols))
    return est.value, list(cols)


def pca_adaptive(A, tol, k0, kmax, oversample=2, i=2, j=6, seed=0, col_scale=None):
    """Rank chosen by doubling from k0 (at most kmax) until the Appendix
    estimate of the error is at most tol (rpca_run_adaptive).  Returns
    (U, S, V, k, eps) with U, S, V cut to rank k."""
    torch = _torch()
    _check_shape(A, "A", _storage_dtypes())
    m, n = A.shape
    if not (float(tol) > 0.0):
        raise ValueError("tol must be positive")
    if int(k0) < 1 or int(kmax) < int(k0) or int(kmax) > min(m, n):
        raise ValueError("needs 1 <= k0 <= kmax <= min(m, n), got k0 = %d, kmax = %d" % (int(k0), int(kmax)))
    if int(oversample) < 0 or int(i) < 0 or int(j) < 1:
        raise ValueError("needs oversample >= 0, i >= 0, j >= 1")
    _check_vec(col_scale, "col_scale", n, torch.float32, A.device)
    _check_device(A, "A")
    cdt = torch.float64 if A.dtype == torch.float64 else torch.float32
    U = torch.empty(m, kmax, dtype=cdt, device=A.device)
    V = torch.empty(n, kmax, dtype=cdt, device=A.device)
    S = torch.empty(kmax, dtype=torch.float64, device=A.device)
    prob = Problem(m, n, int(k0), int(k0) + int(oversample), int(i), ctypes.c_uint64(seed), None, dtype_code(A), 0,
                   0, _stream_ptr())
    mat = Matrix(ctypes.c_void_p(A.data_ptr()), A.stride(0),
                 ctypes.c_void_p(col_scale.data_ptr()) if col_scale is not None else None)
    k_out = ctypes.c_int32()
    eps = ctypes.c_double()
    _check(load_library().rpca_run_adaptive(ctypes.byref(prob), ctypes.byref(mat), float(tol), int(kmax), int(j),
                                            _ptr(U), U.stride(0), _ptr(S), _ptr(V), V.stride(0), ctypes.byref(k_out),
                                            ctypes.byref(eps)))
    k = k_out.value
    return U[:, :k], S[:k], V[:, :k], k, eps.value


def _pca_function():
    torch = _torch()

    class PCAFunction(torch.autograd.Function):
        """(U, S, V) = rank-k PCA of A with gradients of S with respect to A
        (G fixed by the seed); U and V take no gradient."""

        @staticmethod
        def forward(ctx, A, k, l, i, seed):
            obj = PCA(A.shape[0], A.shape[1], k, l, i, dtype_code(A), seed=seed, adjoint=True)
            U, S, V = obj.run(A.detach())
            ctx.obj = obj
            ctx.save_for_backward(A)
            ctx.mark_non_differentiable(U, V)
            return U, S, V

        @staticmethod
        def backward(ctx, gU, gS, gV):
            (A,) = ctx.saved_tensors
            dA = None
            if gS is not None:
                dA = ctx.obj.backward(A.detach(), gS.to(torch.float64)).to(A.dtype)
            ctx.obj.close()
            return dA, None, None, None, None

    return PCAFunction


_PCAF = None


def pca_autograd(A, k, l, i, seed=0):
    """Differentiable rank-k PCA: (U, S, V) with S differentiable in A."""
    global _PCAF
    if _PCAF is None:
        _PCAF = _pca_function()
    return _PCAF.apply(A, k, l, i, seed)


class Batch:
    """Independent PCAs of uneven shapes run together (rpca_batch_*).  BF16
    batches that fit the grouped kernels run every step as one launch over
    all problems (`grouped`); others get one context per problem over
    `nstreams` library streams, replayed as one CUDA graph from the second
    run with the same buffers on."""

    def __init__(self, shapes, k, l, i, dtype=BF16, seeds=None, nstreams=16, stream=None, adjoint=False,
                 grouped=True):
        """adjoint: every problem keeps what backward() needs (m >= n each;
        per-problem form).  grouped=False forces the per-problem form."""
        lib = load_library()
        self.shapes = [(int(m), int(n)) for m, n in shapes]
        self.k, self.dtype = k, dtype
        cnt = len(self.shapes)
        seeds = list(range(cnt)) if seeds is None else list(seeds)
        sp = _stream_ptr(stream)
        flags = (ADJOINT if adjoint else 0) | (0 if grouped else NO_GROUPED)
        arr = (Problem * cnt)()
        for p, (m, n) in enumerate(self.shapes):
            arr[p] = Problem(m, n, k, l, i, ctypes.c_uint64(seeds[p]), None, dtype, flags, 0, sp)
        self.ctx = ctypes.c_void_p()
        status = lib.rpca_batch_init(ctypes.byref(self.ctx), cnt, arr, nstreams)
        if status != OK:
            raise RpcaError(status, lib.rpca_batch_last_error(None).decode())
        self._keep = None

    @property
    def grouped(self):
        """True if the last run (before any run: the batch) is grouped."""
        return bool(load_library().rpca_batch_grouped(self.ctx))

    @property
    def tuning(self):
        """(H-pass stages, T-pass stages, rows per T item, rows per row item,
        L2 prefetch distance)."""
        t = (ctypes.c_int32 * 5)()
        _check(load_library().rpca_batch_get_tuning(self.ctx, t))
        return tuple(t)

    @tuning.setter
    def tuning(self, values):
        values = [int(v) for v in values]
        if len(values) != 5:
            raise ValueError("tuning takes 5 values")
        t = (ctypes.c_int32 * 5)(*values)
        _check(load_library().rpca_batch_set_tuning(self.ctx, t))

    def tune(self, As, cache_path=None, outs=None):
        """Autotunes the grouped kernels on these matrices (rpca_batch_tune;
        cached in the JSON file cache_path) and returns the chosen tuning."""
        outs, args = self._args(As, outs)
        chosen = (ctypes.c_int32 * 5)()
        path = None if cache_path is None else str(cache_path).encode()
        status = load_library().rpca_batch_tune(self.ctx, *args, path, chosen)
        if status != OK:
            raise RpcaError(status, load_library().rpca_batch_last_error(self.ctx).decode())
        return tuple(chosen)

    def _args(self, As, outs):
        torch = _torch()
        cnt = len(self.shapes)
        if len(As) != cnt:
            raise ValueError("expected %d matrices, got %d" % (cnt, len(As)))
        cdt = torch.float64 if self.dtype == F64 else torch.float32
        if outs is None:
            outs = [(torch.empty(m, self.k, dtype=cdt, device="cuda"), torch.empty(self.k, dtype=torch.float64, device="cuda"),
                     torch.empty(n, self.k, dtype=cdt, device="cuda")) for m, n in self.shapes]
        mats = (Matrix * cnt)()
        for p, A in enumerate(As):
            mats[p] = Matrix(ctypes.c_void_p(A.data_ptr()), A.stride(0), None)
        vp = ctypes.c_void_p
        U = (vp * cnt)(*[vp(o[0].data_ptr()) for o in outs])
        S = (vp * cnt)(*[vp(o[1].data_ptr()) for o in outs])
        V = (vp * cnt)(*[vp(o[2].data_ptr()) for o in outs])
        ldu = (ctypes.c_int64 * cnt)(*[o[0].stride(0) for o in outs])
        ldv = (ctypes.c_int64 * cnt)(*[o[2].stride(0) for o in outs])
        self._keep = (mats, U, S, V, ldu, ldv)
        return outs, (mats, U, ldu, S, V, ldv)

    def run(self, As, outs=None):
        """As: list of device tensors; returns [(U, S, V)] (allocated on the
        first call unless given; pass the same list again to replay)."""
        torch = _torch()
        lib = load_library()
        cnt = len(self.shapes)
        cdt = torch.float64 if self.dtype == F64 else torch.float32
        if outs is None:
            outs = [(torch.empty(m, self.k, dtype=cdt, device="cuda"), torch.empty(self.k, dtype=torch.float64, device="cuda"),
                     torch.empty(n, self.k, dtype=cdt, device="cuda")) for m, n in self.shapes]
        mats = (Matrix * cnt)()
        for p, A in enumerate(As):
            mats[p] = Matrix(ctypes.c_void_p(A.data_ptr()), A.stride(0), None)
        vp = ctypes.c_void_p
        U = (vp * cnt)(*[vp(o[0].data_ptr()) for o in outs])
        S = (vp * cnt)(*[vp(o[1].data_ptr()) for o in outs])
        V = (vp * cnt)(*[vp(o[2].data_ptr()) for o in outs])
        ldu = (ctypes.c_int64 * cnt)(*[o[0].stride(0) for o in outs])
        ldv = (ctypes.c_int64 * cnt)(*[o[2].stride(0) for o in outs])
        self._keep = (mats, U, S, V, ldu, ldv)
        status = lib.rpca_batch_run(self.ctx, mats, U, ldu, S, V, ldv)
        if status != OK:
            raise RpcaError(status, lib.rpca_batch_last_error(self.ctx).decode())
        return outs

    def backward(self, As, dSs, dAs=None):
        """dA[p] = sum_j dS[p][j] dsigma_j/dA for every problem of the last
        run (batch made with adjoint=True; As the same device matrices)."""
        torch = _torch()
        lib = load_library()
        cnt = len(self.shapes)
        cdt = torch.float64 if self.dtype == F64 else torch.float32
        dSs = [torch.as_tensor(d, dtype=torch.float64, device="cuda").contiguous() for d in dSs]
        if dAs is None:
            dAs = [torch.empty(m, n, dtype=cdt, device="cuda") for m, n in self.shapes]
        mats = (Matrix * cnt)()
        for p, A in enumerate(As):
            mats[p] = Matrix(ctypes.c_void_p(A.data_ptr()), A.stride(0), None)
        vp = ctypes.c_void_p
        dS = (vp * cnt)(*[vp(d.data_ptr()) for d in dSs])
        dA = (vp * cnt)(*[vp(d.data_ptr()) for d in dAs])
        ld = (ctypes.c_int64 * cnt)(*[d.stride(0) for d in dAs])
        self._keep_b = (mats, dS, dA, ld, dSs)
        status = lib.rpca_batch_backward(self.ctx, mats, dS, dA, ld)
        if status != OK:
            raise RpcaError(status, lib.rpca_batch_last_error(self.ctx).decode())
        return dAs

    def close(self):
        if self.ctx:
            load_library().rpca_batch_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------- single ops
def _storage_dtypes():
    torch = _torch()
    return tuple(d for d in (torch.float64, torch.float32, torch.bfloat16, torch.uint8,
                             getattr(torch, "float8_e4m3fn", None)) if d is not None)


def _check_vec(v, name, n, dtype, device):
    if v is None:
        return
    torch = _torch()
    if not isinstance(v, torch.Tensor) or v.dtype != dtype or v.numel() < n or not v.is_contiguous():
        raise ValueError("%s must be a contiguous %s vector of at least %d entries" % (name, dtype, n))
    if v.device != device:
        raise ValueError("%s is on %s, expected %s" % (name, v.device, device))


def fused_pass(A, X, shift=None, col_scale=None, with_f=True, kernel=0):
    """H = A_c X (and F = A_c^T H): one Step-1 pass.  Returns (H, F)."""
    torch = _torch()
    _check_shape(A, "A", _storage_dtypes())
    m, n = A.shape
    cdt = torch.float64 if A.dtype == torch.float64 else torch.float32
    _check_shape(X, "X", (cdt,), rows=n)
    if X.shape[0] != n:
        raise ValueError("X has %d rows, A has %d columns" % (X.shape[0], n))
    _check_device(A, "A")
    _check_device(X, "X", A.device)
    _check_vec(shift, "shift", n, cdt, A.device)
    _check_vec(col_scale, "col_scale", n, torch.float32, A.device)
    p = X.shape[1]
    H = torch.empty(m, p, dtype=cdt, device=A.device)
    F = torch.empty(n, p, dtype=cdt, device=A.device) if with_f else None
    _check(load_library().rpca_op_fused_pass(
        dtype_code(A), m, n, p, _ptr(A), A.stride(0), _ptr(col_scale), _ptr(shift), _ptr(X),
        X.stride(0), _ptr(H), H.stride(0), _ptr(F), (F.stride(0) if F is not None else 0),
        kernel, _stream_ptr()))
    return H, F


def fused_pass_noalloc(A, X, H=None, F=None, with_f=True):
    """The tensor-core fused pass (BF16 A, FP32 X) through the entry point
    that allocates no device memory; H and F may be passed preallocated.
    Every argument is checked here (type, shape, strides, device) because
    the C entry sees only pointers: raises ValueError."""
    torch = _torch()
    _check_shape(A, "A", (torch.bfloat16,))
    m, n = A.shape
    _check_shape(X, "X", (torch.float32,), rows=n)
    if X.shape[0] != n:
        raise ValueError("X has %d rows, A has %d columns" % (X.shape[0], n))
    p = X.shape[1]
    if H is not None:
        _check_shape(H, "H", (torch.float32,), rows=m, cols=p)
    if F is not None:
        _check_shape(F, "F", (torch.float32,), rows=n, cols=p)
    _check_device(A, "A")
    for t, nm in ((X, "X"), (H, "H"), (F, "F")):
        if t is not None:
            _check_device(t, nm, A.device)
    if H is None:
        H = torch.empty(m, p, dtype=torch.float32, device=A.device)
    if F is None and with_f:
        F = torch.empty(n, p, dtype=torch.float32, device=A.device)
    _check(load_library().rpca_op_fused_pass_noalloc(
        m, n, p, _ptr(A), A.stride(0), _ptr(X), X.stride(0), _ptr(H), H.stride(0), _ptr(F),
        (F.stride(0) if F is not None else 0), _stream_ptr()))
    return H, F


def t_pass(A, Q, shift=None, col_scale=None, kernel=0):
    """T = A_c^T Q (Step 3)."""
    torch = _torch()
    _check_shape(A, "A", _storage_dtypes())
    m, n = A.shape
    cdt = torch.float64 if A.dtype == torch.float64 else torch.float32
    _check_shape(Q, "Q", (cdt,), rows=m)
    if Q.shape[0] != m:
        raise ValueError("Q has %d rows, A has %d" % (Q.shape[0], m))
    _check_device(A, "A")
    _check_device(Q, "Q", A.device)
    _check_vec(shift, "shift", n, cdt, A.device)
    _check_vec(col_scale, "col_scale", n, torch.float32, A.device)
    w = Q.shape[1]
    T = torch.empty(n, w, dtype=cdt, device=A.device)
    _check(load_library().rpca_op_t_pass(
        dtype_code(A), m, n, w, _ptr(A), A.stride(0), _ptr(col_scale), _ptr(shift), _ptr(Q),
        Q.stride(0), _ptr(T), T.stride(0), kernel, _stream_ptr()))
    return T


def qr_inplace(H, nblk, l):
    """Step 2 on H (m x nblk*l): H <- Q."""
    torch = _torch()
    _check_mat(H, "H", (torch.float32, torch.float64), cols=nblk * l)
    f64 = 1 if H.dtype == torch.float64 else 0
    _check(load_library().rpca_op_qr(f64, H.shape[0], nblk, l, _ptr(H), H.stride(0), _stream_ptr()))
    return H


def gram(X, Y=None, kernel=0):
    """C = X^T Y (FP64) for FP32 device matrices."""
    torch = _torch()
    Y = X if Y is None else Y
    _check_mat(X, "X", (torch.float32,))
    _check_mat(Y, "Y", (torch.float32,), rows=X.shape[0], device=X.device)
    m, pp = X.shape
    q = Y.shape[1]
    C = torch.empty(pp, q, dtype=torch.float64, device=X.device)
    _check(load_library().rpca_op_gram(m, pp, q, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0), _ptr(C),
                                       C.stride(0), kernel, _stream_ptr()))
    return C


def apply(X, M, Y=None, alpha=1.0, beta=0.0, kernel=0):
    """Y = beta Y + alpha X M (X FP32, M FP64)."""
    torch = _torch()
    _check_mat(X, "X", (torch.float32,))
    m, pp = X.shape
    _check_mat(M, "M", (torch.float64,), rows=pp, device=X.device)
    q = M.shape[1]
    if Y is None:
        Y = torch.zeros(m, q, dtype=torch.float32, device=X.device)
    _check_mat(Y, "Y", (torch.float32,), rows=m, cols=q, device=X.device)
    _check(load_library().rpca_op_apply(m, pp, q, _ptr(X), X.stride(0), _ptr(M), M.stride(0), alpha, beta,
                                        _ptr(Y), Y.stride(0), kernel, _stream_ptr()))
    return Y


def small_svd(T):
    """Step 4: T = Vt diag(S) W^T; returns (S, Vt, W)."""
    torch = _torch()
    _check_mat(T, "T", (torch.float32, torch.float64))
    n, w = T.shape
    f64 = 1 if T.dtype == torch.float64 else 0
    S = torch.empty(w, dtype=torch.float64, device=T.device)
    Vt = torch.empty(n, w, dtype=T.dtype, device=T.device)
    W = torch.empty(w, w, dtype=torch.float64, device=T.device)
    _check(load_library().rpca_op_small_svd(f64, n, w, _ptr(T), T.stride(0), _ptr(S), _ptr(Vt),
                                            Vt.stride(0), _ptr(W), _stream_ptr()))
    return S, Vt, W

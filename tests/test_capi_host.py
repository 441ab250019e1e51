"""Host-side checks of the C-ABI library: loads without a GPU, exports every
symbol include/rpca.h declares, validates arguments, and its host Philox
stream matches the oracle's independent implementation."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import philox
from paper_1007_5510_gb300 import rpca

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rpca.h")


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rpca_[a-z_0-9]+)\s*\(", src)))


def test_header_and_exports(lib):
    decl = declared_functions()
    assert len(decl) >= 14
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(rpca.EXPORTS) == decl


def test_gaussian_stream_matches_oracle(lib):
    for seed, dom in [(0, 0), (1007, 0), (2 ** 40 + 5, 3)]:
        z_lib = rpca.gaussian(seed, 1001, domain=dom)
        z_orc = philox.gaussian(seed, dom, 1001)
        np.testing.assert_allclose(z_lib, z_orc, rtol=4e-15, atol=4e-15)


def _problem(**kw):
    d = dict(m=100, n=50, k=5, l=7, i=1, seed=1, G=None, dtype=rpca.F32, flags=0, tile_rows=0, stream=None)
    d.update(kw)
    return rpca.Problem(d["m"], d["n"], d["k"], d["l"], d["i"], d["seed"], d["G"], d["dtype"],
                        d["flags"], d["tile_rows"], d["stream"])


@pytest.mark.parametrize("kw", [dict(k=0), dict(k=50), dict(l=4), dict(i=-1), dict(l=30, i=1),
                                dict(m=0), dict(dtype=9), dict(flags=0x100), dict(l=200, i=1, m=900, n=800),
                                dict(flags=0x20)])     # RPCA_HOST_RESIDENT needs RPCA_HOST_A
def test_invalid_arguments(lib, kw):
    ctx = ctypes.c_void_p()
    p = _problem(**kw)
    assert lib.rpca_init(ctypes.byref(ctx), ctypes.byref(p)) == -1
    assert not ctx.value


def test_no_device_or_ok(lib):
    """Valid problem: without a GPU the library says ENODEV (no CPU path)."""
    import torch
    ctx = ctypes.c_void_p()
    p = _problem()
    s = lib.rpca_init(ctypes.byref(ctx), ctypes.byref(p))
    if torch.cuda.is_available():
        assert s == 0
        lib.rpca_destroy(ctx)
    else:
        assert s == -4


def test_strerror(lib):
    for code in rpca.STATUS:
        assert lib.rpca_strerror(code)
    assert lib.rpca_last_error(None) == b""


@pytest.mark.parametrize("n,p", [(4097, 16), (1000, 65), (0, 16), (1000, 0)])
def test_noalloc_rejects_sizes_beyond_its_scratch(lib, n, p):
    """Sizes outside the fixed scratch are refused on the host, before any
    device work (the dummy pointers are never dereferenced)."""
    d = ctypes.c_void_p(256)
    assert lib.rpca_op_fused_pass_noalloc(4096, n, p, d, max(n, 1), d, max(p, 1), d, max(p, 1), d,
                                          max(p, 1), None) == -1


def test_noalloc_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present; the GPU test covers this entry")
    lib = rpca.load_library()
    d = ctypes.c_void_p(256)
    assert lib.rpca_op_fused_pass_noalloc(4096, 1000, 16, d, 1000, d, 16, d, 16, d, 16, None) == -4


@pytest.mark.parametrize("kernel,limit,stage", [(2, 20_000_000, 0), (-1, 20_000_000, 0), (0, 10, 0),
                                                (1, 3_000_000_000, 0), (0, 20_000_000, -2)])
def test_wait_expiry_hook_checks_its_arguments(lib, kernel, limit, stage):
    assert lib.rpca_test_arm_wait_expiry(kernel, limit, stage) == -1


def test_wait_expiry_hook_arms_and_disarms(lib):
    """Arming is host state only (no device work); withhold -1 re-arms the
    default so no later launch is affected."""
    assert lib.rpca_test_arm_wait_expiry(0, 2_000_000_000, -1) == 0
    assert lib.rpca_test_arm_wait_expiry(1, 2_000_000_000, -1) == 0


@pytest.mark.parametrize("flags,expect_einval", [(0x1, True), (0x2, True), (0x0, False)])
def test_adaptive_rank_refuses_centred_or_host_matrices_first(lib, flags, expect_einval):
    """rpca_run_adaptive rejects RPCA_CENTER / RPCA_HOST_A before any run
    (the error estimate takes an uncentred device matrix); a valid call on a
    machine without a GPU reports ENODEV."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("the valid case would run on the GPU")
    m, n, kmax = 100, 50, 10
    A = np.zeros((m, n), np.float32)
    U = np.zeros((m, kmax), np.float32)
    V = np.zeros((n, kmax), np.float32)
    S = np.zeros(kmax, np.float64)
    p = _problem(flags=flags)
    mat = rpca.Matrix(ctypes.c_void_p(A.ctypes.data), n, None)
    k_out, eps = ctypes.c_int32(), ctypes.c_double()
    s = lib.rpca_run_adaptive(ctypes.byref(p), ctypes.byref(mat), 1e-3, kmax, 6, ctypes.c_void_p(U.ctypes.data), kmax,
                              ctypes.c_void_p(S.ctypes.data), ctypes.c_void_p(V.ctypes.data), kmax,
                              ctypes.byref(k_out), ctypes.byref(eps))
    assert s == (-1 if expect_einval else -4)

"""gbs_spmv_dots_noalloc: the allocation-free SpMV-with-dots entry point.

It exists for callers that cannot allocate device memory when they need
the operation (for example code running while a CUDA graph is captured,
or an application whose own allocator owns the GPU).  Its reduction
scratch is a fixed __device__ array inside the library, shared by every
call.  These checks call it through the C ABI twice in a row and compare
with the regular entry point gbs_spmv (which works from a hierarchy handle
built by gbs_build_hierarchy), at the SpMV tolerance used by the other
parity tests: |y - y_ref| <= 1e-13 (|A||x|)_i, and the same relative bound
for the two dot products.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import stokes_inputs as si
from oracle import bsr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06052_gb300 as gb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()
    return gb.load_library()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dtype)


@pytest.mark.parametrize("name,N", [("c2", 9), ("c1", 9)])
def test_noalloc_matches_regular_spmv_twice(name, N):
    s = si.make_system(name, N=N)
    B = s.bdim
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, B, gb.params_default(enable_adjoint=0))
    rp = _dev(s.indptr, torch.int32)
    ci = _dev(s.indices, torch.int32)
    va = _dev(s.data.reshape(-1))
    Ko = bsr.from_arrays(s.indptr, s.indices, s.data, B)
    A = Ko.scipy()
    rng = np.random.default_rng(17)
    y = torch.empty(s.n, dtype=torch.float64, device="cuda")
    for call in range(2):
        xh = rng.standard_normal(s.n)
        wh = rng.standard_normal(s.n)
        x, w = _dev(xh), _dev(wh)
        gb.spmv_dots_noalloc(rp, ci, va, B, x, y, w=w)
        _, dots = gb.spmv_dots_noalloc(rp, ci, va, B, x, y, w=w)
        y_lib = gb.spmv(H, x)
        torch.cuda.synchronize()
        yn = y.cpu().numpy()
        yr = bsr.spmv(Ko, xh)   # the oracle's SpMV
        bound = abs(A) @ np.abs(xh)
        assert np.all(np.abs(yn - yr) <= 1e-13 * bound + 1e-300), call
        assert np.all(np.abs(yn - y_lib.cpu().numpy()) <= 1e-13 * bound + 1e-300), call
        d = dots.cpu().numpy()
        ref_wy = float(np.dot(wh, yr))
        ref_yy = float(np.dot(yr, yr))
        scale_wy = float(np.dot(np.abs(wh), bound))
        assert abs(d[0] - ref_wy) <= 1e-13 * scale_wy + 1e-300, (call, d[0], ref_wy)
        assert abs(d[1] - ref_yy) <= 1e-13 * float(np.dot(bound, bound)), (call, d[1], ref_yy)


def test_noalloc_without_w_reports_zero_first_dot():
    """w = NULL: dots[0] is 0 and dots[1] is y . y, call after call (the
    scratch keeps the previous call's partial sums)."""
    s = si.make_system("c2", N=7)
    rp = _dev(s.indptr, torch.int32)
    ci = _dev(s.indices, torch.int32)
    va = _dev(s.data.reshape(-1))
    Ko = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    rng = np.random.default_rng(23)
    y = torch.empty(s.n, dtype=torch.float64, device="cuda")
    dots = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        xh = rng.standard_normal(s.n)
        gb.spmv_dots_noalloc(rp, ci, va, 4, _dev(xh), y, w=None, dots=dots)
        torch.cuda.synchronize()
        d = dots.cpu().numpy()
        yr = bsr.spmv(Ko, xh)
        bound = abs(Ko.scipy()) @ np.abs(xh)
        assert d[0] == 0.0, call
        assert abs(d[1] - float(np.dot(yr, yr))) <= 1e-13 * float(np.dot(bound, bound)), call


def test_noalloc_rejects_sizes_beyond_the_maximum():
    lib = gb.load_library()
    dots = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dots.data_ptr())
    st = lib.gbs_spmv_dots_noalloc(1, 1, 4, 2 ** 31, p, p, p, p, p, None, p, None)
    assert st == -1
    assert b"maximum" in lib.gbs_last_error()
    st = lib.gbs_spmv_dots_noalloc(2 ** 30, 1, 4, 1, p, p, p, p, p, None, p, None)
    assert st == -1

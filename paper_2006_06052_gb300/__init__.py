"""GB300 solve phase for Stokes saddle-point systems: Python binding.

Thin ctypes layer over the C ABI in ``include/gbstokes.h`` (same names,
argument marshalling only; every step of the solve runs in the CUDA
library).  Device vectors are torch CUDA float64 tensors; the library
works on the current torch stream.  Importing this package does not need
a GPU; calling into the library does, and fails loudly when the compiled
library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from ._build import LIB as _LIB_PATH, build as _build_lib

__all__ = [
    "GbsError", "Params", "Info", "Hierarchy", "params_default", "build_hierarchy",
    "import_hierarchy", "import_schur", "solve", "solve_adjoint", "sampled_outer", "update_values", "spmv",
    "apply_precond", "hierarchy_info", "export_level", "export_level_sizes", "spmv_dots_noalloc", "precond_bytes", "fp64_peak", "load_library", "build", "kernel_launches",
    "GBS_PC_AMG", "GBS_PC_SCHUR", "GBS_BICGSTAB", "GBS_GMRES", "GBS_IDRS", "GBS_FP64", "GBS_FP32",
    "GBS_BF16", "GBS_SPAI0", "GBS_JACOBI", "EXPORTED",
]

GBS_OK, GBS_NOT_CONVERGED = 0, 1
GBS_PC_AMG, GBS_PC_SCHUR = 0, 1
GBS_BICGSTAB, GBS_GMRES, GBS_IDRS = 0, 1, 2
GBS_FP64, GBS_FP32, GBS_BF16 = 0, 1, 2
GBS_SPAI0, GBS_JACOBI, GBS_ILUT = 0, 1, 2

STATUS = {0: "OK", 1: "NOT_CONVERGED", -1: "INVALID", -2: "CUDA", -3: "OOM",
          -4: "BREAKDOWN", -5: "NAN"}

# every symbol include/gbstokes.h declares
EXPORTED = [
    "gbs_params_default", "gbs_build_hierarchy", "gbs_solve", "gbs_solve_adjoint",
    "gbs_sampled_outer", "gbs_update_values", "gbs_spmv", "gbs_apply_precond",
    "gbs_hierarchy_info", "gbs_export_level", "gbs_import_hierarchy", "gbs_destroy",
    "gbs_last_error", "gbs_kernel_launches", "gbs_spmv_dots_noalloc", "gbs_precond_bytes",
    "gbs_outer_format", "gbs_level_apply", "gbs_import_schur", "gbs_fp64_peak",
    "gbs_level_format",
]


class GbsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("gbstokes %s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("precond", ctypes.c_int32), ("krylov", ctypes.c_int32), ("restart", ctypes.c_int32),
        ("tol", ctypes.c_double), ("maxiter", ctypes.c_int32), ("replace_every", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("eps_strong", ctypes.c_double),
        ("coarse_enough", ctypes.c_int32), ("max_levels", ctypes.c_int32),
        ("npre", ctypes.c_int32), ("npost", ctypes.c_int32), ("relax", ctypes.c_int32),
        ("relax_p", ctypes.c_int32), ("jacobi_omega", ctypes.c_double),
        ("smooth_P", ctypes.c_int32), ("power_iters", ctypes.c_int32), ("nvel", ctypes.c_int32),
        ("use_graph", ctypes.c_int32), ("enable_adjoint", ctypes.c_int32),
        ("setup_only", ctypes.c_int32), ("level_format", ctypes.c_int32),
        ("schur_p", ctypes.c_int32), ("schur_order", ctypes.c_int32),
        ("idr_s", ctypes.c_int32), ("idr_seed", ctypes.c_int32),
        ("ilut_p", ctypes.c_double), ("ilut_tau", ctypes.c_double),
        ("ilut_sweeps", ctypes.c_int32), ("ilut_omega", ctypes.c_double),
        ("gmres_reorth", ctypes.c_int32), ("wait_log2", ctypes.c_int32),
        ("iso_blocks", ctypes.c_int32),
    ]


class _Bsr(ctypes.Structure):
    _fields_ = [
        ("n_brows", ctypes.c_int32), ("n_bcols", ctypes.c_int32), ("bdim", ctypes.c_int32),
        ("nnzb", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
        ("vals", ctypes.c_void_p),
    ]


class _Levels(ctypes.Structure):
    _fields_ = [
        ("A", ctypes.c_void_p), ("P", ctypes.c_void_p), ("R", ctypes.c_void_p),
        ("M", ctypes.c_void_p), ("Ainv", ctypes.c_void_p), ("nlev", ctypes.c_int32),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32), ("replacements", ctypes.c_int32), ("converged", ctypes.c_int32),
        ("rel_res", ctypes.c_double), ("ms", ctypes.c_float),
        ("history", ctypes.POINTER(ctypes.c_double)), ("history_cap", ctypes.c_int32),
        ("history_len", ctypes.c_int32),
    ]

    status = 0

    def as_dict(self):
        return dict(iters=self.iters, replacements=self.replacements,
                    converged=bool(self.converged), rel_res=self.rel_res, ms=self.ms,
                    status=STATUS.get(self.status, self.status))


_lib = None


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile the CUDA library in-tree (sm_103a) and return its path."""
    return _build_lib(verbose=verbose, force=force)


def load_library():
    """Load libgbstokes.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("libgbstokes.so is not built (%s); run build() first" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    c = ctypes
    P = c.c_void_p
    sig = {
        "gbs_params_default": [c.POINTER(Params)],
        "gbs_build_hierarchy": [c.POINTER(_Bsr), c.POINTER(Params), P, c.POINTER(P)],
        "gbs_solve": [P, P, P, P, c.POINTER(Info)],
        "gbs_solve_adjoint": [P, P, P, P, c.POINTER(Info)],
        "gbs_sampled_outer": [P, P, P, c.c_double, P, P],
        "gbs_update_values": [P, P, P],
        "gbs_spmv": [P, P, P, c.c_int32, P],
        "gbs_apply_precond": [P, P, P, c.c_int32, P],
        "gbs_hierarchy_info": [P, c.c_int32, c.POINTER(c.c_int32), P, P, c.c_int32,
                               c.POINTER(c.c_int64)],
        "gbs_export_level": [P, c.c_int32, c.c_int32, c.c_int32, c.POINTER(c.c_int32),
                             c.POINTER(c.c_int32), c.POINTER(c.c_int64), P, P, P],
        "gbs_import_hierarchy": [c.POINTER(_Bsr), c.POINTER(_Bsr), c.POINTER(_Bsr),
                                 c.POINTER(P), P, c.c_int32, c.POINTER(Params), P, c.POINTER(P)],
        "gbs_import_schur": [c.POINTER(_Bsr), c.POINTER(_Levels), c.POINTER(_Levels), P,
                             c.POINTER(Params), P, c.POINTER(P)],
        "gbs_fp64_peak": [c.POINTER(c.c_double), c.POINTER(c.c_int32), P, P],
        "gbs_level_format": [P, c.c_int32, c.c_int32, c.POINTER(c.c_int32)],
        "gbs_destroy": [P],
        "gbs_precond_bytes": [P, c.POINTER(c.c_double)],
        "gbs_outer_format": [P, c.POINTER(c.c_int32), c.POINTER(c.c_int64)],
        "gbs_level_apply": [P, c.c_int32, c.c_int32, c.c_int32, P, P, P, P],
        "gbs_spmv_dots_noalloc": [c.c_int32, c.c_int32, c.c_int32, c.c_int64, P, P, P, P, P, P,
                                  P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = c.c_int
    lib.gbs_last_error.argtypes = []
    lib.gbs_last_error.restype = c.c_char_p
    lib.gbs_kernel_launches.argtypes = []
    lib.gbs_kernel_launches.restype = c.c_int64
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().gbs_kernel_launches())


def _check(st):
    if st < 0:
        raise GbsError(st, load_library().gbs_last_error().decode())
    return st


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, n=None, name="tensor"):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError("%s must be a CUDA float64 tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), n))
    return ctypes.c_void_p(t.data_ptr())


def params_default(**overrides) -> Params:
    p = Params()
    _check(load_library().gbs_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError("unknown parameter %r" % k)
        setattr(p, k, v)
    return p


class _HostBsr:
    """Keeps numpy arrays alive while the C struct points at them."""

    def __init__(self, indptr, indices, vals, bdim, n_bcols=None):
        self.indptr = np.ascontiguousarray(indptr, dtype=np.int32)
        self.indices = np.ascontiguousarray(indices, dtype=np.int32)
        self.vals = np.ascontiguousarray(vals, dtype=np.float64).reshape(-1)
        nbr = len(self.indptr) - 1
        self.c = _Bsr(nbr, nbr if n_bcols is None else n_bcols, bdim, len(self.indices),
                      self.indptr.ctypes.data, self.indices.ctypes.data, self.vals.ctypes.data)


@dataclass
class Hierarchy:
    handle: ctypes.c_void_p
    n: int
    bdim: int
    nnzb: int
    params: Params

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.gbs_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    def destroy(self):
        if self.handle:
            _check(load_library().gbs_destroy(self.handle))
            self.handle = None


def build_hierarchy(indptr, indices, vals, bdim, params: Params | None = None,
                    stream=None) -> Hierarchy:
    """Host CSR/BSR arrays of K -> device hierarchy (gbs_build_hierarchy)."""
    lib = load_library()
    params = params or params_default()
    A = _HostBsr(indptr, indices, vals, bdim)
    h = ctypes.c_void_p()
    sp = ctypes.c_void_p(0) if params.setup_only else _stream_ptr(stream)
    _check(lib.gbs_build_hierarchy(ctypes.byref(A.c), ctypes.byref(params), sp, ctypes.byref(h)))
    nb = len(A.indptr) - 1
    return Hierarchy(h, nb * bdim, bdim, len(A.indices), params)


class _LevelSet:
    """Host arrays of one hierarchy in the gbs_levels layout (kept alive
    while the C struct points at them)."""

    def __init__(self, levels_A, levels_P, levels_R, levels_M, Ainv, bdim):
        self.keep = []

        def arr(ls):
            objs = [_HostBsr(*t[:3], bdim, t[3] if len(t) > 3 else None) for t in ls]
            self.keep.extend(objs)
            a = (_Bsr * max(1, len(objs)))()
            for i, o in enumerate(objs):
                a[i] = o.c
            return a

        self.A = arr(levels_A)
        self.P = arr(levels_P)
        self.R = arr(levels_R)
        if levels_M is None:
            self.Ms, self.Mp = [], None
        else:
            self.Ms = [np.ascontiguousarray(m, dtype=np.float64).reshape(-1) for m in levels_M]
            self.Mp = (ctypes.c_void_p * max(1, len(self.Ms)))(
                *[m.ctypes.data for m in self.Ms])
        self.Ai = np.ascontiguousarray(Ainv, dtype=np.float64).reshape(-1)
        self.c = _Levels(ctypes.addressof(self.A), ctypes.addressof(self.P),
                         ctypes.addressof(self.R),
                         ctypes.addressof(self.Mp) if self.Mp is not None else None,
                         self.Ai.ctypes.data, len(levels_A))


def import_hierarchy(levels_A, levels_P, levels_R, levels_M, Ainv, bdim,
                     params: Params | None = None, stream=None) -> Hierarchy:
    """Caller-built levels -> device hierarchy (gbs_import_hierarchy).
    levels_A/P/R: lists of (indptr, indices, vals[, n_bcols]) host arrays."""
    lib = load_library()
    params = params or params_default()
    L = _LevelSet(levels_A, levels_P, levels_R, levels_M, Ainv, bdim)
    h = ctypes.c_void_p()
    _check(lib.gbs_import_hierarchy(L.A, L.P, L.R, L.Mp, ctypes.c_void_p(L.Ai.ctypes.data),
                                    L.c.nlev, ctypes.byref(params), _stream_ptr(stream),
                                    ctypes.byref(h)))
    k0 = L.keep[0]
    nb = len(k0.indptr) - 1
    return Hierarchy(h, nb * bdim, bdim, len(k0.indices), params)


def import_schur(indptr, indices, vals, vel, pres=None, pres_smoother=None,
                 params: Params | None = None, stream=None) -> Hierarchy:
    """Schur pressure correction from caller-built inner hierarchies
    (gbs_import_schur).  (indptr, indices, vals): K in (nvel+1)-blocks.
    vel / pres: (levels_A, levels_P, levels_R, levels_M, Ainv) of the
    velocity AMG (bdim nvel) and the pressure AMG (bdim 1; schur_p = 0);
    pres_smoother: the diagonal pressure smoother (schur_p = 1)."""
    lib = load_library()
    params = params or params_default(precond=GBS_PC_SCHUR)
    nv = params.nvel
    K = _HostBsr(indptr, indices, vals, nv + 1)
    V = _LevelSet(*vel, nv)
    Pl = _LevelSet(*pres, 1) if pres is not None else None
    ms = None
    if pres_smoother is not None:
        ms = np.ascontiguousarray(pres_smoother, dtype=np.float64).reshape(-1)
    h = ctypes.c_void_p()
    _check(lib.gbs_import_schur(ctypes.byref(K.c), ctypes.byref(V.c),
                                ctypes.byref(Pl.c) if Pl is not None else None,
                                ctypes.c_void_p(ms.ctypes.data) if ms is not None else None,
                                ctypes.byref(params), _stream_ptr(stream), ctypes.byref(h)))
    nb = len(K.indptr) - 1
    return Hierarchy(h, nb * (nv + 1), nv + 1, len(K.indices), params)


def _solve(fn, H, b, x, stream, history):
    import torch
    if x is None:
        x = torch.zeros_like(b)
    info = Info()
    hist = None
    if history:
        hist = (ctypes.c_double * history)()
        info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        info.history_cap = history
    st = fn(H.handle, _dptr(b, H.n, "b"), _dptr(x, H.n, "x"), _stream_ptr(stream),
            ctypes.byref(info))
    _check(st)
    info.status = st
    if hist is not None:
        info.hist = list(hist[: info.history_len])
    return x, info


def solve(H: Hierarchy, b, x=None, stream=None, history: int = 0):
    """Solve K x = b (x: initial guess, overwritten).  Returns (x, Info)."""
    return _solve(load_library().gbs_solve, H, b, x, stream, history)


def solve_adjoint(H: Hierarchy, g, lam=None, stream=None, history: int = 0):
    """Solve K^T lam = g.  Returns (lam, Info)."""
    return _solve(load_library().gbs_solve_adjoint, H, g, lam, stream, history)


def sampled_outer(H: Hierarchy, lam, x, alpha=-1.0, grad=None, stream=None):
    """grad[k,a,c] = alpha lam[B i + a] x[B j + c] on K's stored pattern."""
    import torch
    if grad is None:
        grad = torch.empty(H.nnzb * H.bdim * H.bdim, dtype=torch.float64, device=lam.device)
    _check(load_library().gbs_sampled_outer(H.handle, _dptr(lam, H.n, "lam"), _dptr(x, H.n, "x"),
                                            float(alpha),
                                            _dptr(grad, H.nnzb * H.bdim ** 2, "grad"),
                                            _stream_ptr(stream)))
    return grad


def spmv_dots_noalloc(row_ptr, col_idx, vals, bdim, x, y, w=None, dots=None, n_bcols=None,
                      stream=None):
    """y = A x and dots = [w.y, y.y] for a BSR matrix already in device memory
    (torch CUDA tensors: int32 row_ptr/col_idx, float64 vals), through
    gbs_spmv_dots_noalloc, which allocates nothing on the device."""
    import torch
    n_brows = row_ptr.numel() - 1
    if dots is None:
        dots = torch.zeros(2, dtype=torch.float64, device=x.device)
    for t, nm in ((row_ptr, "row_ptr"), (col_idx, "col_idx")):
        if not (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
            raise TypeError("%s must be a contiguous CUDA int32 tensor" % nm)
    nb = n_brows if n_bcols is None else n_bcols
    _check(load_library().gbs_spmv_dots_noalloc(
        n_brows, nb, bdim, col_idx.numel(), ctypes.c_void_p(row_ptr.data_ptr()),
        ctypes.c_void_p(col_idx.data_ptr()), _dptr(vals, col_idx.numel() * bdim * bdim, "vals"),
        _dptr(x, nb * bdim, "x"), _dptr(y, n_brows * bdim, "y"),
        _dptr(w, n_brows * bdim, "w") if w is not None else None, _dptr(dots, 2, "dots"),
        _stream_ptr(stream)))
    return y, dots


def update_values(H: Hierarchy, vals, stream=None):
    _check(load_library().gbs_update_values(H.handle, _dptr(vals, H.nnzb * H.bdim ** 2, "vals"),
                                            _stream_ptr(stream)))


def spmv(H: Hierarchy, x, y=None, transpose=False, stream=None):
    import torch
    if y is None:
        y = torch.empty_like(x)
    _check(load_library().gbs_spmv(H.handle, _dptr(x, H.n, "x"), _dptr(y, H.n, "y"),
                                   int(bool(transpose)), _stream_ptr(stream)))
    return y


def apply_precond(H: Hierarchy, r, z=None, transpose=False, stream=None):
    import torch
    if z is None:
        z = torch.empty_like(r)
    _check(load_library().gbs_apply_precond(H.handle, _dptr(r, H.n, "r"), _dptr(z, H.n, "z"),
                                            int(bool(transpose)), _stream_ptr(stream)))
    return z


def hierarchy_info(H: Hierarchy, which: int = 0):
    lib = load_library()
    nl = ctypes.c_int32()
    cap = 32
    rows = (ctypes.c_int32 * cap)()
    nnz = (ctypes.c_int64 * cap)()
    by = ctypes.c_int64()
    _check(lib.gbs_hierarchy_info(H.handle, which, ctypes.byref(nl), rows, nnz, cap,
                                  ctypes.byref(by)))
    k = nl.value
    return dict(nlevels=k, n_brows=list(rows[:k]), nnzb=list(nnz[:k]), bytes=by.value)


def precond_bytes(H: Hierarchy) -> float:
    """Algorithmic bytes of one preconditioner application (stored formats)."""
    v = ctypes.c_double()
    _check(load_library().gbs_precond_bytes(H.handle, ctypes.byref(v)))
    return v.value


def level_apply(H: Hierarchy, which: int, level: int, op: int, x, f, y=None, stream=None):
    """One level operation as the V-cycle runs it: op 0 y = f - A_l x, op 1 one
    relaxation sweep y = x + S (f - A_l x).  x, f, y: CUDA tensors of the
    level's scalar size, float64 for GBS_FP64 hierarchies, float32 otherwise."""
    import torch
    want = torch.float64 if H.params.precision == GBS_FP64 else torch.float32
    for name, t in (("x", x), ("f", f)):
        if not (t.is_cuda and t.dtype == want and t.is_contiguous()):
            raise GbsError(-1, "%s must be a contiguous CUDA %s tensor" % (name, want))
    if y is None:
        y = torch.empty_like(x)
    if y.dtype != want or y.numel() != x.numel() or f.numel() != x.numel():
        raise GbsError(-1, "x, f, y must have the same size and dtype")
    _check(load_library().gbs_level_apply(H.handle, which, level, op, x.data_ptr(), f.data_ptr(),
                                          y.data_ptr(), _stream_ptr(stream)))
    return y


def fp64_peak(stream=None):
    """(TFLOP/s, SM count): the device's measured FP64 FMA throughput."""
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    t, n = ctypes.c_double(), ctypes.c_int32()
    _check(load_library().gbs_fp64_peak(ctypes.byref(t), ctypes.byref(n),
                                        ctypes.c_void_p(sink.data_ptr()), _stream_ptr(stream)))
    return t.value, n.value


LEVEL_LAYOUTS = ("block", "csr", "sliced", "block slices")


def level_format(H: Hierarchy, which: int, level: int):
    """(layout name, fused) of level `level` of AMG `which`: the layout its
    forward products run in, and whether its zero-guess smoothing step is
    fused with the residual."""
    f = ctypes.c_int32()
    _check(load_library().gbs_level_format(H.handle, which, level, ctypes.byref(f)))
    return LEVEL_LAYOUTS[f.value & 3], bool(f.value & 4)


def level_iso(H: Hierarchy, which: int, level: int) -> bool:
    """Whether level `level` of AMG `which` runs as S (x) I_B: its blocks are
    multiples of the identity and one scalar operator acts on the B
    interleaved components (gbs_params.iso_blocks)."""
    f = ctypes.c_int32()
    _check(load_library().gbs_level_format(H.handle, which, level, ctypes.byref(f)))
    return bool(f.value & 8)


OUTER_FORMATS = ("block", "csr", "sliced")


def outer_format(H: Hierarchy):
    """(layout name, stored value entries) of the outer SpMV of K."""
    f, n = ctypes.c_int32(), ctypes.c_int64()
    _check(load_library().gbs_outer_format(H.handle, ctypes.byref(f), ctypes.byref(n)))
    return OUTER_FORMATS[f.value], n.value


def export_level_sizes(H: Hierarchy, which: int, level: int, part: int):
    """(n_brows, n_bcols, nnzb) of one level piece (see export_level)."""
    lib = load_library()
    nbr, nbc, nnzb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib.gbs_export_level(H.handle, which, level, part, ctypes.byref(nbr), ctypes.byref(nbc),
                                ctypes.byref(nnzb), None, None, None))
    return nbr.value, nbc.value, nnzb.value


def export_level(H: Hierarchy, which: int, level: int, part: int):
    """Host copy of one level piece: part 0 A, 1 P, 2 R -> (indptr, indices, vals
    [nnzb, B, B], n_bcols); 3 -> M [n, B, B]; 4 -> aggregate ids; 5 -> dense Ainv;
    ILUT levels: 6 L, 7 U (scalar CSR: indptr, indices, vals, n) and 8 the diagonal."""
    lib = load_library()
    nbr, nbc, nnzb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    args = (H.handle, which, level, part, ctypes.byref(nbr), ctypes.byref(nbc), ctypes.byref(nnzb))
    _check(lib.gbs_export_level(*args, None, None, None))
    if H.params.precond == GBS_PC_SCHUR:
        B = H.params.nvel if which == 0 else 1
    else:
        B = H.bdim
    if part in (6, 7):
        ptr = np.zeros(nbr.value + 1, dtype=np.int32)
        col = np.zeros(nnzb.value, dtype=np.int32)
        val = np.zeros(nnzb.value)
        _check(lib.gbs_export_level(*args, ptr.ctypes.data, col.ctypes.data, val.ctypes.data))
        return ptr, col, val, nbc.value
    if part == 8:
        val = np.zeros(nbr.value)
        _check(lib.gbs_export_level(*args, None, None, val.ctypes.data))
        return val
    if part in (0, 1, 2):
        ptr = np.zeros(nbr.value + 1, dtype=np.int32)
        col = np.zeros(nnzb.value, dtype=np.int32)
        val = np.zeros(nnzb.value * B * B)
        _check(lib.gbs_export_level(*args, ptr.ctypes.data, col.ctypes.data, val.ctypes.data))
        return ptr, col, val.reshape(-1, B, B), nbc.value
    if part == 3:
        val = np.zeros(nbr.value * B * B)
        _check(lib.gbs_export_level(*args, None, None, val.ctypes.data))
        return val.reshape(-1, B, B)
    if part == 4:
        col = np.zeros(nbr.value, dtype=np.int32)
        _check(lib.gbs_export_level(*args, None, col.ctypes.data, None))
        return col
    val = np.zeros(nbr.value * nbc.value)
    _check(lib.gbs_export_level(*args, None, None, val.ctypes.data))
    return val.reshape(nbr.value, nbc.value)

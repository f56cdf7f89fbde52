"""ctypes binding of ``libsbsolve.so`` (the C ABI declared in ``include/sbsolve.h``).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  Device buffers are passed as torch CUDA tensors (their ``data_ptr``)
or as raw integer device addresses; host diagonals as NumPy arrays.  The library
is loaded from this package directory; if it is missing the import fails with
instructions instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsbsolve.so")

SB_OK = 0
SB_ERR_INVALID_ARG = -1
SB_ERR_SINGULAR = -2
SB_ERR_CUDA = -3
SB_ERR_ALLOC = -4
SB_ERR_UNSUPPORTED = -5
SB_F64 = 0
SB_F32 = 1
SB_ARITH_NATIVE = 0
SB_ARITH_DF32 = 1
ARITH = {"native": SB_ARITH_NATIVE, "df32": SB_ARITH_DF32}
SB_MAT_DIFFUSION_DIRICHLET = 1
SB_MAT_HYPER_HINGED = 2
SB_MAT_HYPER_TRUNCATED = 3
SB_MAT_CH_NOFLUX = 4
SB_MAT_DIFFUSION_PERIODIC = 5
SB_MAT_CH_PERIODIC = 6
MATRIX_KINDS = {"diffusion": 1, "hinged": 2, "truncated": 3, "ch_noflux": 4, "diffusion_periodic": 5,
                "ch_periodic": 6}

_ERR_NAMES = {
    SB_ERR_INVALID_ARG: "SB_ERR_INVALID_ARG",
    SB_ERR_SINGULAR: "SB_ERR_SINGULAR",
    SB_ERR_CUDA: "SB_ERR_CUDA",
    SB_ERR_ALLOC: "SB_ERR_ALLOC",
    SB_ERR_UNSUPPORTED: "SB_ERR_UNSUPPORTED",
}


class SbError(RuntimeError):
    """A negative status returned by the library, with its sb_last_error() text."""

    def __init__(self, code: int, message: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {message}")
        self.code = code


_lib = None

_c_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); the full exported surface of include/sbsolve.h
SIGNATURES = {
    "sb_factor_shared_tri": (ctypes.c_int, [_c_i64, _dp, _dp, _dp, ctypes.POINTER(_vp)]),
    "sb_factor_shared_tri_periodic": (ctypes.c_int, [_c_i64, _dp, _dp, _dp, ctypes.POINTER(_vp)]),
    "sb_factor_shared_penta": (ctypes.c_int, [_c_i64, _dp, _dp, _dp, _dp, _dp, ctypes.POINTER(_vp)]),
    "sb_factor_shared_penta_periodic": (ctypes.c_int, [_c_i64, _dp, _dp, _dp, _dp, _dp,
                                                       ctypes.POINTER(_vp)]),
    "sb_factor_destroy": (None, [_vp]),
    "sb_factor_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_c_i64)]),
    "sb_solve_batched": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i64, ctypes.c_int, _vp]),
    "sb_solve_batched_adjoint": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i64, ctypes.c_int, _vp]),
    "sb_solve_batched_ex": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int,
                                           _c_i64, _c_i64, ctypes.c_int, _vp]),
    "sb_shape_get": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "sb_shape_set": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "sb_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, _c_i64,
                                   _c_i64, ctypes.c_int, _vp, _vp, ctypes.POINTER(ctypes.c_float)]),
    "sb_build_matrix": (ctypes.c_int, [ctypes.c_int, _c_i64, ctypes.c_double, _dp]),
    "sb_host_workspace_bytes": (ctypes.c_int, [_vp, _c_i64, _c_i64, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "sb_solve_batched_host": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, _c_i64,
                                             _c_i64, ctypes.c_int, _c_i64, _vp, ctypes.c_size_t, _vp]),
    "sb_refine_workspace_bytes": (ctypes.c_int, [_vp, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_size_t)]),
    "sb_solve_batched_refined": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i64, ctypes.c_int, ctypes.c_int,
                                                _vp, ctypes.c_size_t, _vp]),
    "sb_solve_batched_refined_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i64, ctypes.c_int,
                                                        ctypes.c_int, _vp]),
    "sb_solve_batched_groups": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _vp, _vp, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               _vp, _vp, _vp]),
    "sb_rollout_workspace_bytes": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64,
                                                  ctypes.POINTER(ctypes.c_size_t)]),
    "sb_rollout_forward": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i64, _c_i64, _c_i64, ctypes.c_int,
                                          _vp, ctypes.c_size_t, _vp]),
    "sb_rollout_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _c_i64, _c_i64, _c_i64, _c_i64,
                                           ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "sb_stepper_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_i64, ctypes.c_double,
                                         ctypes.c_double, ctypes.POINTER(_vp)]),
    "sb_stepper_destroy": (None, [_vp]),
    "sb_stepper_factor": (_vp, [_vp]),
    "sb_stepper_workspace_bytes": (ctypes.c_int, [_vp, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_size_t)]),
    "sb_stepper_run": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i64, ctypes.c_int, _c_i64, ctypes.c_int, _vp,
                                      ctypes.c_size_t, _vp]),
    "sb_stepper_run_coarsening": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i64, ctypes.c_int, _c_i64, _vp, _vp,
                                                 ctypes.c_size_t, _vp]),
    "sb_stepper_set_forcing": (ctypes.c_int, [_vp, ctypes.c_double, _dp]),
    "sb_stepper_refined_workspace_bytes": (ctypes.c_int, [_vp, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_size_t)]),
    "sb_stepper_run_refined": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i64, ctypes.c_int, ctypes.c_int, _c_i64,
                                              ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "sb_stepper_run_forced": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i64, _c_i64, ctypes.c_int, _vp]),
    "sb_device_timeouts": (ctypes.c_int, [ctypes.c_int, _vp]),
    "sb_measure_rates": (ctypes.c_int, [ctypes.c_int, _vp]),
    "sb_last_error": (ctypes.c_char_p, []),
    "sb_version": (ctypes.c_char_p, []),
}


def lib():
    """The loaded library (loaded on first use).  Raises if it was never built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2107_05395_gb300.build` "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != SB_OK:
        raise SbError(rc, lib().sb_last_error().decode())


def _host_f64(v, N):
    arr = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    if arr.shape != (N,):
        raise ValueError(f"diagonal must have shape ({N},), got {arr.shape}")
    return arr


def _dev_ptr(t):
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(t, dtype):
    if dtype is not None:
        return dtype
    import torch
    if t.dtype == torch.float64:
        return SB_F64
    if t.dtype == torch.float32:
        return SB_F32
    raise TypeError(f"unsupported tensor dtype {t.dtype}")


def _batch_shape(t, N, M, ld):
    """(M, ld) for a tensor of shape (N, ld) unless given explicitly."""
    if isinstance(t, int):
        if M is None or ld is None:
            raise ValueError("M and ld are required with raw device pointers")
        return M, ld
    if t.dim() != 2 or t.shape[0] != N or not t.is_contiguous():
        raise ValueError(f"expected a contiguous (N={N}, ld) tensor, got {tuple(t.shape)}")
    ld = t.shape[1] if ld is None else ld
    M = ld if M is None else M
    return M, ld


class Factor:
    """Owns one sb_factor handle (a single device copy of the shared factors)."""

    def __init__(self, handle: int, P: int, N: int, diags):
        self.handle = ctypes.c_void_p(handle)
        self.P = P
        self.N = N
        self.diags = tuple(np.array(d, dtype=np.float64) for d in diags)

    @property
    def kind(self):
        return "tri" if self.P == 1 else "penta"

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().sb_factor_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sb_factor_shared_tri(a, b, c) -> Factor:
    """Factorise the shared tridiagonal matrix (sub a, diag b, super c) once."""
    N = len(b)
    arrs = [_host_f64(v, N) for v in (a, b, c)]
    h = ctypes.c_void_p()
    _check(lib().sb_factor_shared_tri(N, *[x.ctypes.data_as(_dp) for x in arrs], ctypes.byref(h)))
    return Factor(h.value, 1, N, arrs)


def sb_factor_shared_tri_periodic(a, b, c) -> Factor:
    """Factorise a shared periodic tridiagonal matrix (section 3.3): a[0] and c[N-1]
    are the corner entries.  Solves with the handle apply the Sherman-Morrison
    correction."""
    N = len(b)
    arrs = [_host_f64(v, N) for v in (a, b, c)]
    h = ctypes.c_void_p()
    _check(lib().sb_factor_shared_tri_periodic(N, *[x.ctypes.data_as(_dp) for x in arrs],
                                               ctypes.byref(h)))
    return Factor(h.value, 1, N, arrs)


def sb_factor_shared_penta_periodic(a, b, c, d, e) -> Factor:
    """Factorise a shared cyclic pentadiagonal matrix (indices modulo N; a[0], a[1],
    b[0], d[N-1], e[N-2], e[N-1] are the corner entries).  Solves with the handle
    apply the rank-2 Sherman-Morrison-Woodbury correction."""
    N = len(c)
    arrs = [_host_f64(v, N) for v in (a, b, c, d, e)]
    h = ctypes.c_void_p()
    _check(lib().sb_factor_shared_penta_periodic(N, *[x.ctypes.data_as(_dp) for x in arrs],
                                                 ctypes.byref(h)))
    return Factor(h.value, 2, N, arrs)


def sb_factor_shared_penta(a, b, c, d, e) -> Factor:
    """Factorise the shared pentadiagonal matrix (offsets -2..+2) once."""
    N = len(c)
    arrs = [_host_f64(v, N) for v in (a, b, c, d, e)]
    h = ctypes.c_void_p()
    _check(lib().sb_factor_shared_penta(N, *[x.ctypes.data_as(_dp) for x in arrs], ctypes.byref(h)))
    return Factor(h.value, 2, N, arrs)


def sb_factor_info(f: Factor):
    P = ctypes.c_int()
    N = ctypes.c_int64()
    _check(lib().sb_factor_info(f.handle, ctypes.byref(P), ctypes.byref(N)))
    return P.value, N.value


def _solve(fn, f, rhs, x, M, ld, dtype, stream):
    x = rhs if x is None else x
    M, ld = _batch_shape(rhs, f.N, M, ld)
    code = _dtype_code(rhs, dtype) if not isinstance(rhs, int) else dtype
    _check(fn(f.handle, _dev_ptr(rhs), _dev_ptr(x), M, ld, code, _stream_handle(stream)))
    return x


def sb_solve_batched(f: Factor, rhs, x=None, M=None, ld=None, dtype=None, stream=None):
    """x_m = A^{-1} rhs_m for all systems (asynchronous on ``stream``).  ``x``
    defaults to ``rhs`` (in place)."""
    return _solve(lib().sb_solve_batched, f, rhs, x, M, ld, dtype, stream)


def sb_solve_batched_adjoint(f: Factor, rhs, x=None, M=None, ld=None, dtype=None, stream=None):
    """x_m = A^{-T} rhs_m for all systems, with the same factors."""
    return _solve(lib().sb_solve_batched_adjoint, f, rhs, x, M, ld, dtype, stream)


def sb_solve_batched_ex(f: Factor, rhs, x, transpose=False, arith="native", M=None, ld=None,
                        rhs_dtype=None, x_dtype=None, stream=None):
    """General solve: A x = rhs (or A^T x = rhs) with separate rhs / x storage types and
    an arithmetic mode ("native" or "df32", see include/sbsolve.h)."""
    M, ld = _batch_shape(rhs, f.N, M, ld)
    rt = _dtype_code(rhs, rhs_dtype) if not isinstance(rhs, int) else rhs_dtype
    xt = _dtype_code(x, x_dtype) if not isinstance(x, int) else x_dtype
    a = ARITH[arith] if isinstance(arith, str) else int(arith)
    _check(lib().sb_solve_batched_ex(f.handle, 1 if transpose else 0, _dev_ptr(rhs), rt, _dev_ptr(x),
                                     xt, M, ld, a, _stream_handle(stream)))
    return x


SB_ALGO_SEQUENTIAL = 0
SB_ALGO_PARTITIONED = 1
SB_ALGO_STAGED = 2
SB_ALGO_TWO_ENDED = 3


class Shape(ctypes.Structure):
    """sb_shape: threads per CTA, resident CTAs per SM (0 = max), systems per thread,
    algorithm (SB_ALGO_SEQUENTIAL, SB_ALGO_PARTITIONED, SB_ALGO_STAGED or SB_ALGO_TWO_ENDED)."""
    _fields_ = [("threads", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("systems_per_thread", ctypes.c_int), ("algorithm", ctypes.c_int)]

    def as_tuple(self):
        return (self.threads, self.ctas_per_sm, self.systems_per_thread, self.algorithm)


def _arith_code(arith):
    return ARITH[arith] if isinstance(arith, str) else int(arith)


def sb_shape_get(f: Factor, arith="native", rhs_dtype=SB_F64, x_dtype=SB_F64):
    out = Shape()
    _check(lib().sb_shape_get(f.handle, _arith_code(arith), rhs_dtype, x_dtype, ctypes.byref(out)))
    return out.as_tuple()


def sb_shape_set(f: Factor, shape, arith="native", rhs_dtype=SB_F64, x_dtype=SB_F64):
    """shape: (threads, ctas_per_sm, systems_per_thread[, algorithm]); the algorithm
    defaults to SB_ALGO_SEQUENTIAL."""
    s = Shape(*shape)
    _check(lib().sb_shape_set(f.handle, _arith_code(arith), rhs_dtype, x_dtype, ctypes.byref(s)))


def sb_autotune(f: Factor, rhs, x, transpose=False, arith="native", M=None, ld=None, stream=None):
    """Times every candidate launch shape on (rhs, x) and stores the fastest; returns
    ((threads, ctas_per_sm, systems_per_thread, algorithm), ms).  Overwrites x; blocking."""
    M, ld = _batch_shape(rhs, f.N, M, ld)
    best = Shape()
    ms = ctypes.c_float()
    _check(lib().sb_autotune(f.handle, 1 if transpose else 0, _dev_ptr(rhs), _dtype_code(rhs, None),
                             _dev_ptr(x), _dtype_code(x, None), M, ld, _arith_code(arith),
                             _stream_handle(stream), ctypes.byref(best), ctypes.byref(ms)))
    return best.as_tuple(), ms.value


def sb_build_matrix(kind, N: int, coef: float):
    """Diagonals of a workload matrix I + coef*K (see include/sbsolve.h) as a
    tuple of 3 (tridiagonal) or 5 (pentadiagonal) NumPy arrays, offsets -P..P."""
    code = MATRIX_KINDS[kind] if isinstance(kind, str) else int(kind)
    P = 1 if code in (SB_MAT_DIFFUSION_DIRICHLET, SB_MAT_DIFFUSION_PERIODIC) else 2
    out = np.zeros((2 * P + 1) * N, dtype=np.float64)
    _check(lib().sb_build_matrix(code, N, float(coef), out.ctypes.data_as(_dp)))
    return tuple(out.reshape(2 * P + 1, N))


def sb_host_workspace_bytes(f: Factor, M, chunk_systems=0, rhs_dtype=SB_F64, x_dtype=SB_F64):
    out = ctypes.c_size_t()
    _check(lib().sb_host_workspace_bytes(f.handle, M, chunk_systems, rhs_dtype, x_dtype, ctypes.byref(out)))
    return out.value


def sb_solve_batched_host(f: Factor, rhs_host, x_host, work, transpose=False, arith="native",
                          chunk_systems=0, M=None, ld=None, stream=None):
    """Solve a batch held in host memory (CPU torch tensors, ideally pinned):
    chunked host->device copy, solve and device->host copy, overlapped on internal
    streams; asynchronous on `stream`."""
    M, ld = _batch_shape(rhs_host, f.N, M, ld)
    _check(lib().sb_solve_batched_host(f.handle, 1 if transpose else 0, _dev_ptr(rhs_host),
                                       _dtype_code(rhs_host, None), _dev_ptr(x_host), _dtype_code(x_host, None),
                                       M, ld, _arith_code(arith), int(chunk_systems), _dev_ptr(work),
                                       _nbytes(work), _stream_handle(stream)))
    return x_host


def sb_refine_workspace_bytes(f: Factor, M, ld=None):
    out = ctypes.c_size_t()
    _check(lib().sb_refine_workspace_bytes(f.handle, M, M if ld is None else ld, ctypes.byref(out)))
    return out.value


def _nbytes(t):
    return 0 if t is None else (t.numel() * t.element_size())


def sb_solve_batched_refined(f: Factor, rhs, x, n_refine=2, residual_arith="native", work=None,
                             M=None, ld=None, stream=None):
    """FP32 rhs -> FP64 x with FP32 sweeps and n_refine residual corrections."""
    M, ld = _batch_shape(rhs, f.N, M, ld)
    _check(lib().sb_solve_batched_refined(f.handle, _dev_ptr(rhs), _dev_ptr(x), M, ld, int(n_refine),
                                          _arith_code(residual_arith),
                                          None if work is None else _dev_ptr(work), _nbytes(work),
                                          _stream_handle(stream)))
    return x


def sb_solve_batched_refined_noalloc(f: Factor, rhs, x, n_refine=2, residual_arith="native",
                                     M=None, ld=None, stream=None):
    """Refined solve that allocates nothing: the FP32 scratch is the library's own
    16 MiB device array, so (N-1)*ld + M must not exceed 4194304.  Calls that run
    concurrently on the GPU share that array and must not overlap."""
    M, ld = _batch_shape(rhs, f.N, M, ld)
    _check(lib().sb_solve_batched_refined_noalloc(f.handle, _dev_ptr(rhs), _dev_ptr(x), M, ld,
                                                  int(n_refine), _arith_code(residual_arith),
                                                  _stream_handle(stream)))
    return x


def sb_solve_batched_groups(factors, rhs, x, arith="native", n_refine=0, residual_arith="native",
                            work=None, Ms=None, lds=None, stream=None):
    """One launch over several shared-LHS groups (lists of equal length), every
    pass of a refined solve included."""
    G = len(factors)
    shapes = [_batch_shape(rhs[g], factors[g].N, None if Ms is None else Ms[g],
                           None if lds is None else lds[g]) for g in range(G)]
    arr = lambda t, vals: (t * G)(*vals)
    fa = arr(ctypes.c_void_p, [f.handle.value for f in factors])
    ra = arr(ctypes.c_void_p, [_dev_ptr(t) for t in rhs])
    xa = arr(ctypes.c_void_p, [_dev_ptr(t) for t in x])
    Ma = arr(ctypes.c_int64, [s[0] for s in shapes])
    la = arr(ctypes.c_int64, [s[1] for s in shapes])
    wa = arr(ctypes.c_void_p, [0 if work is None else _dev_ptr(w) for w in (work or [None] * G)]) \
        if work is not None else None
    wb = arr(ctypes.c_size_t, [_nbytes(w) for w in work]) if work is not None else None
    _check(lib().sb_solve_batched_groups(G, fa, ra, xa, Ma, la, _dtype_code(rhs[0], None),
                                         _dtype_code(x[0], None), _arith_code(arith), int(n_refine),
                                         _arith_code(residual_arith), wa, wb, _stream_handle(stream)))
    return x


STEP_KINDS = {"diffusion": 1, "hyperdiffusion": 2, "cahn_hilliard": 3}
SCHEMES = {"be": 0, "cn": 1}
BCS = {"dirichlet": 0, "hinged": 1, "truncated": 2, "noflux": 3, "periodic": 4}
RUN_MODES = {"graph": 0, "direct": 1, "unfused": 2}


class Stepper:
    """Owns an sb_stepper (implicit time stepper with a shared, factorised matrix)."""

    def __init__(self, kind, scheme, bc, N, coef, dt=0.0):
        h = ctypes.c_void_p()
        _check(lib().sb_stepper_create(STEP_KINDS[kind], SCHEMES[scheme], BCS[bc], int(N),
                                       float(coef), float(dt), ctypes.byref(h)))
        self.handle = h
        self.kind, self.scheme, self.bc, self.N, self.coef, self.dt = kind, scheme, bc, N, coef, dt

    def factor_handle(self):
        return lib().sb_stepper_factor(self.handle)

    def workspace_bytes(self, M, ld=None):
        out = ctypes.c_size_t()
        _check(lib().sb_stepper_workspace_bytes(self.handle, M, M if ld is None else ld, ctypes.byref(out)))
        return out.value

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().sb_stepper_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sb_stepper_create(kind, scheme, bc, N, coef, dt=0.0) -> Stepper:
    return Stepper(kind, scheme, bc, N, coef, dt)


def sb_stepper_run(st: Stepper, state, nsteps, arith="native", mode="graph", work=None, M=None,
                   ld=None, stream=None):
    """Advance `state` ((N, ld) FP64 device tensor) by nsteps steps in place."""
    M, ld = _batch_shape(state, st.N, M, ld)
    wptr = 0 if work is None else _dev_ptr(work)
    wbytes = 0 if work is None else (work.numel() * work.element_size() if not isinstance(work, int)
                                     else st.workspace_bytes(M, ld))
    _check(lib().sb_stepper_run(st.handle, _dev_ptr(state), M, ld, _arith_code(arith), int(nsteps),
                                RUN_MODES[mode] if isinstance(mode, str) else int(mode), wptr or None,
                                wbytes, _stream_handle(stream)))
    return state


def sb_stepper_refined_workspace_bytes(st: Stepper, M, ld=None):
    out = ctypes.c_size_t()
    _check(lib().sb_stepper_refined_workspace_bytes(st.handle, M, M if ld is None else ld, ctypes.byref(out)))
    return out.value


def sb_stepper_run_refined(st: Stepper, state, nsteps, work, n_refine=2, residual_arith="native", mode="graph",
                           M=None, ld=None, stream=None):
    """Advance `state` by nsteps steps whose solves are FP32 sweeps plus n_refine
    refinement passes with an FP64 (or double-float) residual; `work` holds
    sb_stepper_refined_workspace_bytes() bytes on the device."""
    M, ld = _batch_shape(state, st.N, M, ld)
    _check(lib().sb_stepper_run_refined(st.handle, _dev_ptr(state), M, ld, int(n_refine),
                                        _arith_code(residual_arith), int(nsteps),
                                        RUN_MODES[mode] if isinstance(mode, str) else int(mode),
                                        _dev_ptr(work), _nbytes(work), _stream_handle(stream)))
    return state


def sb_stepper_set_forcing(st: Stepper, adv, profile):
    """Make a periodic Cahn-Hilliard stepper the travelling-wave forced scheme:
    adv * W(C) + amp_m * profile_i is added to each step's right-hand side
    (adv = dt v / dx in grid units; profile: N host values, copied)."""
    g = _host_f64(profile, st.N)
    _check(lib().sb_stepper_set_forcing(st.handle, float(adv), g.ctypes.data_as(_dp)))


def sb_stepper_run_forced(st: Stepper, state, amp, nsteps, mode="graph", M=None, ld=None, stream=None):
    """Advance `state` by nsteps forced steps in place; `amp` is a device FP64 tensor of
    M per-system forcing amplitudes."""
    M, ld = _batch_shape(state, st.N, M, ld)
    _check(lib().sb_stepper_run_forced(st.handle, _dev_ptr(state), _dev_ptr(amp), M, ld, int(nsteps),
                                       RUN_MODES[mode] if isinstance(mode, str) else int(mode),
                                       _stream_handle(stream)))
    return state


def sb_stepper_run_coarsening(st: Stepper, state, nsteps, ell, work, arith="native", M=None, ld=None,
                              stream=None):
    """Advance a Cahn-Hilliard `state` by nsteps fused steps and write the mean
    coarsening length 1/(1 - <C^2>) after each step into `ell` (nsteps FP64 values
    on the device); `work` holds M + 256 doubles."""
    M, ld = _batch_shape(state, st.N, M, ld)
    _check(lib().sb_stepper_run_coarsening(st.handle, _dev_ptr(state), M, ld, _arith_code(arith),
                                           int(nsteps), _dev_ptr(ell), _dev_ptr(work), _nbytes(work),
                                           _stream_handle(stream)))
    return ell


def sb_rollout_workspace_bytes(st: Stepper, M, nsteps, ckpt_every, ld=None):
    out = ctypes.c_size_t()
    _check(lib().sb_rollout_workspace_bytes(st.handle, M, M if ld is None else ld, int(nsteps),
                                            int(ckpt_every), ctypes.byref(out)))
    return out.value


def sb_rollout_forward(st: Stepper, C0, CT, nsteps, ckpt_every, work, arith="native", M=None, ld=None,
                       stream=None):
    M, ld = _batch_shape(C0, st.N, M, ld)
    _check(lib().sb_rollout_forward(st.handle, _dev_ptr(C0), _dev_ptr(CT), M, ld, int(nsteps),
                                    int(ckpt_every), _arith_code(arith), _dev_ptr(work), _nbytes(work),
                                    _stream_handle(stream)))
    return CT


def sb_rollout_backward(st: Stepper, grad_CT, grad_C0, nsteps, ckpt_every, work, grad_param=None,
                        grad_param_per_system=None, arith="native", M=None, ld=None, stream=None):
    M, ld = _batch_shape(grad_CT, st.N, M, ld)
    _check(lib().sb_rollout_backward(
        st.handle, _dev_ptr(grad_CT), _dev_ptr(grad_C0),
        None if grad_param_per_system is None else _dev_ptr(grad_param_per_system),
        None if grad_param is None else _dev_ptr(grad_param), M, ld, int(nsteps), int(ckpt_every),
        _arith_code(arith), _dev_ptr(work), _nbytes(work), _stream_handle(stream)))
    return grad_C0


def sb_device_timeouts(device: int = 0) -> int:
    """CTAs of partitioned solves on ``device`` that timed out waiting for a tile
    copy since the previous call (then reset); synchronises the device."""
    out = ctypes.c_uint()
    _check(lib().sb_device_timeouts(int(device), ctypes.byref(out)))
    return out.value


class _Rates(ctypes.Structure):
    _fields_ = [("fp64_fma_per_s", ctypes.c_double), ("fp32_fma_per_s", ctypes.c_double),
                ("f64_f32_conversions_per_s", ctypes.c_double), ("sm_count", ctypes.c_int)]


def sb_measure_rates(device: int = 0) -> dict:
    """Measured FP64 FMA, FP32 FMA and FP64<->FP32 conversion rates of ``device``
    (per second) and its SM count; blocking."""
    out = _Rates()
    _check(lib().sb_measure_rates(int(device), ctypes.byref(out)))
    return {name: getattr(out, name) for name, _ in _Rates._fields_}


def sb_last_error() -> str:
    return lib().sb_last_error().decode()


def sb_version() -> str:
    return lib().sb_version().decode()

"""Python binding of the GB300 hierarchical Jacobi library (libhj.so).

The functions named ``hj_*`` mirror the C ABI in include/hj.h one to one and
only marshal arguments (ctypes structs, raw device pointers, the CUDA stream
handle).  Every step of the solve runs in the library's CUDA kernels; there is
no CPU or PyTorch fallback: if libhj.so is missing or fails to load, importing
the binding's functions raises.

``Solver`` is a thin convenience wrapper that owns one handle and accepts
torch tensors laid out as the ABI requires (``alloc_grid`` makes such
tensors).  PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

_PKG = Path(__file__).resolve().parent
# HJ_LIBRARY=debug selects the debug build (index checks, guard bands; see _build.py)
LIB_PATH = _PKG / ("libhj_debug.so" if os.environ.get("HJ_LIBRARY") == "debug" else "libhj.so")

# status codes (include/hj.h)
HJ_OK = 0
HJ_ERR_INVALID_ARG = 1
HJ_ERR_NOT_DIAG_DOMINANT = 2
HJ_ERR_UNSUPPORTED = 3
HJ_ERR_CUDA = 4
HJ_ERR_NOT_CONVERGED = 5
HJ_ERR_DIVERGED = 6
HJ_ERR_TIMEOUT = 7
HJ_ERR_NO_MEMORY = 8
HJ_ERR_BOUNDS = 9

HJ_F64, HJ_F32 = 0, 1
HJ_PREC_F64, HJ_PREC_F32, HJ_PREC_F32_IR, HJ_PREC_BF16CORR_IR = 0, 1, 2, 3
HJ_METHOD_HIER, HJ_METHOD_CLASSIC, HJ_METHOD_MG = 0, 1, 2

PRECISIONS = {"f64": HJ_PREC_F64, "f32": HJ_PREC_F32, "f32_ir": HJ_PREC_F32_IR, "bf16corr_ir": HJ_PREC_BF16CORR_IR}


class hj_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("ld", C.c_longlong),
                ("cW", C.c_double), ("cE", C.c_double), ("cS", C.c_double), ("cN", C.c_double),
                ("cD", C.c_double), ("sigma_const", C.c_double), ("sigma", C.c_void_p),
                ("dtype", C.c_int), ("coef", C.c_void_p), ("nz", C.c_int), ("cB", C.c_double),
                ("cT", C.c_double)]


class hj_params(C.Structure):
    _fields_ = [("method", C.c_int), ("tile_x", C.c_int), ("tile_y", C.c_int), ("k", C.c_int),
                ("precision", C.c_int), ("check_every", C.c_int), ("max_cycles", C.c_longlong),
                ("tol", C.c_double), ("fixed_cycles", C.c_longlong), ("inner_tol", C.c_double),
                ("inner_max_cycles", C.c_longlong), ("max_outer", C.c_int), ("persistent", C.c_int),
                ("autotune", C.c_int), ("pipeline", C.c_int), ("tile_threads", C.c_int),
                ("pipeline_stages", C.c_int), ("inner_stall", C.c_int), ("ctas_per_sm", C.c_int),
                ("overlap_x", C.c_int), ("overlap_y", C.c_int), ("in_place", C.c_int), ("tile_z", C.c_int),
                ("mg_levels", C.c_int), ("mg_pre", C.c_int), ("mg_post", C.c_int), ("mg_omega", C.c_double),
                ("mg_coarse_k", C.c_int), ("mg_coarse_cycles", C.c_int)]


class hj_stats(C.Structure):
    _fields_ = [("cycles", C.c_longlong), ("cycles_launched", C.c_longlong),
                ("inner_cycles", C.c_longlong), ("outer_steps", C.c_int), ("res0", C.c_double),
                ("res_final", C.c_double), ("rel_final", C.c_double),
                ("history", C.POINTER(C.c_double)), ("history_cap", C.c_longlong),
                ("history_len", C.c_longlong), ("wall_ms", C.c_double), ("tile_x", C.c_int),
                ("tile_y", C.c_int), ("k", C.c_int), ("tile_threads", C.c_int), ("persistent", C.c_int),
                ("pipeline_stages", C.c_int), ("ctas_per_sm", C.c_int), ("overlap_x", C.c_int),
                ("overlap_y", C.c_int), ("tile_z", C.c_int), ("graphed", C.c_int),
                ("cycle_ms", C.POINTER(C.c_double)), ("cycle_points", C.POINTER(C.c_longlong)),
                ("cycle_cap", C.c_longlong), ("cycle_len", C.c_longlong)]


class HJError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        lib = _lib_or_none()
        msg = lib.hj_last_error().decode() if lib else ""
        name = lib.hj_error_string(code).decode() if lib else str(code)
        super().__init__(f"{where}: {name} ({code}): {msg}")


_lib = None


def _lib_or_none():
    return _lib


def lib():
    """Load libhj.so (raises if it is not built: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                               "(the solver has no CPU fallback)")
        L = C.CDLL(str(LIB_PATH))
        H = C.c_void_p
        L.hj_default_params.argtypes = [C.POINTER(hj_params)]
        L.hj_default_params.restype = None
        L.hj_create.argtypes = [C.POINTER(H), C.POINTER(hj_desc), C.POINTER(hj_params)]
        L.hj_solve.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(hj_stats)]
        L.hj_residual.argtypes = [H, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.c_void_p]
        L.hj_solve_adjoint.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(hj_stats)]
        L.hj_solve_batched.argtypes = [H, C.c_int, C.POINTER(hj_desc), C.POINTER(C.c_void_p),
                                       C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(hj_stats),
                                       C.POINTER(C.c_longlong)]
        L.hj_solve_adjoint_batched.argtypes = [H, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                               C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p, C.POINTER(hj_stats)]
        L.hj_destroy.argtypes = [H]
        L.hj_destroy.restype = None
        L.hj_error_string.argtypes = [C.c_int]
        L.hj_error_string.restype = C.c_char_p
        L.hj_last_error.argtypes = []
        L.hj_last_error.restype = C.c_char_p
        L.hj_tile_shapes.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int]
        L.hj_tile_shapes3d.argtypes = [C.c_int, C.POINTER(C.c_int), C.c_int]
        L.hj_tile_variants.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int]
        L.hj_autotune.argtypes = [C.POINTER(hj_desc), C.POINTER(hj_params), C.POINTER(C.c_double)]
        L.hj_cycles_noalloc.argtypes = [C.POINTER(hj_desc), C.POINTER(hj_params), C.c_void_p, C.c_void_p,
                                        C.c_void_p]
        L.hj_debug_check.argtypes = [C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.hj_debug_selftest.argtypes = []
        for name in ("hj_create", "hj_solve", "hj_residual", "hj_solve_adjoint", "hj_solve_batched",
                     "hj_solve_adjoint_batched",
                     "hj_tile_shapes", "hj_tile_variants", "hj_autotune", "hj_cycles_noalloc", "hj_debug_check",
                     "hj_debug_selftest"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# 1:1 wrappers of the C ABI (raw pointers; ints for device addresses/streams)
# ---------------------------------------------------------------------------

def hj_default_params() -> hj_params:
    p = hj_params()
    lib().hj_default_params(C.byref(p))
    return p


def hj_create(desc: hj_desc, params: hj_params):
    h = C.c_void_p()
    st = lib().hj_create(C.byref(h), C.byref(desc), C.byref(params))
    if st != HJ_OK:
        raise HJError(st, "hj_create")
    return h


def hj_solve(h, f_ptr: int, u_ptr: int, stream: int = 0, stats: hj_stats | None = None) -> int:
    return lib().hj_solve(h, C.c_void_p(f_ptr), C.c_void_p(u_ptr), C.c_void_p(stream),
                          C.byref(stats) if stats is not None else None)


def hj_residual(h, f_ptr: int, u_ptr: int, stream: int = 0):
    a, r = C.c_double(), C.c_double()
    st = lib().hj_residual(h, C.c_void_p(f_ptr), C.c_void_p(u_ptr), C.byref(a), C.byref(r),
                           C.c_void_p(stream))
    if st != HJ_OK:
        raise HJError(st, "hj_residual")
    return a.value, r.value


def hj_solve_adjoint(h, g_ptr: int, u_ptr: int, dl_df_ptr: int, dl_dsigma_ptr: int = 0, stream: int = 0,
                     stats: hj_stats | None = None) -> int:
    return lib().hj_solve_adjoint(h, C.c_void_p(g_ptr), C.c_void_p(u_ptr), C.c_void_p(dl_df_ptr),
                                  C.c_void_p(dl_dsigma_ptr or None), C.c_void_p(stream),
                                  C.byref(stats) if stats is not None else None)


def hj_solve_batched(h, descs, f_ptrs, u_ptrs, stream: int = 0, stats: hj_stats | None = None,
                     cycles_out=None) -> int:
    n = len(descs)
    D = (hj_desc * n)(*descs)
    F = (C.c_void_p * n)(*f_ptrs)
    U = (C.c_void_p * n)(*u_ptrs)
    return lib().hj_solve_batched(h, n, D, F, U, C.c_void_p(stream),
                                  C.byref(stats) if stats is not None else None, cycles_out)


def hj_solve_adjoint_batched(h, g_ptrs, u_ptrs, dl_df_ptrs, dl_dsigma_ptr: int = 0, stream: int = 0,
                             stats: hj_stats | None = None) -> int:
    n = len(g_ptrs)
    G = (C.c_void_p * n)(*g_ptrs)
    U = (C.c_void_p * n)(*u_ptrs)
    L = (C.c_void_p * n)(*dl_df_ptrs)
    return lib().hj_solve_adjoint_batched(h, n, G, U, L, C.c_void_p(dl_dsigma_ptr or None), C.c_void_p(stream),
                                          C.byref(stats) if stats is not None else None)


def hj_destroy(h) -> None:
    if h:
        lib().hj_destroy(h)


def hj_error_string(code: int) -> str:
    return lib().hj_error_string(code).decode()


def hj_last_error() -> str:
    return lib().hj_last_error().decode()


def hj_autotune(desc: hj_desc, params: hj_params):
    """Measure and write the best tile_x, tile_y, k into params; returns the
    predicted milliseconds to tolerance (-1 for a cache hit)."""
    ms = C.c_double()
    st = lib().hj_autotune(C.byref(desc), C.byref(params), C.byref(ms))
    if st != HJ_OK:
        raise HJError(st, "hj_autotune")
    return ms.value


def hj_cycles_noalloc(desc: hj_desc, params: hj_params, f_ptr: int, u_ptr: int, stream: int = 0) -> int:
    """params.fixed_cycles cycles on u in place without any allocation (the
    second iterate buffer is a static 16 MiB array in the library)."""
    return lib().hj_cycles_noalloc(C.byref(desc), C.byref(params), C.c_void_p(f_ptr), C.c_void_p(u_ptr),
                                   C.c_void_p(stream))


def hj_debug_check():
    """(status, site, index) of the debug build's memory checks (see hj.h);
    site -1: the library has no checks compiled in."""
    site, index = C.c_longlong(0), C.c_longlong(0)
    code = lib().hj_debug_check(C.byref(site), C.byref(index))
    return code, site.value, index.value


def hj_debug_selftest() -> int:
    return lib().hj_debug_selftest()


def hj_tile_variants(dim: int, precision: int):
    n = lib().hj_tile_variants(dim, precision, None, 0)
    buf = (C.c_int * (3 * n))()
    lib().hj_tile_variants(dim, precision, buf, n)
    return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(n)]


def hj_tile_shapes(dim: int, precision: int):
    n = lib().hj_tile_shapes(dim, precision, None, 0)
    buf = (C.c_int * (2 * n))()
    lib().hj_tile_shapes(dim, precision, buf, n)
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(n)]


def hj_tile_shapes3d(precision: int):
    n = lib().hj_tile_shapes3d(precision, None, 0)
    buf = (C.c_int * (3 * n))()
    lib().hj_tile_shapes3d(precision, buf, n)
    return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(n)]


# ---------------------------------------------------------------------------
# torch-tensor convenience layer (memory and streams only)
# ---------------------------------------------------------------------------

def padded_ld(nx: int, dtype) -> int:
    """Row pitch in elements: nx + 2 rounded up to a multiple of 32 elements."""
    return ((nx + 2 + 31) // 32) * 32


def alloc_grid(dim: int, nx: int, ny: int, dtype, device="cuda", fill: float = 0.0, nz: int = 1):
    """A (rows, ld) device tensor meeting the ABI's alignment rules, or
    (nz + 2, ny + 2, ld) in 3D; use ``t[..., :nx+2]`` as the logical grid."""
    import torch
    if dim == 3:
        return torch.full((nz + 2, ny + 2, padded_ld(nx, dtype)), fill, dtype=dtype, device=device)
    rows = ny + 2 if dim == 2 else ny
    t = torch.full((rows, padded_ld(nx, dtype)), fill, dtype=dtype, device=device)
    return t


def grid_from(a, dim: int, dtype=None, device="cuda"):
    """Copy a logical (rows, nx+2) (3D: (nz+2, ny+2, nx+2)) array (numpy or
    torch) into a padded device grid."""
    import torch
    src = torch.as_tensor(a)
    dtype = dtype or src.dtype
    nx = src.shape[-1] - 2
    if dim == 3:
        t = alloc_grid(3, nx, src.shape[1] - 2, dtype, device, nz=src.shape[0] - 2)
    else:
        ny = src.shape[0] - 2 if dim == 2 else src.shape[0]
        t = alloc_grid(dim, nx, ny, dtype, device)
    t[..., :nx + 2].copy_(src.to(dtype))
    return t


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def make_desc(dim, nx, ny, ld, cW, cE, cS=0.0, cN=0.0, cD=0.0, sigma_const=0.0, sigma=None,
              dtype=HJ_F64, coef=None, nz=1, cB=0.0, cT=0.0) -> hj_desc:
    """coef: optional device tensor (planes, rows, ld) float64 of per-point
    neighbour coefficients W, E[, S, N]; nz, cB, cT: the 3D extension."""
    return hj_desc(dim, nx, ny, ld, cW, cE, cS, cN, cD, sigma_const,
                   None if sigma is None else int(sigma.data_ptr()), dtype,
                   None if coef is None else int(coef.data_ptr()), nz, cB, cT)


def make_params(**kw) -> hj_params:
    p = hj_default_params()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "method" and isinstance(v, str):
            v = {"hier": HJ_METHOD_HIER, "classic": HJ_METHOD_CLASSIC, "mg": HJ_METHOD_MG}[v]
        setattr(p, k, v)
    return p


class Solver:
    """One hj handle for a fixed grid shape, stencil and parameter set.

    stencil: any object with dim, nx, ny, cW, cE, cS, cN, cD, sigma_const
    attributes; sigma: optional (rows, ld) float64 device tensor; coef:
    optional (planes, rows, ld) float64 device tensor of per-point neighbour
    coefficients W, E[, S, N] (both kept alive by the Solver as the ABI
    requires)."""

    def __init__(self, stencil, params: hj_params | None = None, sigma=None, dtype=None, coef=None, **kw):
        import torch
        self.params = params if params is not None else make_params(**kw)
        self.dim, self.nx, self.ny = stencil.dim, stencil.nx, stencil.ny
        self.nz = getattr(stencil, "nz", 1) if self.dim == 3 else 1
        if dtype is None:
            dtype = torch.float32 if self.params.precision == HJ_PREC_F32 else torch.float64
        self.dtype = dtype
        self.ld = padded_ld(self.nx, dtype)
        self.sigma = sigma
        if sigma is not None and sigma.shape[-1] != self.ld:
            raise ValueError("sigma must be a padded grid with the solver's ld")
        self.coef = coef
        if coef is not None and (coef.dim() != 3 or coef.shape[2] != self.ld or coef.dtype != torch.float64
                                 or not coef.is_contiguous()):
            raise ValueError("coef must be a contiguous float64 (planes, rows, ld) tensor with the solver's ld")
        self.desc = make_desc(self.dim, self.nx, self.ny, self.ld, stencil.cW, stencil.cE, stencil.cS,
                              stencil.cN, stencil.cD, getattr(stencil, "sigma_const", 0.0), sigma,
                              HJ_F64 if dtype == torch.float64 else HJ_F32, coef, self.nz,
                              getattr(stencil, "cB", 0.0), getattr(stencil, "cT", 0.0))
        self.h = hj_create(self.desc, self.params)

    def _check(self, t, name):
        if t.dtype != self.dtype or t.shape[-1] != self.ld or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous padded grid of {self.dtype} with ld={self.ld}")
        if self.dim == 3 and tuple(t.shape[:2]) != (self.nz + 2, self.ny + 2):
            raise ValueError(f"{name} must have shape (nz + 2, ny + 2, ld)")

    def grid(self, fill=0.0):
        return alloc_grid(self.dim, self.nx, self.ny, self.dtype, fill=fill, nz=self.nz)

    def solve(self, f, u, stream=None, history: int = 0, check=True):
        """Solve in place (u: initial guess with Dirichlet ghost ring -> solution).
        Returns a dict of the hj_stats fields (plus 'status')."""
        self._check(f, "f")
        self._check(u, "u")
        st = hj_stats()
        hbuf = None
        if history:
            hbuf = (C.c_double * history)()
            st.history = C.cast(hbuf, C.POINTER(C.c_double))
            st.history_cap = history
        code = hj_solve(self.h, f.data_ptr(), u.data_ptr(), _stream_handle(stream), st)
        out = _stats_dict(st, hbuf)
        out["status"] = code
        if check and code not in (HJ_OK, HJ_ERR_NOT_CONVERGED):
            raise HJError(code, "hj_solve")
        return out

    def residual(self, f, u, stream=None):
        return hj_residual(self.h, f.data_ptr(), u.data_ptr(), _stream_handle(stream))

    def adjoint(self, g, u, dl_df, dl_dsigma=None, stream=None, check=True):
        st = hj_stats()
        code = hj_solve_adjoint(self.h, g.data_ptr(), u.data_ptr(), dl_df.data_ptr(),
                                0 if dl_dsigma is None else dl_dsigma.data_ptr(), _stream_handle(stream), st)
        out = _stats_dict(st, None)
        out["status"] = code
        if check and code not in (HJ_OK, HJ_ERR_NOT_CONVERGED):
            raise HJError(code, "hj_solve_adjoint")
        return out

    def close(self):
        if getattr(self, "h", None):
            hj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(stencil, f, u, sigma=None, coef=None, stream=None, history: int = 0, **params):
    """One call: create a handle for this stencil and parameters, solve A u = f
    in place (u: initial guess with the Dirichlet ghost ring -> solution),
    destroy the handle, return the hj_stats fields as a dict (plus 'status').
    f and u are padded device grids (``grid_from``); sigma / coef as for
    ``Solver``.  For repeated solves keep a ``Solver``: creation validates the
    problem, allocates the workspace and captures graphs once."""
    dtype = f.dtype
    s = Solver(stencil, sigma=sigma, coef=coef, dtype=dtype, **params)
    try:
        return s.solve(f, u, stream=stream, history=history)
    finally:
        s.close()


def _stats_dict(st: hj_stats, hbuf):
    d = {k: getattr(st, k) for k, _ in hj_stats._fields_ if k not in ("history", "cycle_ms", "cycle_points")}
    if hbuf is not None:
        d["history"] = [hbuf[i] for i in range(st.history_len)]
    return d

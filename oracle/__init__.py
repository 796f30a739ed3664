"""CPU oracle for hierarchical Jacobi (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path
(``paper_2006_16465_gb300``) never imports it, and it never imports the
product path: the two share no code.

Everything is computed by ``hj_oracle.c`` (plain C, binary64, no fused
multiply-add); this module only marshals numpy arrays through ctypes.
Grid arrays are C-contiguous float64 numpy arrays of shape (rows, nx + 2)
with the Dirichlet ghost ring (see ``workloads``).

Parity status: every function is pinned by the not-gpu tests in
``tests/test_oracle_pins.py`` (closed-form Jacobi decay, Thomas vs banded LU,
DST and dense direct solves, per-subdomain direct solves, k = 1 equivalence,
central finite differences for the adjoint).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRCS = [_HERE / "hj_oracle.c", _HERE / "hj_oracle3d.c", _HERE / "hj_oracle_mg.c"]
_LIB = _HERE / "libhj_oracle.so"


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math),
    with OpenMP where the compiler has it (the subdomain loop of a cycle and
    the row loop of a classic sweep; results do not depend on the thread
    count, which stays 1 unless set_threads asks for more)."""
    newest = max(s.stat().st_mtime for s in _SRCS + [Path(__file__)])
    if force or not _LIB.exists() or _LIB.stat().st_mtime < newest:
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
        srcs = [str(s) for s in _SRCS]
        out = ["-o", str(_LIB) + ".tmp", "-lm"]
        r = subprocess.run(base + ["-fopenmp"] + srcs + out, capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(base + srcs + out, check=True)
        os.replace(str(_LIB) + ".tmp", _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("cW", C.c_double), ("cE", C.c_double), ("cS", C.c_double),
                ("cN", C.c_double), ("cD", C.c_double), ("sigma_const", C.c_double),
                ("sigma", C.c_void_p), ("coef", C.c_void_p)]


class _Problem3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("cW", C.c_double), ("cE", C.c_double), ("cS", C.c_double), ("cN", C.c_double),
                ("cB", C.c_double), ("cT", C.c_double), ("cD", C.c_double),
                ("sigma_const", C.c_double), ("sigma", C.c_void_p)]


class _MgProblem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("cW", C.c_double), ("cE", C.c_double),
                ("cS", C.c_double), ("cN", C.c_double), ("cD", C.c_double), ("sigma_const", C.c_double)]


_lib = None
_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(str(build()))
        P = C.POINTER(_Problem)
        L.hjo_apply.argtypes = [P, _D, _D]
        L.hjo_residual_sq.argtypes = [P, _D, _D]
        L.hjo_residual_sq.restype = C.c_double
        L.hjo_jacobi_sweep.argtypes = [P, _D, _D, _D]
        L.hjo_hier_cycle.argtypes = [P, _D, _D, _D, C.c_int, C.c_int, C.c_int]
        L.hjo_solve.argtypes = [P, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                C.c_long, _D, C.c_long, C.POINTER(C.c_int)]
        L.hjo_solve.restype = C.c_long
        L.hjo_run_fixed.argtypes = [P, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_long]
        L.hjo_thomas.argtypes = [C.c_long, _D, _D, _D, _D, _D]
        L.hjo_bf16_round.argtypes = [C.c_float]
        L.hjo_bf16_round.restype = C.c_float
        L.hjo_hier_cycle_f32.argtypes = [P, _F, _F, _F, C.c_int, C.c_int, C.c_int, C.c_int]
        L.hjo_residual_sq_f32.argtypes = [P, _F, _F]
        L.hjo_residual_sq_f32.restype = C.c_double
        L.hjo_ir_solve.argtypes = [P, _D, _D, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                   C.c_long, C.c_long, C.c_int, C.c_long, C.c_double, _D, C.c_long,
                                   C.POINTER(C.c_long), C.POINTER(C.c_int)]
        L.hjo_ir_solve.restype = C.c_long
        L.hjo_adjoint.argtypes = [P, _D, _D, _D, _D, C.c_int, C.c_int, C.c_int, C.c_double,
                                  C.c_long, C.POINTER(C.c_int)]
        L.hjo_adjoint.restype = C.c_long
        L.hjo_hier_cycle_ovl.argtypes = [P, _D, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.hjo_solve_ovl.argtypes = [P, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_double, C.c_long, _D, C.c_long, C.POINTER(C.c_int)]
        L.hjo_solve_ovl.restype = C.c_long
        L.hjo_run_fixed_ovl.argtypes = [P, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_long]
        P3 = C.POINTER(_Problem3)
        L.hjo3_apply.argtypes = [P3, _D, _D]
        L.hjo3_residual_sq.argtypes = [P3, _D, _D]
        L.hjo3_residual_sq.restype = C.c_double
        L.hjo3_jacobi_sweep.argtypes = [P3, _D, _D, _D]
        L.hjo3_hier_cycle.argtypes = [P3, _D, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int]
        L.hjo3_solve.argtypes = [P3, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                 C.c_long, _D, C.c_long, C.POINTER(C.c_int)]
        L.hjo3_solve.restype = C.c_long
        L.hjo3_run_fixed.argtypes = [P3, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_long]
        PM = C.POINTER(_MgProblem)
        L.hjo_mg_wcycle.argtypes = [PM, _D, _D, _D, C.c_int, C.c_int, C.c_int, C.c_double]
        L.hjo_mg_restrict.argtypes = [PM, _D, _D, _D]
        L.hjo_mg_prolong_add.argtypes = [PM, _D, _D]
        L.hjo_mg_max_levels.argtypes = [C.c_int, C.c_int]
        L.hjo_mg_max_levels.restype = C.c_int
        L.hjo_mg_vcycle.argtypes = [PM, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_double, C.c_int, C.c_int]
        L.hjo_mg_solve.argtypes = [PM, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_double, C.c_int, C.c_int, C.c_double, C.c_long, _D, C.c_long,
                                   C.POINTER(C.c_int)]
        L.hjo_mg_solve.restype = C.c_long
        L.hjo_paper_smem_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
        L.hjo_paper_smem_bytes.restype = C.c_long
        L.hjo_set_threads.argtypes = [C.c_int]
        L.hjo_set_threads.restype = C.c_int
        L.hjo_set_threads(1)
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Threads for the subdomain loop of a cycle and the row loop of a classic
    sweep (OpenMP build; results are bitwise the same for every count).
    Returns the count in effect (1 without OpenMP)."""
    return int(lib().hjo_set_threads(int(n)))


def _grid(a, dtype=np.float64) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _dp(a):
    return a.ctypes.data_as(_D)


def _fp(a):
    return a.ctypes.data_as(_F)


class Problem:
    """Oracle-side view of a stencil problem (duck-typed from workloads.Stencil)."""

    def __init__(self, st):
        self.st = st
        self.sigma = None if st.sigma is None else _grid(st.sigma)
        if st.dim == 3:
            if getattr(st, "coef", None) is not None:
                raise ValueError("the 3D oracle takes constant neighbour coefficients")
            self.c = _Problem3(st.nx, st.ny, st.nz, st.cW, st.cE, st.cS, st.cN, st.cB, st.cT, st.cD,
                               float(st.sigma_const), None if self.sigma is None else self.sigma.ctypes.data)
            self.shape = (st.nz + 2, st.ny + 2, st.nx + 2)
            return
        coef = getattr(st, "coef", None)
        self.coef = None if coef is None else _grid(coef)   # planes W, E[, S, N] x rows x (nx + 2)
        self.c = _Problem(st.dim, st.nx, st.ny, st.cW, st.cE, st.cS, st.cN, st.cD,
                          float(st.sigma_const),
                          None if self.sigma is None else self.sigma.ctypes.data,
                          None if self.coef is None else self.coef.ctypes.data)
        self.shape = (st.rows, st.nx + 2)

    @property
    def ref(self):
        return C.byref(self.c)


def _prob(st) -> Problem:
    return st if isinstance(st, Problem) else Problem(st)


def _is3(p) -> bool:
    return p.st.dim == 3


def apply(st, u):
    p = _prob(st)
    u = _grid(u)
    out = np.zeros(p.shape)
    (lib().hjo3_apply if _is3(p) else lib().hjo_apply)(p.ref, _dp(u), _dp(out))
    return out


def residual(st, f, u) -> float:
    """||f - A u||_2 over interior points (binary64, x-fastest summation)."""
    p = _prob(st)
    fn = lib().hjo3_residual_sq if _is3(p) else lib().hjo_residual_sq
    return float(np.sqrt(fn(p.ref, _dp(_grid(f)), _dp(_grid(u)))))


def jacobi_sweep(st, f, u):
    p = _prob(st)
    out = np.zeros(p.shape)
    fn = lib().hjo3_jacobi_sweep if _is3(p) else lib().hjo_jacobi_sweep
    fn(p.ref, _dp(_grid(f)), _dp(_grid(u)), _dp(out))
    return out


def hier_cycle(st, f, u, tx, ty, k, tz=1):
    """One hierarchical cycle on tx (x ty (x tz)) subdomains."""
    p = _prob(st)
    out = np.zeros(p.shape)
    if _is3(p):
        lib().hjo3_hier_cycle(p.ref, _dp(_grid(f)), _dp(_grid(u)), _dp(out), tx, ty, tz, k)
    else:
        lib().hjo_hier_cycle(p.ref, _dp(_grid(f)), _dp(_grid(u)), _dp(out), tx, ty, k)
    return out


def hier_cycle_ovl(st, f, u, tx, ty, k, ox, oy=0):
    """One cycle with overlapping subdomains (ox, oy shared points between
    neighbours; Sections 3.4, 4.3)."""
    p = _prob(st)
    out = np.zeros(p.shape)
    lib().hjo_hier_cycle_ovl(p.ref, _dp(_grid(f)), _dp(_grid(u)), _dp(out), tx, ty, k, int(ox), int(oy))
    return out


def run_fixed(st, f, u0, ncycles, tx=32, ty=32, k=1, classic=False, overlap=(0, 0), tz=1):
    """u after exactly ncycles hierarchical cycles (or classic sweeps);
    overlap = (ox, oy) points shared by neighbouring subdomains; tz: the
    subdomain depth of 3D problems."""
    p = _prob(st)
    u = _grid(u0).copy()
    if _is3(p):
        lib().hjo3_run_fixed(p.ref, _dp(_grid(f)), _dp(u), int(classic), tx, ty, tz, k, int(ncycles))
    elif overlap != (0, 0) and not classic:
        lib().hjo_run_fixed_ovl(p.ref, _dp(_grid(f)), _dp(u), tx, ty, k, int(overlap[0]), int(overlap[1]),
                                int(ncycles))
    else:
        lib().hjo_run_fixed(p.ref, _dp(_grid(f)), _dp(u), int(classic), tx, ty, k, int(ncycles))
    return u


def solve(st, f, u0, tol, max_cycles, tx=32, ty=32, k=1, classic=False, hist_cap=0, overlap=(0, 0), tz=1):
    """Returns (u_c, c, status, hist): c = first cycle with ||r_c|| <= tol ||r_0||."""
    p = _prob(st)
    u = _grid(u0).copy()
    hist = np.zeros(max(hist_cap, 1))
    status = C.c_int(0)
    if _is3(p):
        c = lib().hjo3_solve(p.ref, _dp(_grid(f)), _dp(u), int(classic), tx, ty, tz, k, float(tol),
                             int(max_cycles), _dp(hist), int(hist_cap), C.byref(status))
    elif overlap != (0, 0) and not classic:
        c = lib().hjo_solve_ovl(p.ref, _dp(_grid(f)), _dp(u), int(classic), tx, ty, k, int(overlap[0]),
                                int(overlap[1]), float(tol), int(max_cycles), _dp(hist), int(hist_cap),
                                C.byref(status))
    else:
        c = lib().hjo_solve(p.ref, _dp(_grid(f)), _dp(u), int(classic), tx, ty, k, float(tol),
                            int(max_cycles), _dp(hist), int(hist_cap), C.byref(status))
    return u, int(c), int(status.value), hist[:min(hist_cap, c + 1)]


def thomas(a, d, c, b):
    n = len(d)
    x = np.zeros(n)
    lib().hjo_thomas(n, _dp(_grid(a)), _dp(_grid(d)), _dp(_grid(c)), _dp(_grid(b)), _dp(x))
    return x


def bf16_round(x: float) -> float:
    return float(lib().hjo_bf16_round(float(x)))


def hier_cycle_f32(st, rhs, d, tx, ty, k, bf16=False):
    p = _prob(st)
    out = np.zeros(p.shape, dtype=np.float32)
    lib().hjo_hier_cycle_f32(p.ref, _fp(_grid(rhs, np.float32)), _fp(_grid(d, np.float32)),
                             _fp(out), tx, ty, k, int(bf16))
    return out


def residual_f32(st, rhs, d) -> float:
    p = _prob(st)
    return float(np.sqrt(lib().hjo_residual_sq_f32(p.ref, _fp(_grid(rhs, np.float32)),
                                                    _fp(_grid(d, np.float32)))))


def ir_solve(st, f, u0, tol, tx=32, ty=32, k=16, inner_tol=1e-4, inner_max=100000,
             max_outer=50, bf16=False, stall_window=32, stall_rtol=1e-3):
    """Iterative refinement (binary64 residual/update, binary32 inner cycles,
    inner stop on inner_tol, stagnation or inner_max).
    Returns (u, outer_steps, inner_cycles, status, hist)."""
    p = _prob(st)
    u = _grid(u0).copy()
    hist = np.zeros(max_outer + 1)
    tot = C.c_long(0)
    status = C.c_int(0)
    o = lib().hjo_ir_solve(p.ref, _dp(_grid(f)), _dp(u), tx, ty, k, float(tol), float(inner_tol),
                           int(inner_max), int(max_outer), int(bf16), int(stall_window), float(stall_rtol),
                           _dp(hist), max_outer + 1,
                           C.byref(tot), C.byref(status))
    return u, int(o), int(tot.value), int(status.value), hist[:o + 1]


def adjoint(st, g, u, tol=1e-13, max_cycles=10_000_000, tx=32, ty=32, k=16):
    """(lambda, dL/dsigma) for dL/du = g: A^T lambda = g, dL/dsigma = -lambda*u."""
    p = _prob(st)
    lam = np.zeros(p.shape)
    dsig = np.zeros(p.shape)
    status = C.c_int(0)
    lib().hjo_adjoint(p.ref, _dp(_grid(g)), _dp(_grid(u)), _dp(lam), _dp(dsig), tx, ty, k,
                      float(tol), int(max_cycles), C.byref(status))
    return lam, dsig, int(status.value)


def paper_smem_bytes(dim, tx, ty, esize) -> int:
    return int(lib().hjo_paper_smem_bytes(dim, tx, ty, esize))


# ---------------------------------------------------------------------------
# hierarchical Jacobi as a multigrid smoother (hj_oracle_mg.c): 2D, constant
# coefficients and sigma_const
# ---------------------------------------------------------------------------

def _mgp(st) -> _MgProblem:
    if st.dim != 2 or st.sigma is not None or getattr(st, "coef", None) is not None:
        raise ValueError("the multigrid oracle takes 2D constant-coefficient problems (sigma_const only)")
    return _MgProblem(st.nx, st.ny, st.cW, st.cE, st.cS, st.cN, st.cD, float(st.sigma_const))


def mg_coarse_stencil(st):
    """The rediscretised operator one level down: every h^-2 term / 4."""
    import dataclasses
    return dataclasses.replace(st, nx=(st.nx - 1) // 2, ny=(st.ny - 1) // 2, cW=st.cW / 4, cE=st.cE / 4,
                               cS=st.cS / 4, cN=st.cN / 4, cD=st.cD / 4)


def mg_wcycle(st, f, u, tx, ty, k, omega):
    """One weighted hierarchical cycle (damped Jacobi subiterations)."""
    p = _mgp(st)
    out = np.zeros((st.ny + 2, st.nx + 2))
    lib().hjo_mg_wcycle(C.byref(p), _dp(_grid(f)), _dp(_grid(u)), _dp(out), tx, ty, k, float(omega))
    return out


def mg_restrict(st, f, u):
    """Full weighting of f - A u onto the next coarser grid."""
    p = _mgp(st)
    fc = np.zeros(((st.ny - 1) // 2 + 2, (st.nx - 1) // 2 + 2))
    lib().hjo_mg_restrict(C.byref(p), _dp(_grid(f)), _dp(_grid(u)), _dp(fc))
    return fc


def mg_prolong_add(st, e, u):
    """u + bilinear interpolation of the coarse correction e."""
    p = _mgp(st)
    out = _grid(u).copy()
    lib().hjo_mg_prolong_add(C.byref(p), _dp(_grid(e)), _dp(out))
    return out


def mg_max_levels(nx, ny) -> int:
    return int(lib().hjo_mg_max_levels(nx, ny))


def mg_vcycle(st, f, u, levels, pre=1, post=1, tx=32, ty=32, k=4, omega=0.8, coarse_k=64, coarse_cycles=4):
    p = _mgp(st)
    out = _grid(u).copy()
    lib().hjo_mg_vcycle(C.byref(p), _dp(_grid(f)), _dp(out), int(levels), int(pre), int(post), tx, ty, k,
                        float(omega), int(coarse_k), int(coarse_cycles))
    return out


def mg_solve(st, f, u0, tol, max_vcycles, levels, pre=1, post=1, tx=32, ty=32, k=4, omega=0.8, coarse_k=64,
             coarse_cycles=4, hist_cap=0):
    """V-cycles to ||r_c|| <= tol ||r_0||.  Returns (u, c, status, hist)."""
    p = _mgp(st)
    u = _grid(u0).copy()
    hist = np.zeros(max(hist_cap, 1))
    status = C.c_int(0)
    c = lib().hjo_mg_solve(C.byref(p), _dp(_grid(f)), _dp(u), int(levels), int(pre), int(post), tx, ty, k,
                           float(omega), int(coarse_k), int(coarse_cycles), float(tol), int(max_vcycles),
                           _dp(hist), int(hist_cap), C.byref(status))
    return u, int(c), int(status.value), hist[:min(hist_cap, c + 1)]

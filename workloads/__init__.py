"""Seeded synthetic inputs for hierarchical Jacobi (shared by the oracle tests,
the GPU tests and the bench).

This module only *generates problem data*: right-hand sides, initial guesses,
boundary values, screening fields and stencil coefficients of the model PDEs.
It contains none of the solver's arithmetic (no sweep, cycle, residual or
refinement step), so both the CPU oracle and the CUDA path can take their
inputs from here without sharing solver code.

Layout convention (used by every consumer): a grid array is a numpy array of
shape ``(rows, nx + 2)`` holding the interior plus a one-cell ghost ring of
Dirichlet values.

* 2D: ``rows = ny + 2``; interior is ``[1:ny+1, 1:nx+1]``; x (column index i)
  is the fastest axis, matching the row-wise warp layout of Section 4.1.
* 1D: ``rows = copies``; every row is an independent 1D problem with ghosts at
  columns 0 and nx+1 (the 1024 simultaneous copies of Section 3.5 are rows).

Random numbers come from one documented counter-based generator, splitmix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): output i of stream ``seed`` is the splitmix64 finaliser applied
to ``seed + (i + 1) * 0x9E3779B97F4A7C15`` (mod 2^64).  Uniforms use the top
53 bits; normals use the Box-Muller transform on consecutive uniform pairs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the splitmix64 stream ``seed`` (uint64)."""
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """U[0,1) doubles from the top 53 bits of splitmix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, n: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, n, offset)


def normal(seed: int, n: int, mean: float = 0.0, std: float = 1.0) -> np.ndarray:
    """N(mean, std^2) by Box-Muller on uniform pairs (u1 in (0,1], u2 in [0,1))."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)])
    out = np.empty(2 * m)
    out[0::2] = z[:m]
    out[1::2] = z[m:]
    return mean + std * out[:n]


# ---------------------------------------------------------------------------
# Problem description (stencil coefficients of the discretised PDE)
# ---------------------------------------------------------------------------

@dataclass
class Stencil:
    """Constant-coefficient 3-/5-point operator
    (A u)_p = cD u_p + sigma_p u_p + cW u_W + cE u_E + cS u_S + cN u_N.

    Names follow the paper's stencils: cW, cE, cS, cN, cD are a, c, e, f, d of
    the 2D pentadiagonal stencil (Section 4, Eq. 2d-jacobi-stencil) and a, c, d
    of the tridiagonal one (Section 3, Eq. jacobi-stencil-equation-1d)."""
    dim: int
    nx: int
    ny: int
    cW: float
    cE: float
    cS: float = 0.0
    cN: float = 0.0
    cD: float = 0.0
    sigma: np.ndarray | None = None   # grid-shaped array (ghost entries ignored) or None
    sigma_const: float = 0.0          # constant screening added to the diagonal
    # per-point neighbour coefficients (planes W, E in 1D; W, E, S, N in 2D,
    # each grid-shaped) replacing cW..cN: the general tridiagonal a_i, c_i of
    # Section 3 and its 2D analogue; None = constant coefficients
    coef: np.ndarray | None = None
    # 3D seven-point extension (dim = 3): nz interior planes, bottom (z - 1)
    # and top (z + 1) neighbour coefficients
    nz: int = 1
    cB: float = 0.0
    cT: float = 0.0

    @property
    def rows(self) -> int:
        return self.ny + 2 if self.dim >= 2 else self.ny

    @property
    def shape(self) -> tuple:
        """Shape of a grid array: (rows, nx + 2), or (nz + 2, ny + 2, nx + 2) in 3D."""
        if self.dim == 3:
            return (self.nz + 2, self.ny + 2, self.nx + 2)
        return (self.rows, self.nx + 2)


def poisson_stencil(dim: int, nx: int, ny: int = 1, sigma=None, sigma_const: float = 0.0) -> Stencil:
    """Second-order central differences of -u'' (1D) or -Lap u (2D) on the unit
    interval / square with ghost-ring Dirichlet data; hx = 1/(nx+1), hy = 1/(ny+1)
    (Eq. poisson and Eq. 2d-poisson; the 2D diagonal is 2/hx^2 + 2/hy^2)."""
    hx = 1.0 / (nx + 1)
    if dim == 1:
        ix2 = 1.0 / (hx * hx)
        return Stencil(1, nx, ny, -ix2, -ix2, 0.0, 0.0, 2.0 * ix2, sigma, sigma_const)
    hy = 1.0 / (ny + 1)
    ix2 = 1.0 / (hx * hx)
    iy2 = 1.0 / (hy * hy)
    return Stencil(2, nx, ny, -ix2, -ix2, -iy2, -iy2, 2.0 * ix2 + 2.0 * iy2, sigma, sigma_const)


def poisson_stencil3d(nx: int, ny: int, nz: int, sigma=None, sigma_const: float = 0.0) -> Stencil:
    """Seven-point -Lap u on the unit cube (h = 1/(n+1) per axis), the 2D
    stencil of Eq. 2d-poisson extended by the z pair; diagonal 2/hx^2 +
    2/hy^2 + 2/hz^2."""
    ix2, iy2, iz2 = (nx + 1.0) ** 2, (ny + 1.0) ** 2, (nz + 1.0) ** 2
    return Stencil(3, nx, ny, -ix2, -ix2, -iy2, -iy2, 2.0 * (ix2 + iy2 + iz2), sigma, sigma_const,
                   None, nz, -iz2, -iz2)


def zeros_grid(st: Stencil, dtype=np.float64) -> np.ndarray:
    return np.zeros(st.shape, dtype=dtype)


def interior(a: np.ndarray, dim: int) -> np.ndarray:
    if dim == 3:
        return a[1:-1, 1:-1, 1:-1]
    return a[1:-1, 1:-1] if dim == 2 else a[:, 1:-1]


# ---------------------------------------------------------------------------
# Workloads (the configurations the solver is measured on)
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    st: Stencil
    f: np.ndarray           # RHS, grid-shaped (ghost entries zero)
    u0: np.ndarray          # initial guess incl. Dirichlet ghost ring
    meta: dict = field(default_factory=dict)


def poisson1d_sine(N: int = 512, nmodes: int = 8, seed: int = 0) -> Problem:
    """1D -u''=f on (0,1), u(0)=u(1)=0, f_i = sum_{m<=8} a_m sin(m pi x_i),
    x_i = i h, h = 1/(N+1), a_m ~ N(0,1) (seeded), u0 = 0."""
    st = poisson_stencil(1, N, 1)
    a = normal(seed, nmodes)
    x = np.arange(N + 2) / (N + 1.0)
    f = zeros_grid(st)
    for m in range(1, nmodes + 1):
        f[0, :] += a[m - 1] * np.sin(m * np.pi * x)
    f[0, 0] = f[0, -1] = 0.0
    return Problem(st, f, zeros_grid(st), {"a": a, "seed": seed})


def poisson2d_uniform(nx: int = 512, ny: int | None = None, seed: int = 1) -> Problem:
    """2D -Lap u = f on the unit square, zero Dirichlet, f ~ U[-1,1] (seeded), u0 = 0."""
    ny = nx if ny is None else ny
    st = poisson_stencil(2, nx, ny)
    f = zeros_grid(st)
    f[1:-1, 1:-1] = uniform(seed, nx * ny, -1.0, 1.0).reshape(ny, nx)
    return Problem(st, f, zeros_grid(st), {"seed": seed})


def poisson2d_sin_noise(n: int = 512, seed: int = 2) -> Problem:
    """2D Poisson, f = sin(pi x) sin(pi y) + 1e-3 U[-1,1] noise, zero Dirichlet, u0 = 0."""
    st = poisson_stencil(2, n, n)
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    f = zeros_grid(st)
    f[1:-1, 1:-1] = np.outer(np.sin(np.pi * x), np.sin(np.pi * x)) \
        + 1e-3 * uniform(seed, n * n, -1.0, 1.0).reshape(n, n)
    return Problem(st, f, zeros_grid(st), {"seed": seed})


def paper_replica(dim: int, N: int = 1024, copies: int = 1) -> Problem:
    """The paper's timing problems (Sections 3.5 and 4.2): b = 1, initial
    solution 1 at interior points, zero Dirichlet data; residual to drop 1e-4."""
    st = poisson_stencil(dim, N, N if dim == 2 else copies)
    f = zeros_grid(st)
    u0 = zeros_grid(st)
    interior(f, dim)[...] = 1.0
    interior(u0, dim)[...] = 1.0
    return Problem(st, f, u0, {"tol": 1e-4})


def random_bc_problem(dim: int, nx: int, ny: int, seed: int, sigma_kind: str = "none",
                      asym: bool = False) -> Problem:
    """Small general test problem: random RHS, random Dirichlet ghost ring,
    random initial guess, optional per-point or constant screening and an
    optional non-symmetric (but diagonally dominant) stencil."""
    st = poisson_stencil(dim, nx, ny)
    rows = st.rows
    if asym:
        # convection-like perturbation: cW != cE, cS != cN, still diagonally dominant
        st.cW *= 1.3
        st.cE *= 0.7
        if dim == 2:
            st.cS *= 0.8
            st.cN *= 1.2
    if sigma_kind == "field":
        st.sigma = np.zeros((rows, nx + 2))
        interior(st.sigma, dim)[...] = uniform(seed + 101, nx * (ny), 0.0, 50.0).reshape(interior(st.sigma, dim).shape)
    elif sigma_kind == "const":
        st.sigma_const = 37.5
    f = zeros_grid(st)
    interior(f, dim)[...] = uniform(seed, interior(f, dim).size, -1.0, 1.0).reshape(interior(f, dim).shape)
    u0 = uniform(seed + 7, rows * (nx + 2), -0.5, 0.5).reshape(rows, nx + 2)
    return Problem(st, f, u0, {"seed": seed})


def variable_coef_problem(dim: int, nx: int, ny: int, seed: int, contrast: float = 10.0,
                          screening: float = 0.0) -> Problem:
    """Heterogeneous diffusion -div(kappa grad u) + s u = f on the unit square
    (or interval) with the 5-point (3-point) flux form: kappa is a smooth
    positive field with max/min about `contrast`, face values are arithmetic
    means of the two cell values, cW = -kappa_{i-1/2}/h^2 etc., and the
    diagonal (sum of the neighbour magnitudes, plus s) goes in sigma with
    cD = 0.  Random RHS, random Dirichlet ring and initial guess."""
    rows = ny + 2 if dim == 2 else ny
    hx = 1.0 / (nx + 1)
    hy = 1.0 / (ny + 1) if dim == 2 else 1.0
    x = np.arange(nx + 2) * hx
    y = (np.arange(rows) * hy) if dim == 2 else np.zeros(rows)
    ph = uniform(seed + 31, 4, 0.0, 2 * np.pi)
    g = np.sin(2 * np.pi * x[None, :] + ph[0]) * np.cos(2 * np.pi * y[:, None] + ph[1]) + \
        0.5 * np.sin(6 * np.pi * x[None, :] + ph[2])
    kappa = np.exp(np.log(contrast) * 0.5 * (g / 1.5 + 1.0))   # in [1, contrast]
    planes = 4 if dim == 2 else 2
    coef = np.zeros((planes, rows, nx + 2))
    kW = 0.5 * (kappa[:, 1:-1] + kappa[:, :-2])
    kE = 0.5 * (kappa[:, 1:-1] + kappa[:, 2:])
    coef[0][:, 1:-1] = -kW / hx ** 2
    coef[1][:, 1:-1] = -kE / hx ** 2
    if dim == 2:
        kS = 0.5 * (kappa[1:-1, :] + kappa[:-2, :])
        kN = 0.5 * (kappa[1:-1, :] + kappa[2:, :])
        coef[2][1:-1, :] = -kS / hy ** 2
        coef[3][1:-1, :] = -kN / hy ** 2
    sigma = np.abs(coef).sum(axis=0) + screening
    st = Stencil(dim, nx, ny, cW=-1.0 / hx ** 2, cE=-1.0 / hx ** 2,
                 cS=(-1.0 / hy ** 2) if dim == 2 else 0.0, cN=(-1.0 / hy ** 2) if dim == 2 else 0.0,
                 cD=0.0, sigma=sigma, coef=coef)
    f = zeros_grid(st)
    interior(f, dim)[...] = uniform(seed, interior(f, dim).size, -1.0, 1.0).reshape(interior(f, dim).shape)
    u0 = uniform(seed + 7, rows * (nx + 2), -0.5, 0.5).reshape(rows, nx + 2)
    return Problem(st, f, u0, {"seed": seed, "contrast": contrast})


def poisson3d_uniform(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 1,
                      sigma_const: float = 0.0) -> Problem:
    """3D -Lap u + s u = f on the unit cube, zero Dirichlet, f ~ U[-1,1], u0 = 0."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    st = poisson_stencil3d(nx, ny, nz, sigma_const=sigma_const)
    f = zeros_grid(st)
    f[1:-1, 1:-1, 1:-1] = uniform(seed, nx * ny * nz, -1.0, 1.0).reshape(nz, ny, nx)
    return Problem(st, f, zeros_grid(st), {"seed": seed})


def random_bc_problem3d(nx: int, ny: int, nz: int, seed: int, sigma_kind: str = "none",
                        asym: bool = False) -> Problem:
    """Small general 3D test problem: random RHS, random Dirichlet shell and
    initial guess, optional constant or per-point screening and an optional
    non-symmetric (diagonally dominant) stencil."""
    st = poisson_stencil3d(nx, ny, nz)
    if asym:
        st.cW *= 1.3
        st.cE *= 0.7
        st.cS *= 0.8
        st.cN *= 1.2
        st.cB *= 1.1
        st.cT *= 0.9
    if sigma_kind == "field":
        st.sigma = zeros_grid(st)
        st.sigma[1:-1, 1:-1, 1:-1] = uniform(seed + 101, nx * ny * nz, 0.0, 50.0).reshape(nz, ny, nx)
    elif sigma_kind == "const":
        st.sigma_const = 37.5
    f = zeros_grid(st)
    f[1:-1, 1:-1, 1:-1] = uniform(seed, nx * ny * nz, -1.0, 1.0).reshape(nz, ny, nx)
    size = int(np.prod(st.shape))
    u0 = uniform(seed + 7, size, -0.5, 0.5).reshape(st.shape)
    return Problem(st, f, u0, {"seed": seed})


BATCH_SIDES = tuple(range(64, 513, 32))   # {64, 96, ..., 512}: 15 values


def batched_screened(nprob: int = 256, seed: int = 3) -> list[Problem]:
    """256 independent 2D screened-Poisson problems -Lap u + sigma u = f with
    nx, ny drawn independently and uniformly from {64, 96, ..., 512}, one
    constant sigma ~ U[0,100] per problem, f ~ U[-1,1], zero Dirichlet, u0 = 0."""
    sides = np.array(BATCH_SIDES)
    pick = (uniform01(seed, 2 * nprob) * len(sides)).astype(np.int64)
    sig = uniform(seed + 1, nprob, 0.0, 100.0)
    out = []
    for p in range(nprob):
        nx, ny = int(sides[pick[2 * p]]), int(sides[pick[2 * p + 1]])
        st = poisson_stencil(2, nx, ny, sigma_const=float(sig[p]))
        f = zeros_grid(st)
        f[1:-1, 1:-1] = uniform(seed * 1000 + 17 + p, nx * ny, -1.0, 1.0).reshape(ny, nx)
        out.append(Problem(st, f, zeros_grid(st), {"index": p}))
    return out


def fourier_sigma(n: int, seed: int = 5, nmodes: int = 16, kmax: float = 8.0) -> np.ndarray:
    """sigma(x,y) = clip(10 exp(g), 10, 1000), g = sum of 16 random Fourier modes
    A_j cos(2 pi (kx_j x + ky_j y) + phi_j) with integer (kx, ky) != 0,
    |k| <= 8, A_j ~ N(0, 0.5^2), phi_j ~ U[0, 2 pi); sampled at interior points
    x_i = i/(n+1).  Returned grid-shaped with zero ghost ring."""
    cand = [(kx, ky) for kx in range(-8, 9) for ky in range(-8, 9)
            if (kx, ky) != (0, 0) and math.hypot(kx, ky) <= kmax]
    pick = (uniform01(seed, nmodes) * len(cand)).astype(np.int64)
    amp = normal(seed + 1, nmodes, 0.0, 0.5)
    phi = uniform(seed + 2, nmodes, 0.0, 2.0 * np.pi)
    x = np.arange(1, n + 1) / (n + 1.0)
    X, Y = np.meshgrid(x, x, indexing="xy")
    g = np.zeros((n, n))
    for j in range(nmodes):
        kx, ky = cand[pick[j]]
        g += amp[j] * np.cos(2.0 * np.pi * (kx * X + ky * Y) + phi[j])
    sig = np.zeros((n + 2, n + 2))
    sig[1:-1, 1:-1] = np.clip(10.0 * np.exp(g), 10.0, 1000.0)
    return sig


def differentiation_problem(n: int = 1024, nrhs: int = 16, seed: int = 7):
    """Screened Poisson with the Fourier sigma field, a batch of nrhs RHS
    f ~ U[-1,1] and a target u* ~ U[-1,1] drawn from another seed (loss
    L = 0.5 ||u - u*||^2)."""
    sig = fourier_sigma(n, seed)
    st = poisson_stencil(2, n, n, sigma=sig)
    fs = []
    for b in range(nrhs):
        f = zeros_grid(st)
        f[1:-1, 1:-1] = uniform(seed * 100 + b, n * n, -1.0, 1.0).reshape(n, n)
        fs.append(f)
    ustar = zeros_grid(st)
    ustar[1:-1, 1:-1] = uniform(seed * 100 + 99, n * n, -1.0, 1.0).reshape(n, n)
    return st, fs, ustar

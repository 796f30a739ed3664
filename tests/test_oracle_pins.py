"""Pins for the CPU oracle: each check fixes the oracle against something other
than itself -- a closed form, a library direct solver, a value the paper
prints, or an exact equivalence the paper states -- so that a dropped term, a
wrong sign, a wrong index or a transposed operand in oracle/hj_oracle.c fails
at least one test."""
import math
from pathlib import Path

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

import oracle
import workloads as W

GOLDEN = Path(__file__).parent / "golden"


def _golden(name):
    out = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.split("#")[0].strip()
        if line:
            parts = line.split()
            out[parts[0]] = parts[1:]
    return out


# ---------------------------------------------------------------------------
# independent dense assembly (from the operator's definition, by index loops)
# ---------------------------------------------------------------------------

def dense_system(st, f, u):
    """Dense interior matrix A and right-hand side b = f - (ghost terms) of
    A_int x = b, for 1D (every row a separate copy) or 2D."""
    nx = st.nx
    if st.dim == 1:
        rows = range(st.ny)
        n = nx * st.ny
        idx = lambda j, i: j * nx + (i - 1)
    else:
        rows = range(1, st.ny + 1)
        n = nx * st.ny
        idx = lambda j, i: (j - 1) * nx + (i - 1)
    A = np.zeros((n, n))
    b = np.zeros(n)
    for j in rows:
        for i in range(1, nx + 1):
            m = idx(j, i)
            sig = st.sigma_const + (st.sigma[j, i] if st.sigma is not None else 0.0)
            A[m, m] = st.cD + sig
            b[m] = f[j, i]
            cf = getattr(st, "coef", None)
            cw, ce = (st.cW, st.cE) if cf is None else (cf[0][j, i], cf[1][j, i])
            nbrs = [(j, i - 1, cw), (j, i + 1, ce)]
            if st.dim == 2:
                cs, cn = (st.cS, st.cN) if cf is None else (cf[2][j, i], cf[3][j, i])
                nbrs += [(j - 1, i, cs), (j + 1, i, cn)]
            for (jj, ii, c) in nbrs:
                ghost = ii == 0 or ii == nx + 1 or (st.dim == 2 and (jj == 0 or jj == st.ny + 1))
                if ghost:
                    b[m] -= c * u[jj, ii]
                else:
                    A[m, idx(jj, ii)] = c
    return A, b


def to_grid(st, x, like):
    g = like.copy()
    W.interior(g, st.dim)[...] = x.reshape(W.interior(g, st.dim).shape)
    return g


# ---------------------------------------------------------------------------
# generator pin
# ---------------------------------------------------------------------------

def test_splitmix64_reference_output():
    for seed, index, value in (map(int, v) for v in
                               [[k] + rest for k, rest in _golden("splitmix64.txt").items()]):
        assert int(W.splitmix64(seed, 1, index)[0]) == value


# ---------------------------------------------------------------------------
# operator and residual
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,nx,ny,sigma,asym", [(1, 13, 3, "field", True), (2, 9, 7, "field", True),
                                                   (2, 8, 5, "const", False), (1, 16, 1, "none", False)])
def test_apply_and_residual_match_dense(dim, nx, ny, sigma, asym):
    p = W.random_bc_problem(dim, nx, ny, seed=11, sigma_kind=sigma, asym=asym)
    A, b = dense_system(p.st, p.f, p.u0)
    x = W.interior(p.u0, dim).ravel()
    r_dense = b - A @ x
    assert oracle.residual(p.st, p.f, p.u0) == pytest.approx(np.linalg.norm(r_dense), rel=1e-13)
    Au = W.interior(oracle.apply(p.st, p.u0), dim).ravel()
    # A u on the grid includes the ghost contributions: A u = A_int x + (f - b)
    np.testing.assert_allclose(Au, A @ x + (W.interior(p.f, dim).ravel() - b), rtol=1e-13, atol=1e-9)


# ---------------------------------------------------------------------------
# classic Jacobi: closed-form decay of the discrete sine modes
# ---------------------------------------------------------------------------

def test_classic_jacobi_closed_form_1d():
    """u0 = 0, f = sum a_m sin(m pi x): after n sweeps
    u_n = sum (a_m / lam_m)(1 - cos(m pi h)^n) sin(m pi x), lam_m = (4/h^2) sin^2(m pi h / 2)."""
    prob = W.poisson1d_sine(N=127, nmodes=8, seed=0)
    N = prob.st.nx
    h = 1.0 / (N + 1)
    x = np.arange(N + 2) * h
    a = prob.meta["a"]
    for n in (1, 2, 7, 250):
        u = oracle.run_fixed(prob.st, prob.f, prob.u0, n, classic=True)
        exact = np.zeros(N + 2)
        for m in range(1, 9):
            lam = 4.0 / h ** 2 * math.sin(m * math.pi * h / 2) ** 2
            exact += a[m - 1] / lam * (1.0 - math.cos(m * math.pi * h) ** n) * np.sin(m * math.pi * x)
        np.testing.assert_allclose(u[0], exact, rtol=0, atol=1e-12 * np.abs(exact).max())


def test_classic_jacobi_closed_form_2d_rectangular():
    """Mode (p,q) of the 5-point operator with hx != hy is damped per sweep by
    (cos(p pi hx)/hx^2 + cos(q pi hy)/hy^2) / (1/hx^2 + 1/hy^2)."""
    nx, ny = 23, 17
    st = W.poisson_stencil(2, nx, ny)
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    X = np.arange(nx + 2) * hx
    Y = np.arange(ny + 2) * hy
    f = W.zeros_grid(st)
    modes = [(1, 1, 0.7), (3, 2, -1.1), (20, 15, 0.4)]
    for (pp, qq, amp) in modes:
        f += amp * np.outer(np.sin(qq * np.pi * Y), np.sin(pp * np.pi * X))
    f[0, :] = f[-1, :] = 0
    f[:, 0] = f[:, -1] = 0
    u0 = W.zeros_grid(st)
    for n in (1, 5, 40):
        u = oracle.run_fixed(st, f, u0, n, classic=True)
        exact = W.zeros_grid(st)
        for (pp, qq, amp) in modes:
            lam = 2 / hx ** 2 * (1 - math.cos(pp * math.pi * hx)) + 2 / hy ** 2 * (1 - math.cos(qq * math.pi * hy))
            mu = (math.cos(pp * math.pi * hx) / hx ** 2 + math.cos(qq * math.pi * hy) / hy ** 2) / (1 / hx ** 2 + 1 / hy ** 2)
            exact += amp / lam * (1 - mu ** n) * np.outer(np.sin(qq * np.pi * Y), np.sin(pp * np.pi * X))
        np.testing.assert_allclose(u, exact, rtol=0, atol=1e-12 * np.abs(exact).max())


def _sweeps_to_factor_closed_form(lam, mu, chat, factor):
    """First n with ||r_n|| <= factor ||r_0|| for r_n = -sum lam mu^n chat (orthogonal modes)."""
    w = (lam * chat) ** 2
    w0 = w.sum()

    def ratio2(n):
        return float((w * mu ** (2 * n)).sum() / w0)

    lo, hi = 0, 1
    while ratio2(hi) > factor ** 2:
        hi *= 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if ratio2(mid) > factor ** 2:
            lo = mid
        else:
            hi = mid
    return hi


def test_paper_1d_problem_sweep_count_matches_closed_form():
    """Section 3.5's problem (N = 1024, b = 1, initial solution 1, residual
    factor 1e-4): the oracle's classic sweep count equals the closed form."""
    g = _golden("paper_values.txt")
    N = int(g["e1_interior_points"][0])
    factor = float(g["e1_residual_factor"][0])
    prob = W.paper_replica(1, N)
    h = 1.0 / (N + 1)
    m = np.arange(1, N + 1)
    lam = 4.0 / h ** 2 * np.sin(m * np.pi * h / 2) ** 2
    mu = np.cos(m * np.pi * h)
    fhat = scipy.fft.dst(prob.f[0, 1:-1], type=1) / (N + 1)
    u0hat = scipy.fft.dst(prob.u0[0, 1:-1], type=1) / (N + 1)
    chat = u0hat - fhat / lam          # e_0 = u_0 - u*
    n_closed = _sweeps_to_factor_closed_form(lam, mu, chat, factor)
    _, n_oracle, status, _ = oracle.solve(prob.st, prob.f, prob.u0, factor, 10 ** 6, classic=True)
    assert status == 0
    assert n_oracle == n_closed


def test_2d_sweep_count_matches_closed_form():
    """Section 4.2's problem shape (b = 1, initial solution 1, factor 1e-4) on a
    48 x 40 grid: classic sweep count equals the 2D sine-basis closed form."""
    nx, ny = 48, 40
    st = W.poisson_stencil(2, nx, ny)
    f = W.zeros_grid(st)
    u0 = W.zeros_grid(st)
    f[1:-1, 1:-1] = 1.0
    u0[1:-1, 1:-1] = 1.0
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    P, Q = np.meshgrid(np.arange(1, nx + 1), np.arange(1, ny + 1), indexing="xy")
    lam = 2 / hx ** 2 * (1 - np.cos(P * np.pi * hx)) + 2 / hy ** 2 * (1 - np.cos(Q * np.pi * hy))
    mu = 1 - lam / (2 / hx ** 2 + 2 / hy ** 2)
    dst2 = lambda a: scipy.fft.dstn(a, type=1) / ((nx + 1) * (ny + 1))
    chat = dst2(u0[1:-1, 1:-1]) - dst2(f[1:-1, 1:-1]) / lam
    n_closed = _sweeps_to_factor_closed_form(lam.ravel(), mu.ravel(), chat.ravel(), 1e-4)
    _, n_oracle, status, _ = oracle.solve(st, f, u0, 1e-4, 10 ** 6, classic=True)
    assert status == 0 and n_oracle == n_closed


# ---------------------------------------------------------------------------
# hierarchical cycle: exact equivalences of Section 3.3
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,nx,ny,tx,ty", [(1, 100, 3, 32, 1), (2, 70, 45, 32, 16), (2, 64, 64, 32, 32)])
@pytest.mark.parametrize("sigma,asym", [("none", False), ("field", True)])
def test_k1_cycle_is_classic_sweep(dim, nx, ny, tx, ty, sigma, asym):
    """k = 1 is exactly classic Jacobi (Section 3.3), bitwise, ragged tiles too."""
    p = W.random_bc_problem(dim, nx, ny, seed=3, sigma_kind=sigma, asym=asym)
    a = oracle.hier_cycle(p.st, p.f, p.u0, tx, ty, 1)
    b = oracle.jacobi_sweep(p.st, p.f, p.u0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dim", [1, 2])
def test_single_subdomain_cycle_is_k_classic_sweeps(dim):
    """A subdomain covering the whole grid has the Dirichlet ring as its halo,
    so one cycle of k subiterations is k classic sweeps, bitwise."""
    p = W.random_bc_problem(dim, 20, 12 if dim == 2 else 2, seed=5, sigma_kind="field", asym=True)
    k = 9
    a = oracle.hier_cycle(p.st, p.f, p.u0, 32, 32, k)
    b = oracle.run_fixed(p.st, p.f, p.u0, k, classic=True)
    assert np.array_equal(a, b)


def test_large_k_cycle_is_blockwise_direct_solve():
    """As k grows a cycle solves every subdomain exactly with its halo frozen
    at u_in (block Jacobi).  Ragged 11 x 9 grid, 4 x 3 subdomains."""
    p = W.random_bc_problem(2, 11, 9, seed=8, sigma_kind="field", asym=True)
    st, f, u0 = p.st, p.f, p.u0
    tx, ty = 4, 3
    out = oracle.hier_cycle(st, f, u0, tx, ty, 4000)
    ref = u0.copy()
    for j0 in range(1, st.ny + 1, ty):
        for i0 in range(1, st.nx + 1, tx):
            j1, i1 = min(j0 + ty - 1, st.ny), min(i0 + tx - 1, st.nx)
            # local problem with the halo of u0 as Dirichlet data
            loc = W.poisson_stencil(2, i1 - i0 + 1, j1 - j0 + 1)
            loc.cW, loc.cE, loc.cS, loc.cN, loc.cD = st.cW, st.cE, st.cS, st.cN, st.cD
            loc.sigma = st.sigma[j0 - 1:j1 + 2, i0 - 1:i1 + 2]
            A, b = dense_system(loc, f[j0 - 1:j1 + 2, i0 - 1:i1 + 2], u0[j0 - 1:j1 + 2, i0 - 1:i1 + 2])
            x = np.linalg.solve(A, b)
            ref[j0:j1 + 1, i0:i1 + 1] = x.reshape(j1 - j0 + 1, i1 - i0 + 1)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_cycle_is_affine_and_counts_follow_spectral_radius():
    """One cycle is an affine map u -> G u + c.  G (built column by column from
    unit vectors with f = 0 and zero Dirichlet data) has spectral radius rho;
    the oracle's residual must contract asymptotically by rho per cycle."""
    st = W.poisson_stencil(2, 12, 10)
    n = 12 * 10
    tx, ty, k = 4, 4, 3
    zero = W.zeros_grid(st)
    G = np.zeros((n, n))
    for m in range(n):
        e = np.zeros(n)
        e[m] = 1.0
        G[:, m] = W.interior(oracle.hier_cycle(st, zero, to_grid(st, e, zero), tx, ty, k), 2).ravel()
    rho = max(abs(np.linalg.eigvals(G)))
    p = W.poisson2d_uniform(12, 10, seed=4)
    _, c, _, hist = oracle.solve(st, p.f, p.u0, 1e-13, 2000, tx, ty, k, hist_cap=2000)
    rate = (hist[c] / hist[c - 60]) ** (1.0 / 60)
    assert rate == pytest.approx(rho, rel=2e-3)


# ---------------------------------------------------------------------------
# fixed points: direct solvers
# ---------------------------------------------------------------------------

def test_thomas_matches_banded_lu():
    n = 200
    rng_a = W.uniform(21, n, -1, 0)
    rng_c = W.uniform(22, n, -1, 0)
    d = 2.5 + W.uniform(23, n, 0, 1)
    b = W.uniform(24, n, -1, 1)
    ab = np.zeros((3, n))
    ab[0, 1:] = rng_c[:-1]
    ab[1] = d
    ab[2, :-1] = rng_a[1:]
    ref = scipy.linalg.solve_banded((1, 1), ab, b)
    np.testing.assert_allclose(oracle.thomas(rng_a, d, rng_c, b), ref, rtol=1e-13)


@pytest.mark.parametrize("sigma,asym", [("none", False), ("field", True), ("const", False)])
def test_1d_hierarchical_converges_to_thomas(sigma, asym):
    p = W.random_bc_problem(1, 90, 3, seed=13, sigma_kind=sigma, asym=asym)
    st = p.st
    u, c, status, _ = oracle.solve(st, p.f, p.u0, 1e-13, 10 ** 7, 32, 1, 16)
    assert status == 0
    for j in range(st.ny):
        n = st.nx
        sig = st.sigma_const + (st.sigma[j, 1:-1] if st.sigma is not None else 0.0)
        d = st.cD + sig * np.ones(n)
        a = np.full(n, st.cW)
        cc = np.full(n, st.cE)
        b = p.f[j, 1:-1].copy()
        b[0] -= st.cW * p.u0[j, 0]
        b[-1] -= st.cE * p.u0[j, -1]
        x = oracle.thomas(a, d, cc, b)
        np.testing.assert_allclose(u[j, 1:-1], x, rtol=0, atol=1e-9 * np.abs(x).max())


def test_2d_hierarchical_converges_to_dst_solution():
    p = W.poisson2d_uniform(40, 28, seed=9)
    st = p.st
    u, c, status, _ = oracle.solve(st, p.f, p.u0, 1e-12, 10 ** 7, 16, 8, 8)
    assert status == 0
    hx, hy = 1 / (st.nx + 1), 1 / (st.ny + 1)
    P, Q = np.meshgrid(np.arange(1, st.nx + 1), np.arange(1, st.ny + 1), indexing="xy")
    lam = 2 / hx ** 2 * (1 - np.cos(P * np.pi * hx)) + 2 / hy ** 2 * (1 - np.cos(Q * np.pi * hy))
    fh = scipy.fft.dstn(p.f[1:-1, 1:-1], type=1)
    exact = scipy.fft.idstn(fh / lam, type=1)
    kappa = lam.max() / lam.min()
    err = np.linalg.norm(u[1:-1, 1:-1] - exact) / np.linalg.norm(exact)
    assert err <= kappa * 1e-12


@pytest.mark.parametrize("dim,nx,ny", [(2, 16, 16), (2, 13, 7), (1, 16, 4)])
def test_dense_brute_force_small(dim, nx, ny):
    """n <= 16 per side, screening field, non-symmetric stencil, random
    Dirichlet data, ragged subdomains: converged cycles equal a dense solve."""
    p = W.random_bc_problem(dim, nx, ny, seed=17, sigma_kind="field", asym=True)
    A, b = dense_system(p.st, p.f, p.u0)
    x = np.linalg.solve(A, b)
    u, c, status, _ = oracle.solve(p.st, p.f, p.u0, 1e-14, 10 ** 6, 5, 3, 4)
    assert status == 0
    np.testing.assert_allclose(W.interior(u, dim).ravel(), x, rtol=0, atol=1e-11 * np.abs(x).max())


# ---------------------------------------------------------------------------
# values printed in the paper
# ---------------------------------------------------------------------------

def test_paper_shared_memory_sizes():
    g = _golden("paper_values.txt")
    assert oracle.paper_smem_bytes(1, 32, 1, 8) == int(g["smem_bytes_1d_tpb32_fp64"][0])
    assert oracle.paper_smem_bytes(2, 32, 32, 8) == int(g["smem_bytes_2d_32x32_fp64"][0])


# ---------------------------------------------------------------------------
# mixed-precision refinement
# ---------------------------------------------------------------------------

def test_bf16_round_matches_library_conversion():
    torch = pytest.importorskip("torch")
    vals = np.concatenate([W.normal(31, 2000) * 10.0 ** W.uniform(32, 2000, -30, 30),
                           np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, -0.0,
                                     np.inf, -np.inf, 3.3895313892515355e38, 1e-40, -1e-45])])
    vals = vals.astype(np.float32)
    ref = torch.tensor(vals).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.bf16_round(float(v)) for v in vals], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("bf16", [False, True])
def test_iterative_refinement_reaches_direct_solution(bf16):
    n = 48
    p = W.poisson2d_sin_noise(n, seed=2)
    st = p.st
    tol = 1e-10
    u, outer, inner, status, hist = oracle.ir_solve(st, p.f, p.u0, tol, 16, 16, 8,
                                                    inner_tol=1e-2 if bf16 else 1e-4,
                                                    inner_max=20000, max_outer=60, bf16=bf16)
    assert status == 0
    assert hist[-1] <= tol * hist[0]
    assert oracle.residual(st, p.f, u) <= tol * hist[0]
    h = 1 / (n + 1)
    P, Q = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="xy")
    lam = 2 / h ** 2 * (2 - np.cos(P * np.pi * h) - np.cos(Q * np.pi * h))
    exact = scipy.fft.idstn(scipy.fft.dstn(p.f[1:-1, 1:-1], type=1) / lam, type=1)
    kappa = lam.max() / lam.min()
    assert np.linalg.norm(u[1:-1, 1:-1] - exact) / np.linalg.norm(exact) <= kappa * tol
    # refinement needs more than one outer step: the binary32 inner solve alone
    # cannot represent a 1e-10 residual
    assert outer >= 2


def test_f32_inner_cycle_close_to_f64_cycle():
    p = W.random_bc_problem(2, 40, 24, seed=19, sigma_kind="field")
    st = p.st
    z = W.zeros_grid(st)
    d64 = oracle.hier_cycle(st, p.f, z, 16, 8, 6)
    d32 = oracle.hier_cycle_f32(st, p.f.astype(np.float32), z.astype(np.float32), 16, 8, 6)
    np.testing.assert_allclose(d32, d64, rtol=0, atol=1e-6 * np.abs(d64).max())


# ---------------------------------------------------------------------------
# implicit adjoint
# ---------------------------------------------------------------------------

def _dense_loss_and_grads(st, f, u0, ustar):
    A, b = dense_system(st, f, u0)
    x = np.linalg.solve(A, b)
    g = x - W.interior(ustar, st.dim).ravel()
    lam = np.linalg.solve(A.T, g)
    return 0.5 * g @ g, x, lam


def test_adjoint_matches_dense_transpose_and_finite_differences():
    p = W.random_bc_problem(2, 10, 8, seed=23, sigma_kind="field", asym=True)
    st = p.st
    ustar = W.zeros_grid(st)
    ustar[1:-1, 1:-1] = W.uniform(24, 80, -1, 1).reshape(8, 10)
    L, x, lam_dense = _dense_loss_and_grads(st, p.f, p.u0, ustar)
    u = to_grid(st, x, p.u0)
    g = W.zeros_grid(st)
    g[1:-1, 1:-1] = u[1:-1, 1:-1] - ustar[1:-1, 1:-1]
    lam, dsig, status = oracle.adjoint(st, g, u, tol=1e-14, tx=4, ty=4, k=5)
    assert status == 0
    np.testing.assert_allclose(lam[1:-1, 1:-1].ravel(), lam_dense, rtol=0, atol=1e-10 * abs(lam_dense).max())
    # central finite differences of the loss (dense solves).  L is quadratic in
    # f, so a central difference in f is exact up to rounding at any step; in
    # sigma a relative step of 1e-3 balances truncation (~1e-8 relative) against
    # cancellation (L ~ 10 while dL/dsigma ~ 1e-5).
    for (j, i) in [(1, 1), (4, 7), (8, 10), (5, 2)]:
        eps = 1e-3 * st.sigma[j, i]
        sp = st.sigma.copy(); sp[j, i] += eps
        sm = st.sigma.copy(); sm[j, i] -= eps
        st_p = W.Stencil(**{**st.__dict__, "sigma": sp})
        st_m = W.Stencil(**{**st.__dict__, "sigma": sm})
        Lp = _dense_loss_and_grads(st_p, p.f, p.u0, ustar)[0]
        Lm = _dense_loss_and_grads(st_m, p.f, p.u0, ustar)[0]
        assert dsig[j, i] == pytest.approx((Lp - Lm) / (2 * eps), rel=1e-5, abs=1e-12)
        fp = p.f.copy(); fp[j, i] += 1e-2
        fm = p.f.copy(); fm[j, i] -= 1e-2
        Lp = _dense_loss_and_grads(st, fp, p.u0, ustar)[0]
        Lm = _dense_loss_and_grads(st, fm, p.u0, ustar)[0]
        assert lam[j, i] == pytest.approx((Lp - Lm) / 2e-2, rel=1e-6, abs=1e-12)


# ---------------------------------------------------------------------------
# Overlapping subdomains (Sections 3.4 and 4.3)
# ---------------------------------------------------------------------------

def _starts(n, T, o):
    """Subdomain starts at stride T - o; with overlap the last one is moved
    back so that it ends at n (the reading of the paper's non-integer block
    counts, e.g. 1020 / 28 for N = 1024, tpb = 32, o = 4)."""
    if n <= T:
        return [1]
    s = list(range(1, n - T + 2, T - o))
    if s[-1] + T - 1 < n:
        s.append(n - T + 1 if o > 0 else s[-1] + T)
    return s


def _owner_by_distance(n, T, starts):
    """Section 3.4: a point held by two subdomains is contributed by the one
    in which it lies further from an edge (a tie goes to the right one)."""
    own = np.zeros(n + 2, dtype=int)
    for i in range(1, n + 1):
        best, bd = -1, -1
        for j, s in enumerate(starts):
            e = min(s + T - 1, n)
            if s <= i <= e:
                d = min(i - s, e - i)
                if d >= bd:
                    best, bd = j, d
        own[i] = best
    return own


@pytest.mark.parametrize("dim,nx,ny,tx,ty,sigma", [(1, 57, 3, 8, 1, "field"), (2, 23, 19, 8, 6, "field"),
                                                   (2, 30, 17, 10, 5, "none")])
def test_overlap_zero_is_the_plain_cycle(dim, nx, ny, tx, ty, sigma):
    p = W.random_bc_problem(dim, nx, ny, seed=nx, sigma_kind=sigma, asym=True)
    for k in (1, 5):
        a = oracle.hier_cycle(p.st, p.f, p.u0, tx, ty, k)
        b = oracle.hier_cycle_ovl(p.st, p.f, p.u0, tx, ty, k, 0, 0)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dim,nx,ny,tx,ty,ox,oy", [(1, 57, 3, 8, 1, 2, 0), (1, 64, 2, 16, 1, 6, 0),
                                                   (2, 23, 19, 8, 6, 2, 2), (2, 31, 29, 10, 8, 4, 3)])
def test_overlap_k1_cycle_is_classic_sweep(dim, nx, ny, tx, ty, ox, oy):
    """With k = 1 every copy of a shared point takes the same single update
    from u_in, so any overlap gives one classic sweep, bitwise."""
    p = W.random_bc_problem(dim, nx, ny, seed=nx + 1, sigma_kind="field", asym=True)
    a = oracle.hier_cycle_ovl(p.st, p.f, p.u0, tx, ty, 1, ox, oy)
    b = oracle.jacobi_sweep(p.st, p.f, p.u0)
    assert np.array_equal(a, b)


def test_overlap_large_k_is_restricted_additive_schwarz():
    """As k grows every overlapping subdomain is solved exactly with its halo
    frozen at u_in, and each point takes the value of the subdomain that owns
    it (restricted additive Schwarz with exact local solves).  11 x 10 grid,
    4 x 4 subdomains overlapping by 2 (x) and 1 (y), clamped last subdomains."""
    p = W.random_bc_problem(2, 11, 10, seed=3, sigma_kind="field", asym=True)
    st, f, u0 = p.st, p.f, p.u0
    T, ox, oy = 4, 2, 1
    sx, sy = _starts(st.nx, T, ox), _starts(st.ny, T, oy)
    ownx, owny = _owner_by_distance(st.nx, T, sx), _owner_by_distance(st.ny, T, sy)
    out = oracle.hier_cycle_ovl(st, f, u0, T, T, 4000, ox, oy)
    ref = u0.copy()
    for jy, y0 in enumerate(sy):
        for jx, x0 in enumerate(sx):
            x1, y1 = min(x0 + T - 1, st.nx), min(y0 + T - 1, st.ny)
            loc = W.poisson_stencil(2, x1 - x0 + 1, y1 - y0 + 1)
            loc.cW, loc.cE, loc.cS, loc.cN, loc.cD = st.cW, st.cE, st.cS, st.cN, st.cD
            loc.sigma = st.sigma[y0 - 1:y1 + 2, x0 - 1:x1 + 2]
            A, b = dense_system(loc, f[y0 - 1:y1 + 2, x0 - 1:x1 + 2], u0[y0 - 1:y1 + 2, x0 - 1:x1 + 2])
            x = np.linalg.solve(A, b).reshape(y1 - y0 + 1, x1 - x0 + 1)
            for j in range(y0, y1 + 1):
                for i in range(x0, x1 + 1):
                    if ownx[i] == jx and owny[j] == jy:
                        ref[j, i] = x[j - y0, i - x0]
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_overlap_keeps_the_exact_solution_fixed():
    p = W.random_bc_problem(2, 14, 12, seed=5, sigma_kind="field", asym=True)
    A, b = dense_system(p.st, p.f, p.u0)
    ex = p.u0.copy()
    ex[1:-1, 1:-1] = np.linalg.solve(A, b).reshape(12, 14)
    out = oracle.hier_cycle_ovl(p.st, p.f, ex, 6, 5, 7, 2, 2)
    np.testing.assert_allclose(out, ex, rtol=1e-12, atol=1e-13)


def test_overlap_cycle_count_of_the_paper_1d_problem():
    """Section 3.4's best case, k = 16 with 4 overlapping points (tpb 32) on
    the Section 3.5 problem (N = 1024, b = 1, x0 = 1, residual reduced by
    1e-4): 8,093 cycles, the count an independent numpy implementation of
    this reading of the subdomain layout found; without overlap 19,555."""
    p = W.paper_replica(1, 1024, copies=1)
    _, c4, s4, _ = oracle.solve(p.st, p.f, p.u0, 1e-4, 10 ** 7, 32, 1, 16, overlap=(4, 0))
    _, c0, s0, _ = oracle.solve(p.st, p.f, p.u0, 1e-4, 10 ** 7, 32, 1, 16)
    assert s4 == 0 and s0 == 0
    assert c4 == 8093
    assert c0 == 19555


# ---------------------------------------------------------------------------
# Variable neighbour coefficients (the general tridiagonal matrix of Section 3
# and its 2D pentadiagonal analogue)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,nx,ny", [(1, 13, 3), (2, 9, 7)])
def test_variable_coefficients_apply_matches_dense(dim, nx, ny):
    p = W.variable_coef_problem(dim, nx, ny, seed=nx, contrast=20.0, screening=3.0)
    A, b = dense_system(p.st, p.f, p.u0)
    x = W.interior(p.u0, dim).ravel()
    r_dense = b - A @ x
    r = W.interior(p.f - oracle.apply(p.st, p.u0), dim).ravel()
    # apply() sees the ghost ring through u0: move those terms like dense_system does
    np.testing.assert_allclose(r, r_dense, rtol=1e-12, atol=1e-9 * np.abs(b).max())
    assert oracle.residual(p.st, p.f, p.u0) == pytest.approx(np.linalg.norm(r_dense), rel=1e-12)


@pytest.mark.parametrize("dim,nx,ny,tx,ty", [(1, 45, 2, 8, 1), (2, 23, 17, 8, 6)])
def test_variable_coefficients_k1_cycle_is_classic_sweep(dim, nx, ny, tx, ty):
    p = W.variable_coef_problem(dim, nx, ny, seed=5)
    for ovl in ((0, 0), (2, 2 if dim == 2 else 0)):
        a = oracle.hier_cycle_ovl(p.st, p.f, p.u0, tx, ty, 1, *ovl)
        assert np.array_equal(a, oracle.jacobi_sweep(p.st, p.f, p.u0))


def test_variable_coefficients_1d_converges_to_thomas():
    """The general tridiagonal system of Section 3 (a_i, d_i, c_i per row)
    solved by hierarchical cycles agrees with the Thomas algorithm."""
    n = 96
    p = W.variable_coef_problem(1, n, 1, seed=9, contrast=50.0)
    st = p.st
    a = st.coef[0][0, 1:n + 1].copy()
    c = st.coef[1][0, 1:n + 1].copy()
    d = st.sigma[0, 1:n + 1].copy()
    b = p.f[0, 1:n + 1].copy()
    b[0] -= a[0] * p.u0[0, 0]
    b[-1] -= c[-1] * p.u0[0, n + 1]
    x = oracle.thomas(a, d, c, b)
    u, cyc, status, _ = oracle.solve(st, p.f, p.u0, 1e-13, 10 ** 7, 16, 1, 12)
    assert status == 0
    kappa = 4 * 50.0 * (n + 1) ** 2 / (np.pi ** 2)
    assert np.abs(u[0, 1:n + 1] - x).max() <= kappa * 1e-13 * np.abs(x).max()


def test_variable_coefficients_large_k_and_fixed_point_2d():
    p = W.variable_coef_problem(2, 11, 9, seed=4, contrast=30.0, screening=5.0)
    st, f, u0 = p.st, p.f, p.u0
    tx, ty = 4, 3
    out = oracle.hier_cycle(st, f, u0, tx, ty, 4000)
    ref = u0.copy()
    for j0 in range(1, st.ny + 1, ty):
        for i0 in range(1, st.nx + 1, tx):
            j1, i1 = min(j0 + ty - 1, st.ny), min(i0 + tx - 1, st.nx)
            loc = W.Stencil(2, i1 - i0 + 1, j1 - j0 + 1, st.cW, st.cE, st.cS, st.cN, st.cD,
                            sigma=st.sigma[j0 - 1:j1 + 2, i0 - 1:i1 + 2],
                            coef=st.coef[:, j0 - 1:j1 + 2, i0 - 1:i1 + 2])
            A, b = dense_system(loc, f[j0 - 1:j1 + 2, i0 - 1:i1 + 2], u0[j0 - 1:j1 + 2, i0 - 1:i1 + 2])
            ref[j0:j1 + 1, i0:i1 + 1] = np.linalg.solve(A, b).reshape(j1 - j0 + 1, i1 - i0 + 1)
    np.testing.assert_allclose(out, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    A, b = dense_system(st, f, u0)
    ex = u0.copy()
    ex[1:-1, 1:-1] = np.linalg.solve(A, b).reshape(st.ny, st.nx)
    np.testing.assert_allclose(oracle.hier_cycle(st, f, ex, 5, 4, 6), ex, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("dim,nx,ny,tx,ty,k,vc", [(2, 11, 7, 4, 3, 3, False), (2, 9, 10, 5, 4, 2, True),
                                                  (1, 23, 2, 6, 1, 4, False), (1, 17, 3, 5, 1, 3, True)])
def test_cycle_at_finite_k_is_blockwise_jacobi_with_frozen_halos(dim, nx, ny, tx, ty, k, vc):
    """A hierarchical cycle is k Jacobi steps on every subdomain with its
    neighbours in other subdomains (and the ghost ring) held at the cycle's
    input (Sections 3.3, 4.1): built densely here block by block, ragged last
    blocks included, for constant and per-point coefficients."""
    if vc:
        p = W.variable_coef_problem(dim, nx, ny, seed=40 + nx, contrast=6.0, screening=2.0)
    else:
        p = W.random_bc_problem(dim, nx, ny, seed=40 + nx, sigma_kind="field", asym=True)
    A, b = dense_system(p.st, p.f, p.u0)
    d = np.diag(A)
    # block id per interior unknown, in the dense system's order (1D: every
    # row is its own problem)
    blk = np.array([(j * 1000 if dim == 1 else (j // ty) * 1000) + i // tx for j in range(ny) for i in range(nx)])
    same = blk[:, None] == blk[None, :]
    off_in = np.where(same, A, 0.0) - np.diag(d)
    off_out = np.where(same, 0.0, A)
    x0 = W.interior(p.u0, dim).reshape(-1)
    x = x0.copy()
    for _ in range(k):
        x = (b - off_in @ x - off_out @ x0) / d
    got = oracle.hier_cycle(p.st, p.f, p.u0, tx, ty, k)
    np.testing.assert_allclose(W.interior(got, dim).reshape(-1), x, rtol=0, atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("k", [2, 5])
def test_overlap_finite_k_is_local_jacobi_then_owner_selection(k):
    """Each overlapping subdomain runs k Jacobi steps on its own span with the
    halo frozen at u_in (its local dense system), and every point takes the
    value of its owner (Sections 3.4, 4.3).  11 x 10 grid, 4 x 4 subdomains
    overlapping by 2 (x) and 1 (y), clamped last subdomains."""
    p = W.random_bc_problem(2, 11, 10, seed=13 + k, sigma_kind="field", asym=True)
    st, f, u0 = p.st, p.f, p.u0
    T, ox, oy = 4, 2, 1
    sx, sy = _starts(st.nx, T, ox), _starts(st.ny, T, oy)
    ownx, owny = _owner_by_distance(st.nx, T, sx), _owner_by_distance(st.ny, T, sy)
    out = oracle.hier_cycle_ovl(st, f, u0, T, T, k, ox, oy)
    ref = u0.copy()
    for jy, y0 in enumerate(sy):
        for jx, x0 in enumerate(sx):
            x1, y1 = min(x0 + T - 1, st.nx), min(y0 + T - 1, st.ny)
            loc = W.poisson_stencil(2, x1 - x0 + 1, y1 - y0 + 1)
            loc.cW, loc.cE, loc.cS, loc.cN, loc.cD = st.cW, st.cE, st.cS, st.cN, st.cD
            loc.sigma = st.sigma[y0 - 1:y1 + 2, x0 - 1:x1 + 2]
            A, b = dense_system(loc, f[y0 - 1:y1 + 2, x0 - 1:x1 + 2], u0[y0 - 1:y1 + 2, x0 - 1:x1 + 2])
            d = np.diag(A)
            off = A - np.diag(d)
            x = u0[y0:y1 + 1, x0:x1 + 1].reshape(-1).copy()
            for _ in range(k):
                x = (b - off @ x) / d
            x = x.reshape(y1 - y0 + 1, x1 - x0 + 1)
            for j in range(y0, y1 + 1):
                for i in range(x0, x1 + 1):
                    if ownx[i] == jx and owny[j] == jy:
                        ref[j, i] = x[j - y0, i - x0]
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


# ---------------------------------------------------------------------------
# the OpenMP build: subdomains (and classic rows) on several threads give the
# single-thread result bit for bit (each reads u_c only and writes its own points)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,nx,ny,tx,ty,sigma", [(2, 203, 131, 32, 32, "field"), (2, 96, 64, 64, 16, "const"),
                                                    (1, 777, 9, 128, 1, "field")])
def test_threaded_oracle_is_bitwise_the_single_thread_oracle(dim, nx, ny, tx, ty, sigma):
    p = W.random_bc_problem(dim, nx, ny, seed=nx, sigma_kind=sigma, asym=True)
    try:
        ref_h = oracle.run_fixed(p.st, p.f, p.u0, 3, tx, ty, 5)
        ref_c = oracle.run_fixed(p.st, p.f, p.u0, 4, classic=True)
        ref_s = oracle.solve(p.st, p.f, p.u0, 1e-2, 10 ** 5, tx, ty, 5)
        for th in (2, 3, 8):
            got = oracle.set_threads(th)
            assert np.array_equal(oracle.run_fixed(p.st, p.f, p.u0, 3, tx, ty, 5), ref_h), got
            assert np.array_equal(oracle.run_fixed(p.st, p.f, p.u0, 4, classic=True), ref_c), got
            u, c, status, _ = oracle.solve(p.st, p.f, p.u0, 1e-2, 10 ** 5, tx, ty, 5)
            assert c == ref_s[1] and status == ref_s[2] and np.array_equal(u, ref_s[0])
    finally:
        oracle.set_threads(1)


def test_refinement_stagnation_rule_stops_at_the_bf16_fixed_point():
    """The inner solve of the refinement stops when ||r|| moved by at most
    1e-3 (relative) over a window of cycles.  With the correction stored in
    bfloat16 the cycles reach a bitwise fixed point (found here by brute force:
    iterate until a cycle changes nothing); the rule must stop the inner solve
    no later than the first window check after it, and at a residual within
    1e-3 of the fixed point's."""
    p = W.poisson2d_sin_noise(48, seed=2)
    st = p.st
    W_ = st.nx + 2
    u0 = np.zeros_like(p.f)
    r = (p.f - oracle.apply(st, u0)).astype(np.float32)
    r[0, :] = r[-1, :] = 0
    r[:, 0] = r[:, -1] = 0
    d = np.zeros_like(r)
    c_fp = None
    for c in range(20000):
        nd = oracle.hier_cycle_f32(st, r, d, 16, 16, 8, bf16=True)
        if np.array_equal(nd, d):
            c_fp = c
            break
        d = nd
    assert c_fp is not None and c_fp > 0
    r_fp = oracle.residual_f32(st, r, d)
    window = 32
    m = 1
    while (m - 1) * window < c_fp:
        m += 1
    bound = m * window
    _, outer, inner, status, hist = oracle.ir_solve(st, p.f, u0, 1e-30, 16, 16, 8, inner_tol=0.0, inner_max=10 ** 6,
                                                    max_outer=1, bf16=True, stall_window=window, stall_rtol=1e-3)
    assert outer == 1 and status == 1
    assert window <= inner <= bound, (inner, c_fp, bound)
    # here the residual keeps moving until the fixed point, so the rule fires
    # exactly at that first check (cycle 352 for a fixed point at cycle 297)
    assert inner == bound
    # the correction it stopped with sits at the fixed point's residual (to the rule's 1e-3)
    dd = np.zeros_like(r)
    for _ in range(inner):
        dd = oracle.hier_cycle_f32(st, r, dd, 16, 16, 8, bf16=True)
    assert abs(oracle.residual_f32(st, r, dd) - r_fp) <= 2e-3 * r_fp

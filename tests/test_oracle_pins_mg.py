"""Pins for the multigrid oracle (hierarchical Jacobi cycles with damped
subiterations as the smoother of a geometric V-cycle; full-weighting
restriction, bilinear prolongation, rediscretised coarse operators), checked
against dense matrices built here from the definitions: the prolongation P
and restriction R = P^T / 4, the damped Jacobi step, a two-level cycle as a
dense affine map with an exact coarse solve, the V-cycle's contraction on
Poisson and convergence to the dense solution."""
import numpy as np
import pytest

import oracle
import workloads as W


def dense2d(st, f, u):
    """Dense interior A and b = f - (ghost terms) of a 2D constant stencil."""
    nx, ny = st.nx, st.ny
    n = nx * ny
    A = np.zeros((n, n))
    b = np.zeros(n)
    idx = lambda j, i: (j - 1) * nx + (i - 1)
    for j in range(1, ny + 1):
        for i in range(1, nx + 1):
            m = idx(j, i)
            A[m, m] = st.cD + st.sigma_const
            b[m] = f[j, i]
            for (jj, ii, c) in [(j, i - 1, st.cW), (j, i + 1, st.cE), (j - 1, i, st.cS), (j + 1, i, st.cN)]:
                if ii == 0 or ii == nx + 1 or jj == 0 or jj == ny + 1:
                    b[m] -= c * u[jj, ii]
                else:
                    A[m, idx(jj, ii)] = c
    return A, b


def dense_prolongation(nx, ny):
    """Bilinear interpolation from the (nx-1)/2 x (ny-1)/2 coarse interior to
    the nx x ny fine interior, coarse point (I, J) on fine point (2I, 2J),
    zero coarse ghosts: weights 1, 1/2, 1/4 by parity of (i, j)."""
    ncx, ncy = (nx - 1) // 2, (ny - 1) // 2
    P = np.zeros((nx * ny, ncx * ncy))
    for j in range(1, ny + 1):
        for i in range(1, nx + 1):
            xs = [(i // 2, 1.0)] if i % 2 == 0 else [((i - 1) // 2, 0.5), ((i + 1) // 2, 0.5)]
            ys = [(j // 2, 1.0)] if j % 2 == 0 else [((j - 1) // 2, 0.5), ((j + 1) // 2, 0.5)]
            for (I, wx) in xs:
                for (J, wy) in ys:
                    if 1 <= I <= ncx and 1 <= J <= ncy:
                        P[(j - 1) * nx + (i - 1), (J - 1) * ncx + (I - 1)] += wx * wy
    return P


def interior(a):
    return a[1:-1, 1:-1].reshape(-1)


def test_level_count():
    assert oracle.mg_max_levels(127, 127) == 7
    assert oracle.mg_max_levels(127, 63) == 6
    assert oracle.mg_max_levels(128, 127) == 1
    assert oracle.mg_max_levels(1, 1) == 1
    assert oracle.mg_max_levels(7, 3) == 2


@pytest.mark.parametrize("nx,ny", [(7, 7), (15, 7), (9, 13)])
def test_prolongation_and_restriction_are_the_dense_operators(nx, ny):
    p = W.random_bc_problem(2, nx, ny, seed=nx * ny, sigma_kind="const", asym=True)
    P = dense_prolongation(nx, ny)
    ncx, ncy = (nx - 1) // 2, (ny - 1) // 2
    e = np.zeros((ncy + 2, ncx + 2))
    e[1:-1, 1:-1] = W.uniform(5, ncx * ncy, -1, 1).reshape(ncy, ncx)
    got = oracle.mg_prolong_add(p.st, e, p.u0)
    np.testing.assert_allclose(interior(got) - interior(p.u0), P @ interior(e), rtol=0, atol=1e-15)
    A, b = dense2d(p.st, p.f, p.u0)
    r = b - A @ interior(p.u0)
    fc = oracle.mg_restrict(p.st, p.f, p.u0)
    np.testing.assert_allclose(interior(fc), 0.25 * P.T @ r, rtol=1e-12, atol=1e-12 * np.abs(r).max())
    assert not fc[0].any() and not fc[-1].any() and not fc[:, 0].any() and not fc[:, -1].any()


@pytest.mark.parametrize("omega", [0.8, 0.5, 1.0])
def test_weighted_cycle_single_subdomain_is_damped_jacobi(omega):
    p = W.random_bc_problem(2, 9, 7, seed=3, sigma_kind="const", asym=True)
    A, b = dense2d(p.st, p.f, p.u0)
    d = np.diag(A)
    x = interior(p.u0)
    for _ in range(3):
        x = x + omega * (b - A @ x) / d
    got = oracle.mg_wcycle(p.st, p.f, p.u0, 16, 16, 3, omega)
    np.testing.assert_allclose(interior(got), x, rtol=1e-12, atol=1e-12)


def test_weighted_cycle_with_omega_one_is_the_plain_cycle():
    p = W.random_bc_problem(2, 45, 37, seed=4, sigma_kind="const", asym=True)
    a = oracle.mg_wcycle(p.st, p.f, p.u0, 16, 8, 5, 1.0)
    b = oracle.hier_cycle(p.st, p.f, p.u0, 16, 8, 5)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(b).max())


@pytest.mark.parametrize("shape", [(7, 7), (11, 5), (5, 9)])
@pytest.mark.parametrize("pre,post,k,omega", [(1, 1, 2, 0.8), (2, 1, 3, 0.6), (0, 2, 1, 0.8)])
def test_two_level_cycle_is_the_dense_affine_map(pre, post, k, omega, shape):
    """Smooth (damped Jacobi on one subdomain), restrict the residual with
    R = P^T / 4, solve the rediscretised coarse system exactly, prolongate,
    smooth again.  Rectangular grids with a non-symmetric stencil catch an x/y
    or W/E mix-up in any step."""
    nx, ny = shape
    p = W.random_bc_problem(2, nx, ny, seed=6 + nx, sigma_kind="const", asym=True)
    st = p.st
    A, b = dense2d(st, p.f, p.u0)
    d = np.diag(A)
    P = dense_prolongation(nx, ny)
    cst = oracle.mg_coarse_stencil(st)
    ncx, ncy = (nx - 1) // 2, (ny - 1) // 2
    Ac, _ = dense2d(cst, np.zeros((ncy + 2, ncx + 2)), np.zeros((ncy + 2, ncx + 2)))

    def smooth(x, cycles):
        for _ in range(cycles * k):
            x = x + omega * (b - A @ x) / d
        return x

    x = smooth(interior(p.u0), pre)
    ec = np.linalg.solve(Ac, 0.25 * P.T @ (b - A @ x))
    x = smooth(x + P @ ec, post)
    got = oracle.mg_vcycle(st, p.f, p.u0, 2, pre, post, nx, ny, k, omega, coarse_k=400, coarse_cycles=2)
    np.testing.assert_allclose(interior(got), x, rtol=0, atol=1e-12 * np.abs(x).max())
    assert np.array_equal(got[0], p.u0[0]) and np.array_equal(got[:, -1], p.u0[:, -1])


def test_vcycle_contracts_poisson_and_reaches_the_dense_solution():
    """V(1,1) with k = 4 damped sweeps per cycle on 32 x 32 subdomains: the
    textbook contraction of a weighted-Jacobi V-cycle (well below 0.2 per
    cycle) and the direct solution at the end."""
    p = W.random_bc_problem(2, 31, 31, seed=8, sigma_kind="const")
    L = oracle.mg_max_levels(31, 31)
    u, c, status, hist = oracle.mg_solve(p.st, p.f, p.u0, 1e-11, 100, L, 1, 1, 32, 32, 4, 0.8, hist_cap=100)
    assert status == 0 and c <= 20
    rates = hist[1:c + 1] / hist[:c]
    assert rates.max() < 0.2
    A, b = dense2d(p.st, p.f, p.u0)
    xs = np.linalg.solve(A, b)
    np.testing.assert_allclose(interior(u), xs, rtol=0, atol=1e-9 * np.abs(xs).max())
    # the Poisson problem of the bench family: V(2,2), k = 2, 127^2
    q = W.poisson2d_uniform(127, 127, seed=1)
    _, c2, s2, h2 = oracle.mg_solve(q.st, q.f, q.u0, 1e-10, 100, oracle.mg_max_levels(127, 127), 2, 2, 32, 32,
                                    2, 0.8, hist_cap=100)
    assert s2 == 0 and (h2[1:c2 + 1] / h2[:c2]).max() < 0.15


def test_two_level_cycle_with_tiles_equals_dense_blockwise_smoothing():
    """With 4 x 3 subdomains the smoothing cycle is damped Jacobi on each
    block with its halo frozen at the cycle start: built densely here block
    by block, then the same two-level map."""
    nx, ny, tx, ty, k, omega = 9, 7, 4, 3, 3, 0.7
    p = W.random_bc_problem(2, nx, ny, seed=21, sigma_kind="const", asym=True)
    st = p.st
    A, b = dense2d(st, p.f, p.u0)
    d = np.diag(A)
    P = dense_prolongation(nx, ny)
    cst = oracle.mg_coarse_stencil(st)
    Ac, _ = dense2d(cst, np.zeros((5, 6)), np.zeros((5, 6)))
    blk = np.array([((j // ty) * 100 + (i // tx)) for j in range(ny) for i in range(nx)])
    same = blk[:, None] == blk[None, :]
    Ain, Aout = np.where(same, A, 0.0), np.where(same, 0.0, A)

    def cycle(x):
        x0 = x.copy()
        for _ in range(k):   # neighbours in other blocks stay at x0
            x = x + omega * (b - Ain @ x - Aout @ x0) / d
        return x

    x = cycle(interior(p.u0))
    ec = np.linalg.solve(Ac, 0.25 * P.T @ (b - A @ x))
    x = cycle(x + P @ ec)
    got = oracle.mg_vcycle(st, p.f, p.u0, 2, 1, 1, tx, ty, k, omega, coarse_k=400, coarse_cycles=2)
    np.testing.assert_allclose(interior(got), x, rtol=0, atol=1e-12 * np.abs(x).max())

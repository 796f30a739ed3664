"""Pins for the 3D seven-point oracle (the 2D stencil of Section 4 extended by
a bottom/top pair; hierarchical cycles of Section 4.1 on tx x ty x tz
subdomains), checked against what the definitions fix: a dense matrix built
here from the stencil, the dense Jacobi step, the closed-form decay of the
lowest sine mode, the k = 1 equivalence with a classic sweep, the large-k
limit (a direct solve per subdomain with its halo frozen) and the discrete
solution as a fixed point.  Non-symmetric stencils (cW != cE, cS != cN,
cB != cT) make a swapped or mis-signed neighbour fail."""
import numpy as np
import pytest

import oracle
import workloads as W


def dense_system3d(st, f, u, box=None):
    """Dense A and b = f - (known-value terms) of A x = b over the interior,
    or over the sub-box ((x0, x1), (y0, y1), (z0, z1)) with every value
    outside it taken from u."""
    if box is None:
        box = ((1, st.nx), (1, st.ny), (1, st.nz))
    (x0, x1), (y0, y1), (z0, z1) = box
    nxb, nyb, nzb = x1 - x0 + 1, y1 - y0 + 1, z1 - z0 + 1
    n = nxb * nyb * nzb

    def idx(z, y, x):
        return ((z - z0) * nyb + (y - y0)) * nxb + (x - x0)

    def inside(z, y, x):
        return x0 <= x <= x1 and y0 <= y <= y1 and z0 <= z <= z1

    A = np.zeros((n, n))
    b = np.zeros(n)
    for z in range(z0, z1 + 1):
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                m = idx(z, y, x)
                A[m, m] = st.cD + st.sigma_const + (st.sigma[z, y, x] if st.sigma is not None else 0.0)
                b[m] = f[z, y, x]
                for (zz, yy, xx, c) in [(z, y, x - 1, st.cW), (z, y, x + 1, st.cE), (z, y - 1, x, st.cS),
                                        (z, y + 1, x, st.cN), (z - 1, y, x, st.cB), (z + 1, y, x, st.cT)]:
                    if inside(zz, yy, xx):
                        A[m, idx(zz, yy, xx)] = c
                    else:
                        b[m] -= c * u[zz, yy, xx]
    return A, b


def interior_vec(a):
    return W.interior(a, 3).reshape(-1)


@pytest.mark.parametrize("sigma,asym", [("none", False), ("field", True), ("const", True)])
def test_3d_apply_and_residual_match_dense(sigma, asym):
    p = W.random_bc_problem3d(5, 4, 3, seed=2, sigma_kind=sigma, asym=asym)
    A, b = dense_system3d(p.st, p.f, p.u0)
    x = interior_vec(p.u0)
    # A u on the interior = A_int x + ghost terms = A_int x + (f - b)
    au = interior_vec(oracle.apply(p.st, p.u0))
    np.testing.assert_allclose(au, A @ x + (interior_vec(p.f) - b), rtol=1e-13, atol=1e-9)
    r = oracle.residual(p.st, p.f, p.u0)
    assert r == pytest.approx(np.linalg.norm(b - A @ x), rel=1e-12)


@pytest.mark.parametrize("sigma,asym", [("none", False), ("field", True)])
def test_3d_classic_sweep_is_the_dense_jacobi_step(sigma, asym):
    p = W.random_bc_problem3d(6, 5, 4, seed=3, sigma_kind=sigma, asym=asym)
    A, b = dense_system3d(p.st, p.f, p.u0)
    d = np.diag(A)
    x = interior_vec(p.u0)
    want = (b - (A - np.diag(d)) @ x) / d
    got = oracle.jacobi_sweep(p.st, p.f, p.u0)
    np.testing.assert_allclose(interior_vec(got), want, rtol=1e-12, atol=1e-12)
    # the ghost shell carries over
    mask = np.ones(p.st.shape, bool)
    W.interior(mask, 3)[...] = False
    assert np.array_equal(got[mask], p.u0[mask])


def test_3d_classic_sweep_closed_form_decay():
    """-Lap on an (nx, ny, nz) box: the lowest sine mode is an eigenvector of
    the Jacobi iteration matrix with eigenvalue sum_a cos(pi h_a) 2/h_a^2
    over sum_a 2/h_a^2."""
    nx, ny, nz = 11, 7, 5
    st = W.poisson_stencil3d(nx, ny, nz)
    hs = [1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1)]
    lam = sum(np.cos(np.pi * h) * 2 / h ** 2 for h in hs) / sum(2 / h ** 2 for h in hs)
    x = np.arange(nx + 2) * hs[0]
    y = np.arange(ny + 2) * hs[1]
    z = np.arange(nz + 2) * hs[2]
    mode = np.sin(np.pi * z)[:, None, None] * np.sin(np.pi * y)[None, :, None] * np.sin(np.pi * x)[None, None, :]
    mode[0], mode[-1] = 0.0, 0.0
    mode[:, 0], mode[:, -1] = 0.0, 0.0
    mode[:, :, 0], mode[:, :, -1] = 0.0, 0.0
    f = W.zeros_grid(st)
    u = oracle.run_fixed(st, f, mode, 5, classic=True)
    np.testing.assert_allclose(u, lam ** 5 * mode, rtol=0, atol=1e-13)


@pytest.mark.parametrize("tile", [(4, 3, 2), (8, 8, 8), (3, 5, 7), (32, 4, 4)])
@pytest.mark.parametrize("sigma,asym", [("none", False), ("field", True)])
def test_3d_k1_cycle_is_classic_sweep(tile, sigma, asym):
    p = W.random_bc_problem3d(11, 9, 7, seed=4, sigma_kind=sigma, asym=asym)
    a = oracle.hier_cycle(p.st, p.f, p.u0, tile[0], tile[1], 1, tz=tile[2])
    b = oracle.jacobi_sweep(p.st, p.f, p.u0)
    assert np.array_equal(a, b)


def test_3d_single_subdomain_cycle_is_k_classic_sweeps():
    p = W.random_bc_problem3d(6, 5, 4, seed=5, sigma_kind="field", asym=True)
    a = oracle.hier_cycle(p.st, p.f, p.u0, 8, 8, 7, tz=8)
    b = oracle.run_fixed(p.st, p.f, p.u0, 7, classic=True)
    assert np.array_equal(a, b)


def test_3d_large_k_cycle_is_blockwise_direct_solve():
    """With k large, each subdomain's interior solves its block system with
    the halo frozen at u_in (ragged last subdomains included)."""
    p = W.random_bc_problem3d(7, 5, 6, seed=6, sigma_kind="field", asym=True)
    tx, ty, tz = 3, 2, 4
    got = oracle.hier_cycle(p.st, p.f, p.u0, tx, ty, 4000, tz=tz)
    want = p.u0.copy()
    for z0 in range(1, 7, tz):
        for y0 in range(1, 6, ty):
            for x0 in range(1, 8, tx):
                box = ((x0, min(x0 + tx - 1, 7)), (y0, min(y0 + ty - 1, 5)), (z0, min(z0 + tz - 1, 6)))
                A, b = dense_system3d(p.st, p.f, p.u0, box)
                sol = np.linalg.solve(A, b)
                (a0, a1), (b0, b1), (c0, c1) = box
                want[c0:c1 + 1, b0:b1 + 1, a0:a1 + 1] = sol.reshape(c1 - c0 + 1, b1 - b0 + 1, a1 - a0 + 1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_3d_discrete_solution_is_a_fixed_point_and_solve_reaches_it():
    p = W.random_bc_problem3d(9, 6, 5, seed=7, sigma_kind="const", asym=True)
    A, b = dense_system3d(p.st, p.f, p.u0)
    xs = np.linalg.solve(A, b)
    us = p.u0.copy()
    W.interior(us, 3)[...] = xs.reshape(5, 6, 9)
    one = oracle.hier_cycle(p.st, p.f, us, 4, 4, 16, tz=2)
    np.testing.assert_allclose(one, us, rtol=0, atol=1e-12 * np.abs(us).max())
    u, c, status, hist = oracle.solve(p.st, p.f, p.u0, 1e-11, 100000, 4, 4, 16, tz=2, hist_cap=100000)
    assert status == 0
    assert hist[c] <= 1e-11 * hist[0] < hist[c - 1]
    np.testing.assert_allclose(u, us, rtol=0, atol=1e-9 * np.abs(us).max())
    # the history is the residual of every iterate
    assert hist[0] == pytest.approx(oracle.residual(p.st, p.f, p.u0), rel=1e-15)


@pytest.mark.parametrize("tile,k", [((3, 2, 2), 3), ((4, 3, 5), 2), ((2, 5, 1), 4)])
def test_3d_cycle_at_finite_k_is_blockwise_jacobi_with_frozen_halos(tile, k):
    """A cycle is k Jacobi steps on every subdomain, its neighbours in other
    subdomains (and the ghost shell) held at the cycle's input: built densely
    here block by block (ragged last blocks included)."""
    nx, ny, nz = 7, 5, 6
    tx, ty, tz = tile
    p = W.random_bc_problem3d(nx, ny, nz, seed=30 + k, sigma_kind="field", asym=True)
    A, b = dense_system3d(p.st, p.f, p.u0)
    d = np.diag(A)
    blk = np.array([((z // tz) * 10000 + (y // ty) * 100 + x // tx)
                    for z in range(nz) for y in range(ny) for x in range(nx)])
    same = blk[:, None] == blk[None, :]
    off_in = np.where(same, A, 0.0) - np.diag(d)
    off_out = np.where(same, 0.0, A)
    x0 = interior_vec(p.u0)
    x = x0.copy()
    for _ in range(k):
        x = (b - off_in @ x - off_out @ x0) / d
    got = oracle.hier_cycle(p.st, p.f, p.u0, tx, ty, k, tz=tz)
    np.testing.assert_allclose(interior_vec(got), x, rtol=0, atol=1e-12 * np.abs(x).max())

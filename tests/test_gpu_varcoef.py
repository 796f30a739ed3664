"""GPU parity for per-point neighbour coefficients (the general tridiagonal
a_i, c_i of Section 3 and its five-point analogue): the thread-per-point
kernel called through the C ABI against the CPU oracle on the same seeded
heterogeneous-diffusion problems.

Tolerances: binary64 cycles follow the oracle's evaluation order without
fused multiply-add and must agree bitwise at equal cycle counts; binary32
cycles (binary32 -c/d and 1/d planes) stay within 1e-5 (relative, max norm)
of the binary64 oracle on these small grids.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import gpu_solver, rel_max, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("tile", [(32, 32), (32, 8), (16, 16), (8, 4)])
@pytest.mark.parametrize("shape,screening", [((70, 45), 0.0), ((64, 64), 50.0), ((97, 33), 0.0)])
def test_f64_varcoef_cycles_match_oracle_2d(tile, shape, screening):
    torch = _torch()
    nx, ny = shape
    p = W.variable_coef_problem(2, nx, ny, seed=nx + ny, contrast=20.0, screening=screening)
    for k, ncyc in [(1, 3), (5, 4), (16, 2)]:
        s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f64", fixed_cycles=ncyc)
        u = to_dev(p.u0, 2, torch.float64)
        s.solve(to_dev(p.f, 2, torch.float64), u)
        ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile[0], tile[1], k)
        assert np.array_equal(to_host(u, nx), ref), (tile, k, rel_max(to_host(u, nx), ref))
        s.close()


@pytest.mark.parametrize("tile", [32, 64, 256, 1024])
@pytest.mark.parametrize("n,copies", [(300, 3), (1000, 1)])
def test_f64_varcoef_cycles_match_oracle_1d(tile, n, copies):
    torch = _torch()
    p = W.variable_coef_problem(1, n, copies, seed=n, contrast=10.0)
    for k, ncyc in [(1, 3), (32, 3)]:
        s = gpu_solver(p, tile_x=tile, k=k, precision="f64", fixed_cycles=ncyc)
        u = to_dev(p.u0, 1, torch.float64)
        s.solve(to_dev(p.f, 1, torch.float64), u)
        ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile, 1, k)
        assert np.array_equal(to_host(u, n), ref), (tile, k)
        s.close()


@pytest.mark.parametrize("dim", [1, 2])
def test_f64_varcoef_classic_sweeps_match_oracle(dim):
    torch = _torch()
    p = W.variable_coef_problem(dim, 77, 41 if dim == 2 else 3, seed=5, contrast=8.0, screening=3.0)
    s = gpu_solver(p, method="classic", precision="f64", fixed_cycles=9)
    u = to_dev(p.u0, dim, torch.float64)
    s.solve(to_dev(p.f, dim, torch.float64), u)
    ref = oracle.run_fixed(p.st, p.f, p.u0, 9, classic=True)
    assert np.array_equal(to_host(u, p.st.nx), ref)
    s.close()


@pytest.mark.parametrize("dim,shape,tile,k", [(2, (96, 80), (32, 32), 16), (2, (70, 45), (16, 16), 8),
                                              (1, (512, 2), (128, 1), 32)])
def test_f64_varcoef_convergence_matches_oracle(dim, shape, tile, k):
    """Same stopping cycle, iterate and residual history as the oracle."""
    torch = _torch()
    nx, ny = shape
    p = W.variable_coef_problem(dim, nx, ny, seed=19, contrast=10.0, screening=1.0)
    tol = 1e-8
    s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f64", tol=tol, check_every=16)
    u = to_dev(p.u0, dim, torch.float64)
    out = s.solve(to_dev(p.f, dim, torch.float64), u, history=100000)
    uo, c, status, hist = oracle.solve(p.st, p.f, p.u0, tol, 10 ** 7, tile[0], tile[1], k, hist_cap=100000)
    assert status == 0 and out["status"] == 0 and out["persistent"] == 0
    assert out["cycles"] == c
    assert np.array_equal(to_host(u, nx), uo)
    np.testing.assert_allclose(np.array(out["history"]), hist[:c + 1], rtol=1e-9, atol=1e-12 * hist[0])
    assert oracle.residual(p.st, p.f, uo) <= tol * oracle.residual(p.st, p.f, p.u0)
    s.close()


def test_varcoef_with_constant_planes_equals_constant_coefficient_solver():
    """Planes holding the constant cW..cN give the constant-coefficient
    iterates (binary64: the same products in the same order)."""
    torch = _torch()
    p = W.random_bc_problem(2, 70, 45, seed=3, sigma_kind="field", asym=False)
    st = p.st
    rows = st.ny + 2
    planes = np.zeros((4, rows, st.nx + 2))
    for i, c in enumerate([st.cW, st.cE, st.cS, st.cN]):
        planes[i][1:-1, 1:-1] = c
    import dataclasses
    st_vc = dataclasses.replace(st, coef=planes)
    ref = oracle.run_fixed(st, p.f, p.u0, 4, 32, 32, 6)
    ref_vc = oracle.run_fixed(st_vc, p.f, p.u0, 4, 32, 32, 6)
    assert rel_max(ref_vc, ref) <= 1e-13
    s = gpu_solver(st_vc, tile_x=32, tile_y=32, k=6, precision="f64", fixed_cycles=4)
    u = to_dev(p.u0, 2, torch.float64)
    s.solve(to_dev(p.f, 2, torch.float64), u)
    assert np.array_equal(to_host(u, st.nx), ref_vc)
    s.close()


@pytest.mark.parametrize("dim,tile", [(2, (32, 32)), (2, (16, 8)), (1, (256, 1))])
def test_f32_varcoef_cycles_close_to_oracle_and_solve_converges(dim, tile):
    torch = _torch()
    nx, ny = (150, 120) if dim == 2 else (700, 3)
    p = W.variable_coef_problem(dim, nx, ny, seed=23, contrast=10.0, screening=2.0)
    s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=8, precision="f32", fixed_cycles=6)
    u = to_dev(p.u0, dim, torch.float32)
    s.solve(to_dev(p.f, dim, torch.float32), u)
    ref = oracle.run_fixed(p.st, p.f, p.u0, 6, tile[0], tile[1], 8)
    assert rel_max(to_host(u, nx), ref) <= 1e-5
    s.close()
    s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=8, precision="f32", tol=1e-4, check_every=8)
    u = to_dev(p.u0, dim, torch.float32)
    out = s.solve(to_dev(p.f, dim, torch.float32), u)
    assert out["status"] == 0
    r = oracle.residual(p.st, p.f, to_host(u, nx))
    assert r <= 1.01e-4 * oracle.residual(p.st, p.f, p.u0)
    s.close()


def test_varcoef_residual_api_matches_oracle():
    torch = _torch()
    p = W.variable_coef_problem(2, 90, 61, seed=2, contrast=30.0)
    s = gpu_solver(p, tile_x=32, tile_y=32, k=4, precision="f64", fixed_cycles=1)
    a, r = s.residual(to_dev(p.f, 2, torch.float64), to_dev(p.u0, 2, torch.float64))
    ro = oracle.residual(p.st, p.f, p.u0)
    assert a == pytest.approx(ro, rel=1e-12)
    assert r == pytest.approx(ro / np.linalg.norm(W.interior(p.f, 2)), rel=1e-12)
    s.close()


def test_varcoef_is_rejected_where_unsupported():
    import paper_2006_16465_gb300 as hj
    torch = _torch()
    p = W.variable_coef_problem(2, 64, 64, seed=1)
    for kw, code in [(dict(precision="f32_ir"), hj.HJ_ERR_UNSUPPORTED),
                     (dict(persistent=1), hj.HJ_ERR_UNSUPPORTED),
                     (dict(pipeline=1), hj.HJ_ERR_UNSUPPORTED),
                     (dict(overlap_x=4, overlap_y=4), hj.HJ_ERR_UNSUPPORTED),
                     (dict(tile_x=64, tile_y=32), hj.HJ_ERR_UNSUPPORTED)]:
        params = dict(tile_x=32, tile_y=32, precision="f64")
        params.update(kw)
        with pytest.raises(hj.HJError) as e:
            gpu_solver(p, **params)
        assert e.value.code == code, kw
    # a coefficient plane that breaks diagonal dominance
    st = p.st
    import dataclasses
    bad = st.coef.copy()
    bad[0][10, 10] *= 3.0
    with pytest.raises(hj.HJError) as e:
        gpu_solver(dataclasses.replace(st, coef=bad), tile_x=32, tile_y=32, precision="f64")
    assert e.value.code == hj.HJ_ERR_NOT_DIAG_DOMINANT
    # the adjoint is built for constant coefficients
    s = gpu_solver(p, tile_x=32, tile_y=32, precision="f64", tol=1e-8)
    g = to_dev(p.f, 2, torch.float64)
    u = to_dev(p.u0, 2, torch.float64)
    with pytest.raises(hj.HJError) as e:
        s.adjoint(g, u, torch.zeros_like(u))
    assert e.value.code == hj.HJ_ERR_UNSUPPORTED
    s.close()


def test_varcoef_is_rejected_by_batched_and_noalloc_entry_points():
    """Both entry points take constant neighbour coefficients only; a
    descriptor with coefficient planes is refused before any launch."""
    import paper_2006_16465_gb300 as hj
    torch = _torch()
    p = W.variable_coef_problem(2, 64, 64, seed=4)
    st = p.st
    f = to_dev(p.f, 2, torch.float64)
    u = to_dev(p.u0, 2, torch.float64)
    planes = torch.zeros((4, st.ny + 2, f.shape[1]), dtype=torch.float64, device="cuda")
    planes[:, :, :st.nx + 2] = torch.as_tensor(st.coef)
    sig = to_dev(st.sigma, 2, torch.float64)
    d = hj.make_desc(2, st.nx, st.ny, f.shape[1], st.cW, st.cE, st.cS, st.cN, st.cD, st.sigma_const, sig, hj.HJ_F64,
                     planes)
    code = hj.hj_cycles_noalloc(d, hj.make_params(fixed_cycles=2, precision="f64"), f.data_ptr(), u.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert code == hj.HJ_ERR_UNSUPPORTED
    q = W.poisson2d_uniform(64, 64, seed=1)
    s = gpu_solver(q, tile_x=32, tile_y=32, k=16, precision="f32_ir", tol=1e-8)
    cyc = (hj.C.c_longlong * 1)()
    code = hj.hj_solve_batched(s.h, [d], [f.data_ptr()], [u.data_ptr()], 0, None, cyc)
    assert code == hj.HJ_ERR_UNSUPPORTED
    s.close()
    assert np.array_equal(to_host(u, st.nx), p.u0)

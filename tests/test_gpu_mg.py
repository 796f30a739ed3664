"""GPU parity for multigrid V-cycles whose smoother is the hierarchical cycle
with damped Jacobi subiterations (full-weighting restriction, bilinear
prolongation, rediscretised coarse operators), called through the C ABI,
against the multigrid oracle on the same seeded inputs.

Tolerances: binary64 evaluates every sum in the oracle's order without fused
multiply-add, so V-cycles must agree bitwise at equal counts; binary32 stays
within 1e-5 (relative, max norm) of the binary64 oracle after two V-cycles."""
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


CASES = [((127, 127), (32, 32), 1, 1, 2, 0.8), ((95, 47), (16, 8), 2, 1, 4, 0.6), ((63, 31), (32, 8), 0, 2, 3, 0.8),
         ((255, 63), (32, 16), 1, 2, 2, 1.0)]


@pytest.mark.parametrize("shape,tile,pre,post,k,omega", CASES)
def test_f64_vcycles_match_oracle(shape, tile, pre, post, k, omega):
    torch = _torch()
    nx, ny = shape
    p = W.random_bc_problem(2, nx, ny, seed=nx + ny, sigma_kind="const", asym=True)
    L = oracle.mg_max_levels(nx, ny)
    s = gpu_solver(p, method="mg", precision="f64", tile_x=tile[0], tile_y=tile[1], k=k, mg_pre=pre, mg_post=post,
                   mg_omega=omega, fixed_cycles=2)
    u = to_dev(p.u0, 2, torch.float64)
    s.solve(to_dev(p.f, 2, torch.float64), u)
    ref = p.u0
    for _ in range(2):
        ref = oracle.mg_vcycle(p.st, p.f, ref, L, pre, post, tile[0], tile[1], k, omega)
    got = to_host(u, nx)
    assert np.array_equal(got, ref), rel_max(got, ref)
    s.close()


@pytest.mark.parametrize("levels", [3, 4, 6])
def test_f64_vcycles_with_fewer_levels_match_oracle(levels):
    torch = _torch()
    p = W.random_bc_problem(2, 127, 63, seed=3, sigma_kind="const", asym=True)
    s = gpu_solver(p, method="mg", precision="f64", tile_x=32, tile_y=16, k=3, mg_levels=levels, fixed_cycles=3)
    u = to_dev(p.u0, 2, torch.float64)
    s.solve(to_dev(p.f, 2, torch.float64), u)
    ref = p.u0
    for _ in range(3):
        ref = oracle.mg_vcycle(p.st, p.f, ref, levels, 1, 1, 32, 16, 3, 0.8)
    assert np.array_equal(to_host(u, 127), ref)
    s.close()


@pytest.mark.parametrize("shape,pre,post,k", [((127, 127), 1, 1, 4), ((255, 127), 2, 2, 2)])
def test_f64_mg_solve_matches_oracle(shape, pre, post, k):
    """Same V-cycle count, iterate and residual history as the oracle."""
    torch = _torch()
    nx, ny = shape
    p = W.random_bc_problem(2, nx, ny, seed=7, sigma_kind="const")
    tol = 1e-10
    s = gpu_solver(p, method="mg", precision="f64", tile_x=32, tile_y=32, k=k, mg_pre=pre, mg_post=post, tol=tol,
                   max_cycles=200)
    u = to_dev(p.u0, 2, torch.float64)
    out = s.solve(to_dev(p.f, 2, torch.float64), u, history=1000)
    L = oracle.mg_max_levels(nx, ny)
    uo, c, status, hist = oracle.mg_solve(p.st, p.f, p.u0, tol, 1000, L, pre, post, 32, 32, k, 0.8, hist_cap=1000)
    assert status == 0 and out["status"] == 0
    assert out["cycles"] == c and c <= 20
    assert np.array_equal(to_host(u, nx), uo)
    np.testing.assert_allclose(np.array(out["history"]), hist[:c + 1], rtol=1e-9, atol=1e-13 * hist[0])
    assert oracle.residual(p.st, p.f, uo) <= tol * oracle.residual(p.st, p.f, p.u0)
    s.close()


def test_f32_vcycles_close_to_oracle_and_solve_converges():
    torch = _torch()
    p = W.random_bc_problem(2, 127, 95, seed=11, sigma_kind="const", asym=True)
    s = gpu_solver(p, method="mg", precision="f32", tile_x=32, tile_y=32, k=2, fixed_cycles=2)
    u = to_dev(p.u0, 2, torch.float32)
    s.solve(to_dev(p.f, 2, torch.float32), u)
    L = oracle.mg_max_levels(127, 95)
    ref = p.u0
    for _ in range(2):
        ref = oracle.mg_vcycle(p.st, p.f, ref, L, 1, 1, 32, 32, 2, 0.8)
    assert rel_max(to_host(u, 127), ref) <= 1e-5
    s.close()
    # binary32 storage of u floors the relative residual near eps |u| / h^2:
    # 1e-4 is reachable at 63^2
    q = W.poisson2d_uniform(63, 63, seed=1)
    s = gpu_solver(q, method="mg", precision="f32", tile_x=32, tile_y=32, k=2, mg_pre=2, mg_post=2, tol=1e-4,
                   max_cycles=50)
    u = to_dev(q.u0, 2, torch.float32)
    out = s.solve(to_dev(q.f, 2, torch.float32), u)
    assert out["status"] == 0 and out["cycles"] <= 12
    r = oracle.residual(q.st, q.f, to_host(u, 63))
    assert r <= 1.01e-4 * oracle.residual(q.st, q.f, q.u0)
    s.close()


def test_f32_mg_stops_at_the_storage_floor():
    """A target below binary32's residual floor ends with NOT_CONVERGED once
    the residual stops falling, not after max_cycles."""
    import paper_2006_16465_gb300 as hj
    torch = _torch()
    q = W.poisson2d_uniform(511, 511, seed=1)
    s = gpu_solver(q, method="mg", precision="f32", k=2, tol=1e-12, max_cycles=200)
    u = to_dev(q.u0, 2, torch.float32)
    out = s.solve(to_dev(q.f, 2, torch.float32), u)
    assert out["status"] == hj.HJ_ERR_NOT_CONVERGED
    assert out["cycles"] < 60 and out["rel_final"] < 1e-2
    s.close()


def test_mg_host_pointer_solve_equals_device_solve():
    import paper_2006_16465_gb300 as hj
    torch = _torch()
    p = W.random_bc_problem(2, 63, 63, seed=12, sigma_kind="const")
    s = gpu_solver(p, method="mg", precision="f64", fixed_cycles=3)
    f = to_dev(p.f, 2, torch.float64)
    u = to_dev(p.u0, 2, torch.float64)
    s.solve(f, u)
    fh, uh = f.cpu(), to_dev(p.u0, 2, torch.float64).cpu()
    assert hj.hj_solve(s.h, fh.data_ptr(), uh.data_ptr(), 0, None) == hj.HJ_OK
    assert torch.equal(uh, u.cpu())
    s.close()


def test_mg_is_rejected_where_unsupported():
    import paper_2006_16465_gb300 as hj
    torch = _torch()
    p = W.poisson2d_uniform(127, 127, seed=1)
    for st, kw, code in [(W.poisson2d_uniform(128, 127).st, {}, hj.HJ_ERR_INVALID_ARG),
                         (p.st, dict(mg_omega=1.5), hj.HJ_ERR_INVALID_ARG),
                         (p.st, dict(mg_levels=1), hj.HJ_ERR_INVALID_ARG),
                         (W.poisson2d_uniform(255, 255).st, dict(mg_levels=3), hj.HJ_ERR_UNSUPPORTED),
                         (p.st, dict(precision="f32_ir"), hj.HJ_ERR_UNSUPPORTED),
                         (p.st, dict(tile_x=64, tile_y=32), hj.HJ_ERR_INVALID_ARG),
                         (W.random_bc_problem(2, 63, 63, seed=1, sigma_kind="field").st, {}, hj.HJ_ERR_UNSUPPORTED),
                         (W.poisson3d_uniform(31).st, {}, hj.HJ_ERR_UNSUPPORTED)]:
        params = dict(method="mg", precision="f64")
        params.update(kw)
        with pytest.raises(hj.HJError) as e:
            gpu_solver(st, **params)
        assert e.value.code == code, kw
    s = gpu_solver(p, method="mg", precision="f64", tol=1e-8, max_cycles=100)
    g = to_dev(p.f, 2, torch.float64)
    with pytest.raises(hj.HJError) as e:
        s.adjoint(g, to_dev(p.u0, 2, torch.float64), torch.zeros_like(g))
    assert e.value.code == hj.HJ_ERR_UNSUPPORTED
    s.close()

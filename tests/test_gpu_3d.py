"""GPU parity for the 3D seven-point extension (the five-point stencil of
Section 4 plus a bottom/top pair, hierarchical cycles on TX x TY x TZ
subdomains), called through the C ABI, against the 3D oracle on the same
seeded inputs.

Tolerances: binary64 cycles follow the oracle's evaluation order without
fused multiply-add and must agree bitwise at equal cycle counts; binary32
cycles stay within 1e-5 (relative, max norm) of the binary64 oracle on these
small grids (six fused multiply-adds per update, a few cycles)."""
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


def _shapes(prec):
    import paper_2006_16465_gb300 as hj
    return hj.hj_tile_shapes3d(hj.PRECISIONS[prec])


@pytest.mark.parametrize("pipeline", [0, 1])
@pytest.mark.parametrize("shape,sigma,asym", [((37, 21, 13), "none", True), ((32, 16, 16), "const", False),
                                               ((50, 9, 20), "const", True)])
def test_f64_3d_cycles_match_oracle(shape, sigma, asym, pipeline):
    """pipeline = 1: persistent warps prefetching the next subdomain's box
    with cp.async (small grids: a warp walks several subdomains); 0: one
    warp per subdomain, loads issued directly."""
    torch = _torch()
    nx, ny, nz = shape
    p = W.random_bc_problem3d(nx, ny, nz, seed=nx + ny + nz, sigma_kind=sigma, asym=asym)
    for tile in _shapes("f64"):
        for k, ncyc in [(1, 3), (5, 2), (16, 2)]:
            s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], tile_z=tile[2], k=k, precision="f64",
                           fixed_cycles=ncyc, pipeline=pipeline)
            u = to_dev(p.u0, 3, torch.float64)
            s.solve(to_dev(p.f, 3, torch.float64), u)
            ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile[0], tile[1], k, tz=tile[2])
            got = to_host(u, nx)
            assert np.array_equal(got, ref), (tile, k, rel_max(got, ref))
            s.close()


def test_f64_3d_classic_sweeps_match_oracle():
    torch = _torch()
    p = W.random_bc_problem3d(45, 19, 11, seed=5, sigma_kind="const", asym=True)
    s = gpu_solver(p, method="classic", precision="f64", fixed_cycles=7)
    u = to_dev(p.u0, 3, torch.float64)
    s.solve(to_dev(p.f, 3, torch.float64), u)
    ref = oracle.run_fixed(p.st, p.f, p.u0, 7, classic=True)
    assert np.array_equal(to_host(u, 45), ref)
    s.close()


@pytest.mark.parametrize("method,k,pipeline", [("hier", 8, 0), ("hier", 32, 0), ("hier", 8, 1), ("classic", 1, 0)])
def test_f64_3d_convergence_matches_oracle(method, k, pipeline):
    """Same stopping cycle, iterate and residual history as the oracle."""
    torch = _torch()
    p = W.random_bc_problem3d(40, 24, 18, seed=9, sigma_kind="const", asym=True)
    tol = 1e-8
    tile = (16, 4, 8)
    s = gpu_solver(p, method=method, tile_x=tile[0], tile_y=tile[1], tile_z=tile[2], k=k, precision="f64",
                   tol=tol, check_every=16, pipeline=pipeline, max_cycles=100000)
    u = to_dev(p.u0, 3, torch.float64)
    out = s.solve(to_dev(p.f, 3, torch.float64), u, history=100000)
    uo, c, status, hist = oracle.solve(p.st, p.f, p.u0, tol, 10 ** 7, tile[0], tile[1], k,
                                       classic=(method == "classic"), hist_cap=100000, tz=tile[2])
    assert status == 0 and out["status"] == 0
    assert out["cycles"] == c
    if method == "hier":
        assert (out["tile_x"], out["tile_y"], out["tile_z"]) == tile
    assert np.array_equal(to_host(u, 40), uo)
    np.testing.assert_allclose(np.array(out["history"]), hist[:c + 1], rtol=1e-9, atol=1e-12 * hist[0])
    s.close()


def test_f32_3d_cycles_close_to_oracle_and_solve_converges():
    torch = _torch()
    p = W.random_bc_problem3d(70, 33, 21, seed=23, sigma_kind="const", asym=True)
    for tile in _shapes("f32"):
        for pipeline in (0, 1):
            s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], tile_z=tile[2], k=6, precision="f32", fixed_cycles=4,
                           pipeline=pipeline)
            u = to_dev(p.u0, 3, torch.float32)
            s.solve(to_dev(p.f, 3, torch.float32), u)
            ref = oracle.run_fixed(p.st, p.f, p.u0, 4, tile[0], tile[1], 6, tz=tile[2])
            assert rel_max(to_host(u, 70), ref) <= 1e-5, (tile, pipeline)
            s.close()
    q = W.poisson3d_uniform(48, 40, 36, seed=3)
    s = gpu_solver(q, precision="f32", k=8, tol=1e-4, check_every=8, max_cycles=100000)
    u = to_dev(q.u0, 3, torch.float32)
    out = s.solve(to_dev(q.f, 3, torch.float32), u)
    assert out["status"] == 0 and (out["tile_x"], out["tile_y"], out["tile_z"]) == _shapes("f32")[0]
    r = oracle.residual(q.st, q.f, to_host(u, 48))
    assert r <= 1.01e-4 * oracle.residual(q.st, q.f, q.u0)
    s.close()


def test_3d_residual_api_matches_oracle():
    torch = _torch()
    p = W.random_bc_problem3d(29, 17, 12, seed=4, sigma_kind="const", asym=True)
    s = gpu_solver(p, precision="f64")
    a, r = s.residual(to_dev(p.f, 3, torch.float64), to_dev(p.u0, 3, torch.float64))
    ro = oracle.residual(p.st, p.f, p.u0)
    assert a == pytest.approx(ro, rel=1e-12)
    assert r == pytest.approx(ro / np.linalg.norm(W.interior(p.f, 3)), rel=1e-12)
    s.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 3), (17, 1, 2), (3, 2, 40)])
def test_3d_degenerate_grids(shape):
    torch = _torch()
    nx, ny, nz = shape
    p = W.random_bc_problem3d(nx, ny, nz, seed=8, sigma_kind="const")
    s = gpu_solver(p, precision="f64", k=4, fixed_cycles=3)
    u = to_dev(p.u0, 3, torch.float64)
    s.solve(to_dev(p.f, 3, torch.float64), u)
    t = _shapes("f64")[0]
    ref = oracle.run_fixed(p.st, p.f, p.u0, 3, t[0], t[1], 4, tz=t[2])
    assert np.array_equal(to_host(u, nx), ref)
    s.close()


def test_3d_host_pointer_solve_equals_device_solve():
    import paper_2006_16465_gb300 as hj
    torch = _torch()
    p = W.random_bc_problem3d(33, 20, 10, seed=12, sigma_kind="const", asym=True)
    s = gpu_solver(p, precision="f64", k=4, fixed_cycles=5)
    f = to_dev(p.f, 3, torch.float64)
    u = to_dev(p.u0, 3, torch.float64)
    s.solve(f, u)
    fh, uh = f.cpu(), to_dev(p.u0, 3, torch.float64).cpu()
    code = hj.hj_solve(s.h, fh.data_ptr(), uh.data_ptr(), 0, None)
    assert code == hj.HJ_OK
    assert torch.equal(uh, u.cpu())
    s.close()


# ---------------------------------------------------------------------------
# binary32 TMA-pipelined kernel (grids of at least 8 subdomains per SM with
# the automatic pipeline choice): one warp per CTA walks subdomains, the next
# one's boxes copied in while the current one sweeps.  It stages the same
# values (the copy engine's zero fill beyond the ghost shell for the one-warp
# kernel's checked loads) and runs the same sweep steps, so its iterates equal
# the one-warp kernel's bit for bit; both stay within 1e-5 of the oracle.
# ---------------------------------------------------------------------------

BIG3 = (200, 100, 60)   # 1,352 to 2,600 subdomains for the built binary32 shapes


@pytest.mark.parametrize("ctas_per_sm", [0, 1, 2])
def test_f32_3d_pipelined_walk_equals_one_warp_kernel_and_oracle(ctas_per_sm):
    """ctas_per_sm 1 and 2 make every CTA walk many subdomains (stage reuse,
    mbarrier phase flips, refills after the proxy fence); 0 = full residency."""
    torch = _torch()
    nx, ny, nz = BIG3
    p = W.random_bc_problem3d(nx, ny, nz, seed=31, sigma_kind="const", asym=True)
    shapes = _shapes("f32") if ctas_per_sm == 1 else _shapes("f32")[:1]
    for tile in shapes:
        outs = []
        for pipeline in (-1, 0):
            s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], tile_z=tile[2], k=5, precision="f32", fixed_cycles=3,
                           pipeline=pipeline, ctas_per_sm=ctas_per_sm)
            u = to_dev(p.u0, 3, torch.float32)
            out = s.solve(to_dev(p.f, 3, torch.float32), u)
            # every shape at least 16 wide has the pipelined kernel (8-wide boxes do not)
            want = 1 if (pipeline == -1 and tile[0] >= 16) else 0
            assert out["pipeline_stages"] == want, (tile, pipeline, out["pipeline_stages"])
            outs.append(to_host(u, nx))
            s.close()
        assert np.array_equal(outs[0], outs[1]), (tile, rel_max(outs[0], outs[1]))
        ref = oracle.run_fixed(p.st, p.f, p.u0, 3, tile[0], tile[1], 5, tz=tile[2])
        assert rel_max(outs[0], ref) <= 1e-5, (tile, rel_max(outs[0], ref))


def test_f32_3d_pipelined_converging_solve_equals_one_warp_kernel():
    """The deferred residual fold (one partial per CTA, folded by the next
    launch over three rotating iterate buffers) stops at the one-warp
    kernel's cycle with the same iterate; the oracle's residual of the
    returned iterate meets the tolerance."""
    torch = _torch()
    nx, ny, nz = BIG3
    q = W.poisson3d_uniform(nx, ny, nz, seed=5)
    res = []
    for pipeline in (-1, 0):
        s = gpu_solver(q, precision="f32", k=8, tol=1e-3, check_every=8, max_cycles=100000, pipeline=pipeline,
                       ctas_per_sm=2)
        u = to_dev(q.u0, 3, torch.float32)
        out = s.solve(to_dev(q.f, 3, torch.float32), u)
        assert out["status"] == 0
        res.append((out["cycles"], to_host(u, nx)))
        s.close()
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])
    r = oracle.residual(q.st, q.f, res[0][1])
    assert r <= 1.01e-3 * oracle.residual(q.st, q.f, q.u0)

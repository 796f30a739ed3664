"""GPU parity of the TMA-pipelined cycle kernel in its steady state: every CTA
walks many subdomains (Sections 3.3 and 4.1: one cycle stages each subdomain
with its halo, runs k subiterations, writes the interior back).

The pipelined kernel launches min(subdomains, CTAs per SM x SMs) CTAs, and
CTA b takes subdomains b, b + grid, b + 2 grid, ...  With many more
subdomains than CTAs, every CTA reuses its copy stages several times: the
mbarrier phase flips, a stage is refilled after the proxy fence, and the last
CTA (which also folds the previous launch's residual) has fewer subdomains
than the others.  These grids force that walk at 1 to 11 CTAs per SM.

Tolerances: binary64 bitwise against the oracle (same evaluation order, no
fused multiply-add); binary32 within 1e-5 relative (max norm) of the binary64
oracle at equal cycles.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import gpu_solver, rel_max, to_dev, to_host

pytestmark = pytest.mark.gpu

PIPE = dict(pipeline=1, persistent=0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _torch():
    import torch
    return torch


def _nsm():
    torch = _torch()
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _ntiles(nx, ny, tile):
    return ((nx + tile[0] - 1) // tile[0]) * ((ny + tile[1] - 1) // tile[1])


@pytest.mark.parametrize("ctas_per_sm", [1, 2])
@pytest.mark.parametrize("shape,tile,sigma,asym", [
    ((1000, 760), (32, 32), "field", True),    # ragged in x and y, 768 subdomains
    ((2048, 2048), (32, 32), "const", False),  # 4096 subdomains
    ((2048, 2048), (64, 64), "field", False),  # 1024 subdomains
])
def test_f64_tile_walk_bitwise_equals_oracle(shape, tile, sigma, asym, ctas_per_sm):
    torch = _torch()
    nx, ny = shape
    assert _ntiles(nx, ny, tile) >= 2 * ctas_per_sm * _nsm(), "the grid must make every CTA walk subdomains"
    p = W.random_bc_problem(2, nx, ny, seed=nx + 7 * ctas_per_sm, sigma_kind=sigma, asym=asym)
    f = to_dev(p.f, 2, torch.float64)
    for k, ncyc in [(1, 3), (4, 4), (9, 5)]:
        s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f64", fixed_cycles=ncyc,
                       ctas_per_sm=ctas_per_sm, **PIPE)
        u = to_dev(p.u0, 2, torch.float64)
        out = s.solve(f, u)
        assert out["pipeline_stages"] == 2 and out["ctas_per_sm"] == ctas_per_sm
        got = to_host(u, nx)
        ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile[0], tile[1], k)
        assert np.array_equal(got, ref), f"not bitwise: tile {tile} k={k} cycles={ncyc} rel {rel_max(got, ref):.3e}"
        s.close()


@pytest.mark.parametrize("launch,shape,tile,sigma", [
    # the bench's launch: one warp per 32x32 subdomain, one copy stage, 11 CTAs per SM
    ((32, 1, 11), (4100, 3000), (32, 32), "none"),
    ((32, 1, 11), (4100, 3000), (32, 32), "field"),
    ((32, 2, 2), (2000, 1500), (32, 32), "field"),
    ((64, 1, 3), (2000, 1500), (32, 32), "const"),
    ((0, 1, 2), (2048, 2048), (64, 64), "none"),
    ((0, 2, 1), (2048, 2048), (128, 32), "field"),
])
def test_f32_tile_walk_close_to_oracle(launch, shape, tile, sigma):
    torch = _torch()
    th, stages, cps = launch
    nx, ny = shape
    assert _ntiles(nx, ny, tile) >= 2 * cps * _nsm()
    p = W.random_bc_problem(2, nx, ny, seed=ny + stages, sigma_kind=sigma, asym=sigma != "none")
    k, ncyc = 4, 3
    s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f32", fixed_cycles=ncyc,
                   tile_threads=th, pipeline_stages=stages, ctas_per_sm=cps, **PIPE)
    u = to_dev(p.u0, 2, torch.float32)
    out = s.solve(to_dev(p.f, 2, torch.float32), u)
    assert out["pipeline_stages"] == stages and out["ctas_per_sm"] == cps
    got = to_host(u, nx)
    ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile[0], tile[1], k)
    assert rel_max(got, ref) <= 1e-5
    s.close()


@pytest.mark.parametrize("ctas_per_sm,check_every", [(1, 7), (2, 6)])
def test_f64_tile_walk_converging_solve_stops_with_the_oracle(ctas_per_sm, check_every):
    """Fused residual with the deferred fold while CTAs walk subdomains: the
    same stopping cycle, the same iterate (bitwise) and the same history."""
    torch = _torch()
    nx, ny = 1000, 760
    p = W.random_bc_problem(2, nx, ny, seed=21, sigma_kind="field", asym=True)
    tol = 1e-2
    s = gpu_solver(p, tile_x=32, tile_y=32, k=8, precision="f64", tol=tol, check_every=check_every,
                   ctas_per_sm=ctas_per_sm, **PIPE)
    u = to_dev(p.u0, 2, torch.float64)
    out = s.solve(to_dev(p.f, 2, torch.float64), u, history=100000)
    uo, c, status, hist = oracle.solve(p.st, p.f, p.u0, tol, 10 ** 5, 32, 32, 8, hist_cap=100000)
    assert status == 0 and out["status"] == 0 and out["persistent"] == 0
    assert c >= 10, "the solve must run many launches"
    assert out["cycles"] == c
    assert np.array_equal(to_host(u, nx), uo)
    gh = np.array(out["history"])
    assert len(gh) == c + 1
    np.testing.assert_allclose(gh, hist[:c + 1], rtol=1e-9, atol=1e-12 * hist[0])
    s.close()


def test_f32_tile_walk_converging_solve_at_the_bench_launch():
    """Binary32 solve with the bench's launch shape on a grid where every CTA
    walks subdomains: it meets the tolerance by the oracle's own residual and
    stops within 2 % of the oracle's cycle count."""
    torch = _torch()
    nx, ny = 4100, 3000
    p = W.random_bc_problem(2, nx, ny, seed=5, sigma_kind="none")
    tol = 0.05
    s = gpu_solver(p, tile_x=32, tile_y=32, k=4, precision="f32", tol=tol, check_every=12, tile_threads=32,
                   pipeline_stages=1, ctas_per_sm=11, **PIPE)
    u = to_dev(p.u0, 2, torch.float32)
    out = s.solve(to_dev(p.f, 2, torch.float32), u)
    assert out["status"] == 0
    _, c, status, _ = oracle.solve(p.st, p.f, p.u0, tol, 10 ** 5, 32, 32, 4)
    assert status == 0
    r0 = oracle.residual(p.st, p.f, p.u0)
    assert oracle.residual(p.st, p.f, to_host(u, nx)) <= tol * r0 * (1 + 1e-3)
    assert abs(out["cycles"] - c) <= max(1, 0.02 * c)
    s.close()

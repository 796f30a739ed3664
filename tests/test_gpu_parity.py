"""GPU parity: the CUDA path (called through the C ABI) against the CPU oracle
on the same seeded inputs.

Tolerances (written here; each follows from the arithmetic on both sides):
  * binary64 cycles use the oracle's evaluation order without fused
    multiply-add: max |u_gpu - u_oracle| <= 1e-12 max |u_oracle| at equal cycle
    counts (bitwise equality is expected and reported);
  * binary32 cycles: relative residual within 1e-5 of the oracle's, and
    u within 1e-5 (relative, max norm) of the binary64 oracle at equal cycles
    on small grids;
  * refinement: the returned u meets tol and matches the oracle's refinement
    result within kappa * tol.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import gpu_solver, rel_max, to_dev, to_host

pytestmark = pytest.mark.gpu

F64_TILES_2D = [(32, 32), (32, 16), (32, 8), (32, 64), (64, 32), (64, 64)]
F32_TILES_2D = [(32, 32), (32, 16), (32, 8), (32, 64), (64, 32), (64, 64), (128, 32), (128, 64)]
TILES_1D = [32, 64, 128, 256]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _torch():
    import torch
    return torch


# ---------------------------------------------------------------------------
# binary64 hierarchical cycles: equal cycle counts
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pipeline", [0, 1])
@pytest.mark.parametrize("tile", F64_TILES_2D)
@pytest.mark.parametrize("shape,sigma,asym", [((70, 45), "field", True), ((64, 64), "none", False),
                                               ((97, 130), "const", False)])
def test_f64_cycles_match_oracle_2d(tile, shape, sigma, asym, pipeline):
    """pipeline=1: TMA-staged kernel (CTAs walk tile lists); 0: one CTA per tile."""
    torch = _torch()
    nx, ny = shape
    p = W.random_bc_problem(2, nx, ny, seed=nx + ny, sigma_kind=sigma, asym=asym)
    for k, ncyc in [(1, 3), (5, 4), (16, 2)]:
        s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f64", fixed_cycles=ncyc,
                       pipeline=pipeline)
        f = to_dev(p.f, 2, torch.float64)
        u = to_dev(p.u0, 2, torch.float64)
        s.solve(f, u)
        got = to_host(u, nx)
        ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile[0], tile[1], k)
        assert rel_max(got, ref) <= 1e-12, (tile, k, ncyc)
        assert np.array_equal(got, ref), f"not bitwise for tile {tile} k={k}"
        s.close()


@pytest.mark.parametrize("threads", [0, 32])
@pytest.mark.parametrize("tile", TILES_1D)
@pytest.mark.parametrize("n,copies,sigma,asym", [(512, 1, "none", False), (300, 5, "field", True),
                                                   (1000, 3, "const", True)])
def test_f64_cycles_match_oracle_1d(tile, n, copies, sigma, asym, threads):
    """threads=0 splits each subdomain over the most warps built (fewer
    subdomains than SMs here); 32 gives every subdomain one warp."""
    torch = _torch()
    p = W.random_bc_problem(1, n, copies, seed=n, sigma_kind=sigma, asym=asym)
    for k, ncyc in [(1, 3), (32, 3)]:
        s = gpu_solver(p, tile_x=tile, k=k, precision="f64", fixed_cycles=ncyc, tile_threads=threads)
        f = to_dev(p.f, 1, torch.float64)
        u = to_dev(p.u0, 1, torch.float64)
        s.solve(f, u)
        got = to_host(u, n)
        ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile, 1, k)
        assert np.array_equal(got, ref), (tile, k)
        s.close()


@pytest.mark.parametrize("dim", [1, 2])
def test_f64_classic_sweeps_match_oracle(dim):
    torch = _torch()
    p = W.random_bc_problem(dim, 77, 41 if dim == 2 else 3, seed=5, sigma_kind="field", asym=True)
    s = gpu_solver(p, method="classic", precision="f64", fixed_cycles=9)
    f = to_dev(p.f, dim, torch.float64)
    u = to_dev(p.u0, dim, torch.float64)
    s.solve(f, u)
    ref = oracle.run_fixed(p.st, p.f, p.u0, 9, classic=True)
    assert np.array_equal(to_host(u, p.st.nx), ref)


@pytest.mark.parametrize("prec,shape,sigma", [("f64", (2000, 1500), "field"), ("f64", (1031, 97), "none"),
                                              ("f32", (4100, 3000), "field"), ("f32", (130, 7), "const")])
def test_classic_sweeps_on_large_ragged_grids(prec, shape, sigma):
    """The vectorised classic sweep walks many blocks per CTA (grid-stride),
    with ragged edges in x (vectors holding ghost and padding columns) and y:
    binary64 bitwise against the oracle, binary32 within 1e-5."""
    torch = _torch()
    nx, ny = shape
    p = W.random_bc_problem(2, nx, ny, seed=nx + 1, sigma_kind=sigma, asym=True)
    dt = torch.float64 if prec == "f64" else torch.float32
    s = gpu_solver(p, method="classic", precision=prec, fixed_cycles=4)
    u = to_dev(p.u0, 2, dt)
    s.solve(to_dev(p.f, 2, dt), u)
    got = to_host(u, nx)
    ref = oracle.run_fixed(p.st, p.f, p.u0, 4, classic=True)
    if prec == "f64":
        assert np.array_equal(got, ref)
    else:
        assert rel_max(got, ref) <= 1e-5
    # the ghost ring (Dirichlet data) is untouched
    ghost = p.u0.astype(np.float32).astype(np.float64) if prec == "f32" else p.u0
    for sl in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
        assert np.array_equal(got[sl], ghost[sl])
    s.close()


# ---------------------------------------------------------------------------
# converging solves: same stopping cycle, same iterate, same residual history
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("dim,shape,tile,k,method", [
    (2, (96, 80), (32, 32), 8, "hier"),
    (2, (70, 45), (32, 16), 4, "hier"),
    (2, (48, 48), (32, 32), 1, "classic"),
    (1, (512, 1), (128, 1), 32, "hier"),
    (1, (700, 4), (64, 1), 16, "hier"),
])
def test_f64_convergence_matches_oracle(dim, shape, tile, k, method, persistent):
    """persistent=1: one cooperative launch iterates all cycles (device-side
    grid barrier; for the classic method the grid-sync variant); 0: CUDA
    graphs of check_every launches."""
    torch = _torch()
    nx, ny = shape
    if dim == 1 and ny == 1:
        p = W.poisson1d_sine(nx, seed=0)
    else:
        p = W.random_bc_problem(dim, nx, ny, seed=7, sigma_kind="field")
    tol = 1e-6
    s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f64", tol=tol, check_every=16,
                   method=method, persistent=persistent)
    f = to_dev(p.f, dim, torch.float64)
    u = to_dev(p.u0, dim, torch.float64)
    out = s.solve(f, u, history=100000)
    assert out["persistent"] == persistent
    uo, c, status, hist = oracle.solve(p.st, p.f, p.u0, tol, 10 ** 7, tile[0], tile[1], k,
                                       classic=(method == "classic"), hist_cap=100000)
    assert status == 0 and out["status"] == 0
    assert out["cycles"] == c
    assert np.array_equal(to_host(u, nx), uo)
    gh = np.array(out["history"])
    assert len(gh) == c + 1
    np.testing.assert_allclose(gh, hist[:c + 1], rtol=1e-9, atol=1e-12 * hist[0])
    assert out["res_final"] == pytest.approx(hist[c], rel=1e-9)
    s.close()


# The TMA-pipelined kernel folds each launch's residual partials in the next
# launch and rotates three iterate buffers; these cases pin that control path
# (forced with pipeline=1, persistent=0) to the oracle's stopping rule.
PIPE = dict(pipeline=1, persistent=0)


@pytest.mark.parametrize("check_every", [16, 6, 7])
@pytest.mark.parametrize("shape,tile,k,sigma", [
    ((96, 80), (32, 32), 8, "field"),
    ((70, 45), (32, 16), 4, "const"),
    ((130, 97), (64, 32), 16, "none"),
])
def test_f64_pipelined_convergence_matches_oracle(shape, tile, k, sigma, check_every):
    torch = _torch()
    nx, ny = shape
    p = W.random_bc_problem(2, nx, ny, seed=nx + 3, sigma_kind=sigma)
    tol = 1e-6
    s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f64", tol=tol, check_every=check_every,
                   **PIPE)
    f = to_dev(p.f, 2, torch.float64)
    u = to_dev(p.u0, 2, torch.float64)
    out = s.solve(f, u, history=100000)
    assert out["persistent"] == 0
    uo, c, status, hist = oracle.solve(p.st, p.f, p.u0, tol, 10 ** 7, tile[0], tile[1], k, hist_cap=100000)
    assert status == 0 and out["status"] == 0
    assert out["cycles"] == c
    assert np.array_equal(to_host(u, nx), uo)
    gh = np.array(out["history"])
    assert len(gh) == c + 1
    np.testing.assert_allclose(gh, hist[:c + 1], rtol=1e-9, atol=1e-12 * hist[0])
    assert out["res_final"] == pytest.approx(hist[c], rel=1e-9)
    s.close()


@pytest.mark.parametrize("max_cycles", [1, 2, 5, 6, 7, 13])
def test_pipelined_cycle_cap_returns_last_iterate(max_cycles):
    torch = _torch()
    import paper_2006_16465_gb300 as hj
    p = W.random_bc_problem(2, 72, 66, seed=max_cycles, sigma_kind="field", asym=True)
    s = gpu_solver(p, tile_x=32, tile_y=32, k=3, precision="f64", tol=1e-14, max_cycles=max_cycles,
                   check_every=4, **PIPE)
    f = to_dev(p.f, 2, torch.float64)
    u = to_dev(p.u0, 2, torch.float64)
    out = s.solve(f, u, check=False, history=64)
    assert out["status"] == hj.HJ_ERR_NOT_CONVERGED and out["cycles"] == max_cycles
    ref = oracle.run_fixed(p.st, p.f, p.u0, max_cycles, 32, 32, 3)
    assert np.array_equal(to_host(u, 72), ref)
    assert out["res_final"] == pytest.approx(oracle.residual(p.st, p.f, ref), rel=1e-12)
    # every folded residual is in the history: ||r_0|| .. ||r_{max_cycles-1}||
    assert len(out["history"]) == max_cycles
    s.close()


def test_pipelined_zero_rhs_converges_at_cycle_zero_and_nan_diverges():
    torch = _torch()
    import paper_2006_16465_gb300 as hj
    p = W.poisson2d_uniform(64, 64, seed=3)
    s = gpu_solver(p, precision="f64", tol=1e-8, **PIPE)
    out = s.solve(to_dev(W.zeros_grid(p.st), 2, torch.float64), to_dev(W.zeros_grid(p.st), 2, torch.float64))
    assert out["status"] == 0 and out["cycles"] == 0 and out["res_final"] == 0.0
    fh = p.f.copy()
    fh[10, 10] = np.nan
    out = s.solve(to_dev(fh, 2, torch.float64), to_dev(p.u0, 2, torch.float64), check=False)
    assert out["status"] == hj.HJ_ERR_DIVERGED
    s.close()


def test_pipelined_reuse_with_new_boundary_values():
    """The third buffer takes each solve's ghost ring (Dirichlet data)."""
    torch = _torch()
    s = None
    for seed in (11, 12, 13):
        p = W.random_bc_problem(2, 80, 70, seed=seed, sigma_kind="none")
        if s is None:
            s = gpu_solver(p, tile_x=32, tile_y=32, k=4, precision="f64", tol=1e-7, check_every=12, **PIPE)
        u = to_dev(p.u0, 2, torch.float64)
        out = s.solve(to_dev(p.f, 2, torch.float64), u)
        uo, c, status, _ = oracle.solve(p.st, p.f, p.u0, 1e-7, 10 ** 7, 32, 32, 4)
        assert out["cycles"] == c and np.array_equal(to_host(u, 80), uo), seed
    s.close()


def test_f32_pipelined_solve_matches_graph_solve():
    """Binary32 with the pipelined kernel: same stopping cycle and iterate as
    the one-CTA-per-tile kernel (same arithmetic per point)."""
    torch = _torch()
    p = W.poisson2d_uniform(160, 128, seed=4)
    outs = []
    for eng in (PIPE, dict(pipeline=0, persistent=0)):
        s = gpu_solver(p, tile_x=32, tile_y=32, k=8, precision="f32", tol=1e-5, check_every=10, **eng)
        u = to_dev(p.u0, 2, torch.float32)
        out = s.solve(to_dev(p.f, 2, torch.float32), u, history=100000)
        assert out["status"] == 0
        outs.append((out, to_host(u, 160)))
        s.close()
    (a, ua), (b, ub) = outs
    assert a["cycles"] == b["cycles"]
    assert np.array_equal(ua, ub)
    np.testing.assert_allclose(a["history"], b["history"], rtol=1e-6)


def test_pipelined_launch_shapes_give_the_same_iterates():
    """Threads per subdomain, copy stages and CTAs per SM change the launch,
    not the arithmetic: every shape stops at the same cycle with the same
    iterate."""
    torch = _torch()
    p = W.random_bc_problem(2, 200, 170, seed=9, sigma_kind="field", asym=True)
    sig = to_dev(p.st.sigma, 2, torch.float64)
    import paper_2006_16465_gb300 as hj
    outs = []
    for th, stg, cps in [(32, 1, 0), (32, 2, 0), (64, 1, 3), (32, 1, 2), (64, 2, 1)]:
        s = hj.Solver(p.st, sigma=sig, tile_x=32, tile_y=32, k=6, precision="f32", tol=1e-5, check_every=10,
                      tile_threads=th, pipeline_stages=stg, ctas_per_sm=cps, **PIPE)
        u = to_dev(p.u0, 2, torch.float32)
        out = s.solve(to_dev(p.f, 2, torch.float32), u)
        assert out["status"] == 0 and out["pipeline_stages"] == stg and out["ctas_per_sm"] == cps
        outs.append((out["cycles"], to_host(u, 200)))
        s.close()
    for c, u in outs[1:]:
        assert c == outs[0][0]
        assert np.array_equal(u, outs[0][1])


def test_residual_api_matches_oracle():
    torch = _torch()
    for dim, nx, ny in [(2, 90, 70), (1, 333, 3)]:
        p = W.random_bc_problem(dim, nx, ny, seed=4, sigma_kind="field", asym=True)
        s = gpu_solver(p, precision="f64")
        f = to_dev(p.f, dim, torch.float64)
        u = to_dev(p.u0, dim, torch.float64)
        a, r = s.residual(f, u)
        ro = oracle.residual(p.st, p.f, p.u0)
        assert a == pytest.approx(ro, rel=1e-12)
        assert r == pytest.approx(ro / np.linalg.norm(W.interior(p.f, dim)), rel=1e-12)
        s.close()


def test_f32_residual_is_the_binary64_residual_of_the_stored_values():
    """Binary32 grids: the residual is formed in binary64 from the exact
    binary64 values of the stored binary32 numbers (converted by integer
    operations on the GPU, by the instruction for subnormals), so it equals
    the oracle's binary64 residual of the upcast arrays.  The grids carry
    signed zeros, subnormals and large values in the iterate, the RHS and the
    boundary ring (2D with a sigma field, 1D, 3D)."""
    torch = _torch()
    rng = np.random.default_rng(17)
    cases = [(2, W.random_bc_problem(2, 77, 53, seed=6, sigma_kind="field", asym=True), 77),
             (1, W.random_bc_problem(1, 301, 2, seed=7, sigma_kind="const", asym=True), 301),
             (3, W.random_bc_problem3d(23, 17, 11, seed=8, sigma_kind="const", asym=True), 23)]
    specials = np.array([0.0, -0.0, 1e-40, -3e-42, 1.4e-45, 3.0e38, -2.5e37, 1.17549435e-38], np.float32)
    for dim, p, nx in cases:
        f32 = p.f.astype(np.float32)
        u32 = p.u0.astype(np.float32)
        for a in (f32, u32):
            flat = a.reshape(-1)
            idx = rng.choice(flat.size, size=min(40, flat.size // 4), replace=False)
            flat[idx] = specials[rng.integers(0, specials.size, idx.size)]
        s = gpu_solver(p, precision="f32")
        got, _ = s.residual(to_dev(f32, dim, torch.float32), to_dev(u32, dim, torch.float32))
        ref = oracle.residual(p.st, f32.astype(np.float64), u32.astype(np.float64))
        assert np.isfinite(ref) and got == pytest.approx(ref, rel=1e-12), (dim, got, ref)
        s.close()


# ---------------------------------------------------------------------------
# binary32 cycles
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pipeline", [0, 1])
@pytest.mark.parametrize("tile", F32_TILES_2D)
def test_f32_cycles_close_to_oracle(tile, pipeline):
    torch = _torch()
    nx, ny = 150, 100
    p = W.random_bc_problem(2, nx, ny, seed=9, sigma_kind="none")
    ncyc, k = 20, 8
    s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f32", fixed_cycles=ncyc,
                   pipeline=pipeline)
    f = to_dev(p.f, 2, torch.float32)
    u = to_dev(p.u0, 2, torch.float32)
    s.solve(f, u)
    got = to_host(u, nx)
    ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile[0], tile[1], k)
    assert rel_max(got, ref) <= 1e-5
    r0 = oracle.residual(p.st, p.f, p.u0)
    assert abs(oracle.residual(p.st, p.f, got) - oracle.residual(p.st, p.f, ref)) / r0 <= 1e-5
    s.close()


@pytest.mark.parametrize("pipeline", [0, 1])
@pytest.mark.parametrize("sigma", ["field", "const"])
@pytest.mark.parametrize("dim", [1, 2])
def test_f32_screened_and_1d_close_to_oracle(dim, sigma, pipeline):
    torch = _torch()
    if dim == 1 and pipeline == 1:
        pytest.skip("the TMA pipeline is a 2D kernel")
    p = W.random_bc_problem(dim, 200, 60 if dim == 2 else 4, seed=12, sigma_kind=sigma, asym=True)
    s = gpu_solver(p, tile_x=32 if dim == 2 else 128, tile_y=32, k=6, precision="f32", fixed_cycles=15,
                   pipeline=pipeline)
    f = to_dev(p.f, dim, torch.float32)
    u = to_dev(p.u0, dim, torch.float32)
    s.solve(f, u)
    ref = oracle.run_fixed(p.st, p.f, p.u0, 15, 32 if dim == 2 else 128, 32, 6)
    assert rel_max(to_host(u, 200), ref) <= 1e-5
    s.close()


def test_f32_solve_reaches_tolerance_and_oracle_agrees():
    torch = _torch()
    p = W.poisson2d_uniform(128, 128, seed=1)
    s = gpu_solver(p, tile_x=32, tile_y=32, k=16, precision="f32", tol=1e-5, check_every=32)
    f = to_dev(p.f, 2, torch.float32)
    u = to_dev(p.u0, 2, torch.float32)
    out = s.solve(f, u, history=100000)
    assert out["status"] == 0
    uo, c, status, _ = oracle.solve(p.st, p.f, p.u0, 1e-5, 10 ** 6, 32, 32, 16)
    rel_gpu = oracle.residual(p.st, p.f, to_host(u, 128)) / oracle.residual(p.st, p.f, p.u0)
    rel_orc = oracle.residual(p.st, p.f, uo) / oracle.residual(p.st, p.f, p.u0)
    assert abs(rel_gpu - rel_orc) <= 1e-5
    assert abs(out["cycles"] - c) <= max(2, 0.02 * c)
    s.close()


# ---------------------------------------------------------------------------
# mixed-precision iterative refinement
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("engine", ["persistent", "graph", "pipeline"])
@pytest.mark.parametrize("prec", ["f32_ir", "bf16corr_ir"])
def test_refinement_reaches_tolerance_and_matches_oracle(prec, engine):
    torch = _torch()
    n = 96
    p = W.poisson2d_sin_noise(n, seed=2)
    tol = 1e-10
    inner_tol = 1e-4 if prec == "f32_ir" else 1e-2
    eng = {"persistent": dict(persistent=1, pipeline=0), "graph": dict(persistent=0, pipeline=0),
           "pipeline": dict(persistent=0, pipeline=1)}[engine]
    s = gpu_solver(p, tile_x=32, tile_y=32, k=16, precision=prec, tol=tol, inner_tol=inner_tol,
                   check_every=16, max_outer=60, **eng)
    f = to_dev(p.f, 2, torch.float64)
    u = to_dev(p.u0, 2, torch.float64)
    out = s.solve(f, u, history=64)
    assert out["status"] == 0
    r0 = oracle.residual(p.st, p.f, p.u0)
    ug = to_host(u, n)
    assert oracle.residual(p.st, p.f, ug) <= tol * r0 * 1.0001
    uo, outer, inner, status, hist = oracle.ir_solve(p.st, p.f, p.u0, tol, 32, 32, 16, inner_tol=inner_tol,
                                                     bf16=(prec == "bf16corr_ir"))
    assert status == 0
    h = 1 / (n + 1)
    kappa = (8 / h ** 2) / (2 * np.pi ** 2)
    assert np.abs(ug - uo).max() <= kappa * tol * np.abs(uo).max()
    # the step counts follow the oracle's refinement: the binary64 outer steps
    # are the same computation (within one step: the inner binary32 cycles fuse
    # multiply-adds on the GPU and do not in the oracle, so each inner solve
    # ends within a few cycles of the oracle's), and ||r_0|| is the same number
    assert out["outer_steps"] >= 2
    assert abs(out["outer_steps"] - outer) <= 1, (out["outer_steps"], outer)
    assert abs(out["inner_cycles"] - inner) <= 0.1 * inner + 32, (out["inner_cycles"], inner)
    assert out["history"][0] == pytest.approx(hist[0], rel=1e-12)
    s.close()


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32_ir", 1e-10)])
def test_adjoint_matches_oracle(prec, tol):
    torch = _torch()
    p = W.random_bc_problem(2, 80, 64, seed=21, sigma_kind="field", asym=True)
    st = p.st
    u_star, _, _, _ = oracle.solve(st, p.f, p.u0, 1e-13, 10 ** 7, 32, 32, 16)
    g = W.zeros_grid(st)
    g[1:-1, 1:-1] = W.uniform(5, 80 * 64, -1, 1).reshape(64, 80)
    s = gpu_solver(p, tile_x=32, tile_y=32, k=16, precision=prec, tol=tol, check_every=32)
    gd = to_dev(g, 2, torch.float64)
    ud = to_dev(u_star, 2, torch.float64)
    lam = to_dev(W.zeros_grid(st), 2, torch.float64)
    dsig = to_dev(W.zeros_grid(st), 2, torch.float64)
    out = s.adjoint(gd, ud, lam, dsig)
    assert out["status"] == 0
    lam_o, dsig_o, status = oracle.adjoint(st, g, u_star, tol=1e-13)
    assert status == 0
    L = to_host(lam, 80)
    assert rel_max(L, lam_o) <= 1e-6
    assert rel_max(to_host(dsig, 80), dsig_o) <= 1e-6
    assert np.all(L[0] == 0) and np.all(L[-1] == 0) and np.all(L[:, 0] == 0) and np.all(L[:, 81] == 0)
    s.close()


# ---------------------------------------------------------------------------
# interfaces and edge cases
# ---------------------------------------------------------------------------

def test_host_pointer_solve_equals_device_solve():
    torch = _torch()
    import paper_2006_16465_gb300 as hj
    p = W.random_bc_problem(2, 64, 40, seed=2)
    s = gpu_solver(p, tile_x=32, tile_y=32, k=4, precision="f64", fixed_cycles=6)
    f = to_dev(p.f, 2, torch.float64)
    u = to_dev(p.u0, 2, torch.float64)
    s.solve(f, u)
    fh = f.cpu().pin_memory()
    uh = to_dev(p.u0, 2, torch.float64).cpu()          # pageable host memory
    code = hj.hj_solve(s.h, fh.data_ptr(), uh.data_ptr(), 0, None)
    assert code == 0
    assert torch.equal(uh, u.cpu())
    s.close()


def test_zero_rhs_and_exact_guess_converge_at_cycle_zero():
    torch = _torch()
    p = W.poisson2d_uniform(40, 40, seed=3)
    f = to_dev(W.zeros_grid(p.st), 2, torch.float64)
    u = to_dev(W.zeros_grid(p.st), 2, torch.float64)
    s = gpu_solver(p, precision="f64", tol=1e-8)
    out = s.solve(f, u)
    assert out["status"] == 0 and out["cycles"] == 0 and out["res_final"] == 0.0
    s.close()


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (33, 1), (31, 33)])
def test_tiny_and_degenerate_grids(shape):
    torch = _torch()
    nx, ny = shape
    p = W.random_bc_problem(2, nx, ny, seed=nx * 10 + ny, sigma_kind="field")
    s = gpu_solver(p, tile_x=32, tile_y=32, k=3, precision="f64", fixed_cycles=5)
    f = to_dev(p.f, 2, torch.float64)
    u = to_dev(p.u0, 2, torch.float64)
    s.solve(f, u)
    assert np.array_equal(to_host(u, nx), oracle.run_fixed(p.st, p.f, p.u0, 5, 32, 32, 3))
    s.close()


def test_not_converged_returns_last_iterate():
    torch = _torch()
    import paper_2006_16465_gb300 as hj
    p = W.poisson2d_uniform(64, 64, seed=8)
    s = gpu_solver(p, precision="f64", tol=1e-12, max_cycles=13, check_every=4, k=2)
    f = to_dev(p.f, 2, torch.float64)
    u = to_dev(p.u0, 2, torch.float64)
    out = s.solve(f, u, check=False)
    assert out["status"] == hj.HJ_ERR_NOT_CONVERGED and out["cycles"] == 13
    ref = oracle.run_fixed(p.st, p.f, p.u0, 13, 32, 32, 2)
    assert np.array_equal(to_host(u, 64), ref)
    assert out["res_final"] == pytest.approx(oracle.residual(p.st, p.f, ref), rel=1e-12)
    s.close()


def test_nonfinite_rhs_reports_divergence():
    torch = _torch()
    import paper_2006_16465_gb300 as hj
    p = W.poisson2d_uniform(64, 64, seed=8)
    fh = p.f.copy()
    fh[10, 10] = np.nan
    s = gpu_solver(p, precision="f64", tol=1e-8)
    out = s.solve(to_dev(fh, 2, torch.float64), to_dev(p.u0, 2, torch.float64), check=False)
    assert out["status"] == hj.HJ_ERR_DIVERGED
    s.close()


def test_solver_reuse_and_graph_cache():
    torch = _torch()
    p = W.random_bc_problem(2, 100, 90, seed=31)
    s = gpu_solver(p, tile_x=32, tile_y=32, k=4, precision="f64", tol=1e-7, check_every=8)
    f = to_dev(p.f, 2, torch.float64)
    outs = []
    for _ in range(3):
        u = to_dev(p.u0, 2, torch.float64)
        outs.append((s.solve(f, u)["cycles"], to_host(u, 100)))
    assert outs[0][0] == outs[1][0] == outs[2][0]
    assert np.array_equal(outs[0][1], outs[2][1])
    s.close()


# ---------------------------------------------------------------------------
# batched persistent scheduler
# ---------------------------------------------------------------------------

def _batch(nprob=7, seed=11):
    sides = [64, 96, 128, 160]
    out = []
    for i in range(nprob):
        nx, ny = sides[i % 4], sides[(i * 3 + 1) % 4]
        st = W.poisson_stencil(2, nx, ny, sigma_const=float(W.uniform(seed, nprob, 0.0, 100.0)[i]))
        f = W.zeros_grid(st)
        f[1:-1, 1:-1] = W.uniform(seed * 100 + i, nx * ny, -1, 1).reshape(ny, nx)
        out.append(W.Problem(st, f, W.zeros_grid(st)))
    return out


@pytest.mark.parametrize("prec", ["f32_ir", "bf16corr_ir"])
def test_batched_equals_individual_solves_and_oracle(prec):
    torch = _torch()
    import paper_2006_16465_gb300 as hj
    probs = _batch()
    tol = 1e-8
    params = dict(tile_x=32, tile_y=32, k=16, precision=prec, tol=tol, inner_tol=1e-4, max_outer=60)
    # batched
    s = gpu_solver(probs[0], **params)
    fs = [to_dev(q.f, 2, torch.float64) for q in probs]
    us = [to_dev(q.u0, 2, torch.float64) for q in probs]
    descs = [hj.make_desc(2, q.st.nx, q.st.ny, f.shape[1], q.st.cW, q.st.cE, q.st.cS, q.st.cN, q.st.cD,
                          q.st.sigma_const) for q, f in zip(probs, fs)]
    cyc = (hj.C.c_longlong * len(probs))()
    code = hj.hj_solve_batched(s.h, descs, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], 0, None, cyc)
    assert code == 0, hj.hj_last_error()
    s.close()
    for i, q in enumerate(probs):
        # one problem alone through the same persistent engine: bitwise identical
        si = gpu_solver(q, persistent=1, **params)
        ui = to_dev(q.u0, 2, torch.float64)
        out = si.solve(to_dev(q.f, 2, torch.float64), ui)
        assert out["status"] == 0
        assert torch.equal(ui, us[i]), f"problem {i}"
        assert out["inner_cycles"] == cyc[i]
        si.close()
        ug = to_host(us[i], q.st.nx)
        r0 = oracle.residual(q.st, q.f, q.u0)
        assert oracle.residual(q.st, q.f, ug) <= tol * r0 * 1.0001
        uo, _, _, st, _ = oracle.ir_solve(q.st, q.f, q.u0, tol, 32, 32, 16, inner_tol=1e-4,
                                          bf16=(prec == "bf16corr_ir"))
        assert st == 0
        hx, hy = 1 / (q.st.nx + 1), 1 / (q.st.ny + 1)
        kappa = (4 / hx ** 2 + 4 / hy ** 2 + q.st.sigma_const) / (np.pi ** 2 * 2 + q.st.sigma_const)
        assert np.abs(ug - uo).max() <= 2 * kappa * tol * np.abs(uo).max()


@pytest.mark.parametrize("sigma", [False, True])
def test_batched_tma_staging_equals_plain_staging(sigma):
    """The persistent engine stages subdomains by TMA with prefetch unless
    pipeline = 0; both stagings give the same iterates and cycle counts."""
    torch = _torch()
    import paper_2006_16465_gb300 as hj
    probs = _batch()
    runs = []
    for pipeline in (-1, 0):
        params = dict(tile_x=32, tile_y=32, k=16, precision="f32_ir", tol=1e-8, inner_tol=1e-4, max_outer=60,
                      pipeline=pipeline)
        sig = None
        if sigma:
            q0 = probs[0]
            sg = W.zeros_grid(q0.st)
            sg[1:-1, 1:-1] = W.uniform(77, q0.st.nx * q0.st.ny, 0.0, 40.0).reshape(q0.st.ny, q0.st.nx)
            sig = to_dev(sg, 2, torch.float64)
        s = hj.Solver(probs[0].st, **params)
        fs = [to_dev(q.f, 2, torch.float64) for q in probs]
        us = [to_dev(q.u0, 2, torch.float64) for q in probs]
        descs = [hj.make_desc(2, q.st.nx, q.st.ny, f.shape[1], q.st.cW, q.st.cE, q.st.cS, q.st.cN, q.st.cD,
                              q.st.sigma_const, sig if (sigma and i == 0) else None)
                 for i, (q, f) in enumerate(zip(probs, fs))]
        cyc = (hj.C.c_longlong * len(probs))()
        code = hj.hj_solve_batched(s.h, descs, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], 0, None, cyc)
        assert code == 0, hj.hj_last_error()
        runs.append((us, list(cyc)))
        s.close()
    (ua, ca), (ub, cb) = runs
    assert ca == cb
    for i in range(len(probs)):
        assert torch.equal(ua[i], ub[i]), f"problem {i}"


_TIMEOUT_SCRIPT = r"""
import os, sys
sys.path.insert(0, os.getcwd())
os.environ["HJ_TEST_SKIP_BARRIER_CTA"] = "0"
os.environ["HJ_TEST_BARRIER_TIMEOUT_NS"] = "50000000"
import torch
import paper_2006_16465_gb300 as hj
import workloads as W
p = W.poisson2d_uniform(128, 128, seed=1)
s = hj.Solver(p.st, tile_x=32, tile_y=32, k=4, precision="f64", tol=1e-8, persistent=1)
out = s.solve(hj.grid_from(p.f, 2, torch.float64), hj.grid_from(p.u0, 2, torch.float64), check=False)
print("STATUS", out["status"], hj.hj_last_error())
s.close()
"""


def test_bounded_grid_barrier_reports_timeout():
    """One CTA of the persistent launch leaves before the grid barrier (test
    hook); the others give up after 50 ms and the call returns HJ_ERR_TIMEOUT
    instead of hanging.  Runs in a child process (the handle is unusable
    afterwards)."""
    import subprocess
    import sys
    import os
    import paper_2006_16465_gb300 as hj
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _TIMEOUT_SCRIPT], cwd=root, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("STATUS")][0]
    assert int(line.split()[1]) == hj.HJ_ERR_TIMEOUT, line


def test_batched_with_sigma_field_and_batched_adjoint_equal_single_calls():
    """Several right-hand sides sharing one per-point sigma field: the batched
    solve and the batched adjoint equal per-problem hj_solve / hj_solve_adjoint
    bitwise (same tile code, same refinement decisions), and dL/dsigma is the
    sum of the per-problem gradients."""
    torch = _torch()
    import paper_2006_16465_gb300 as hj
    nx, ny, B = 96, 80, 3
    sig = W.fourier_sigma(nx, seed=5)[: ny + 2, :]
    st = W.poisson_stencil(2, nx, ny, sigma=sig)
    fs = [to_dev(np.pad(W.uniform(60 + b, nx * ny, -1, 1).reshape(ny, nx), 1), 2, torch.float64) for b in range(B)]
    sg = to_dev(sig, 2, torch.float64)
    params = dict(tile_x=32, tile_y=32, k=16, precision="f32_ir", tol=1e-9, persistent=1)
    s = hj.Solver(st, sigma=sg, **params)
    us = [torch.zeros_like(f) for f in fs]
    code = hj.hj_solve_batched(s.h, [s.desc] * B, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], 0)
    assert code == 0, hj.hj_last_error()
    gs = [to_dev(np.pad(W.uniform(70 + b, nx * ny, -1, 1).reshape(ny, nx), 1), 2, torch.float64) for b in range(B)]
    lams = [torch.zeros_like(f) for f in fs]
    dsig = torch.zeros_like(fs[0])
    code = hj.hj_solve_adjoint_batched(s.h, [g.data_ptr() for g in gs], [u.data_ptr() for u in us],
                                       [l.data_ptr() for l in lams], dsig.data_ptr(), 0)
    assert code == 0, hj.hj_last_error()
    dsum = torch.zeros_like(dsig)
    for b in range(B):
        ub = torch.zeros_like(fs[b])
        out = s.solve(fs[b], ub)
        assert out["status"] == 0
        assert torch.equal(ub, us[b])
        lam = torch.zeros_like(ub)
        ds = torch.zeros_like(ub)
        s.adjoint(gs[b], ub, lam, ds)
        assert torch.equal(lam, lams[b])
        dsum += ds
    assert torch.equal(dsum, dsig)
    s.close()


# ---------------------------------------------------------------------------
# overlapping subdomains (Sections 3.4, 4.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("tile,ovl", [((32, 32), (2, 2)), ((32, 32), (4, 4)), ((32, 16), (6, 3)),
                                      ((64, 32), (10, 2)), ((32, 8), (4, 0))])
@pytest.mark.parametrize("shape,sigma,asym", [((97, 130), "field", True), ((70, 45), "const", False)])
def test_f64_overlap_cycles_match_oracle_2d(tile, ovl, shape, sigma, asym):
    torch = _torch()
    nx, ny = shape
    p = W.random_bc_problem(2, nx, ny, seed=nx + ovl[0], sigma_kind=sigma, asym=asym)
    for k, ncyc in [(1, 2), (5, 3), (16, 2)]:
        s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f64", fixed_cycles=ncyc,
                       overlap_x=ovl[0], overlap_y=ovl[1], persistent=0)
        u = to_dev(p.u0, 2, torch.float64)
        s.solve(to_dev(p.f, 2, torch.float64), u)
        ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile[0], tile[1], k, overlap=ovl)
        assert np.array_equal(to_host(u, nx), ref), (tile, ovl, k)
        s.close()


@pytest.mark.parametrize("tile,ovl,threads", [(32, 2, 0), (64, 4, 0), (128, 8, 0), (128, 4, 32), (256, 12, 0)])
def test_f64_overlap_cycles_match_oracle_1d(tile, ovl, threads):
    torch = _torch()
    p = W.random_bc_problem(1, 700, 3, seed=ovl, sigma_kind="field", asym=True)
    for k, ncyc in [(1, 2), (32, 3)]:
        s = gpu_solver(p, tile_x=tile, k=k, precision="f64", fixed_cycles=ncyc, overlap_x=ovl, tile_threads=threads,
                       persistent=0)
        u = to_dev(p.u0, 1, torch.float64)
        s.solve(to_dev(p.f, 1, torch.float64), u)
        ref = oracle.run_fixed(p.st, p.f, p.u0, ncyc, tile, 1, k, overlap=(ovl, 0))
        assert np.array_equal(to_host(u, 700), ref), (tile, ovl, k)
        s.close()


@pytest.mark.parametrize("dim,shape,tile,k,ovl", [(2, (96, 80), (32, 32), 16, (4, 4)),
                                                  (2, (130, 97), (32, 16), 8, (2, 6)),
                                                  (1, (1024, 1), (32, 1), 16, (4, 0))])
def test_f64_overlap_convergence_matches_oracle(dim, shape, tile, k, ovl):
    """Same stopping cycle, iterate and residual history as the oracle; the
    1D case is the Section 3.5 problem (one copy) at k = 16, o = 4."""
    torch = _torch()
    nx, ny = shape
    if dim == 1:
        p = W.paper_replica(1, 1024, copies=1)
        tol = 1e-4
    else:
        p = W.random_bc_problem(2, nx, ny, seed=17, sigma_kind="field")
        tol = 1e-6
    s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=k, precision="f64", tol=tol, check_every=32,
                   overlap_x=ovl[0], overlap_y=ovl[1])
    u = to_dev(p.u0, dim, torch.float64)
    out = s.solve(to_dev(p.f, dim, torch.float64), u, history=100000)
    uo, c, status, hist = oracle.solve(p.st, p.f, p.u0, tol, 10 ** 7, tile[0], tile[1], k, hist_cap=100000,
                                       overlap=ovl)
    assert status == 0 and out["status"] == 0 and out["persistent"] == 0
    assert out["cycles"] == c
    if dim == 1:
        assert c == 8093
    assert np.array_equal(to_host(u, nx), uo)
    np.testing.assert_allclose(np.array(out["history"]), hist[:c + 1], rtol=1e-9, atol=1e-12 * hist[0])
    s.close()


def test_f32_overlap_cycles_close_to_oracle_and_refinement_converges():
    torch = _torch()
    p = W.random_bc_problem(2, 150, 120, seed=23, sigma_kind="field", asym=True)
    for tile, ovl in [((32, 32), (4, 4)), ((64, 64), (8, 6)), ((32, 16), (2, 2))]:
        s = gpu_solver(p, tile_x=tile[0], tile_y=tile[1], k=8, precision="f32", fixed_cycles=6,
                       overlap_x=ovl[0], overlap_y=ovl[1])
        u = to_dev(p.u0, 2, torch.float32)
        s.solve(to_dev(p.f, 2, torch.float32), u)
        ref = oracle.run_fixed(p.st, p.f, p.u0, 6, tile[0], tile[1], 8, overlap=ovl)
        assert rel_max(to_host(u, 150), ref) <= 1e-5, (tile, ovl)
        s.close()
    q = W.poisson2d_sin_noise(96, seed=2)
    s = gpu_solver(q, tile_x=32, tile_y=32, k=16, precision="f32_ir", tol=1e-10, inner_tol=1e-4, overlap_x=4,
                   overlap_y=4)
    u = to_dev(q.u0, 2, torch.float64)
    out = s.solve(to_dev(q.f, 2, torch.float64), u)
    assert out["status"] == 0
    assert oracle.residual(q.st, q.f, to_host(u, 96)) <= 1e-10 * oracle.residual(q.st, q.f, q.u0) * 1.0001
    s.close()


def test_overlap_is_rejected_where_unsupported():
    import paper_2006_16465_gb300 as hj
    p = W.poisson2d_uniform(64, 64, seed=1)
    for kw, code in [(dict(overlap_x=32), hj.HJ_ERR_INVALID_ARG), (dict(overlap_x=4, persistent=1), hj.HJ_ERR_UNSUPPORTED),
                     (dict(overlap_x=4, pipeline=1), hj.HJ_ERR_UNSUPPORTED),
                     (dict(overlap_x=4, method="classic"), hj.HJ_ERR_INVALID_ARG),
                     (dict(overlap_x=-2), hj.HJ_ERR_INVALID_ARG)]:
        with pytest.raises(hj.HJError) as e:
            gpu_solver(p, tile_x=32, tile_y=32, precision="f64", **kw)
        assert e.value.code == code, kw


# ---------------------------------------------------------------------------
# in-place variant (one global array, as the listing of Appendix A)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("engine", ["graph", "persistent", "pipeline"])
def test_in_place_converges_to_the_solution(engine):
    """Scheduling decides which halo values a subdomain sees, so only what is
    unique is compared: the converged solution (within kappa * tol of the
    oracle's) and the exact residual of the returned array."""
    torch = _torch()
    eng = {"graph": dict(persistent=0, pipeline=0), "persistent": dict(persistent=1, pipeline=0),
           "pipeline": dict(persistent=0, pipeline=1)}[engine]
    p = W.random_bc_problem(2, 96, 80, seed=41, sigma_kind="field")
    tol = 1e-8
    s = gpu_solver(p, tile_x=32, tile_y=32, k=8, precision="f64", tol=tol, check_every=16, in_place=1, **eng)
    u = to_dev(p.u0, 2, torch.float64)
    out = s.solve(to_dev(p.f, 2, torch.float64), u)
    assert out["status"] == 0
    ug = to_host(u, 96)
    r0 = oracle.residual(p.st, p.f, p.u0)
    assert oracle.residual(p.st, p.f, ug) <= tol * r0 * 1.0001
    assert out["res_final"] == pytest.approx(oracle.residual(p.st, p.f, ug), rel=1e-9)
    uo, c, st, _ = oracle.solve(p.st, p.f, p.u0, tol, 10 ** 7, 32, 32, 8)
    assert st == 0
    h = 1 / 97
    kappa = (8 / h ** 2) / (2 * np.pi ** 2)
    assert np.abs(ug - uo).max() <= 2 * kappa * tol * np.abs(uo).max()
    assert out["cycles"] <= 1.3 * c
    s.close()


def test_in_place_binary32_status_uses_exact_residuals():
    """The section 4.2 problem from x0 = 1: the first cycle's staged data in
    place is not u_0 alone, so the initial residual is taken exactly."""
    torch = _torch()
    p = W.paper_replica(2, 256, copies=1)
    s = gpu_solver(p, tile_x=32, tile_y=32, k=4, precision="f32", tol=1e-4, in_place=1)
    u = to_dev(p.u0, 2, torch.float32)
    out = s.solve(to_dev(p.f, 2, torch.float32), u)
    assert out["status"] == 0
    ug = to_host(u, 256)
    assert out["res0"] == pytest.approx(oracle.residual(p.st, p.f, p.u0), rel=1e-6)
    # the returned array may be one cycle past the checked iterate, and the
    # binary32 fused residual differs from the exact one in the 5th digit
    assert oracle.residual(p.st, p.f, ug) <= 1e-4 * out["res0"] * 1.01
    assert out["res_final"] == pytest.approx(oracle.residual(p.st, p.f, ug), rel=1e-6)
    s.close()


def test_in_place_refinement_and_1d():
    torch = _torch()
    q = W.poisson2d_sin_noise(96, seed=2)
    s = gpu_solver(q, tile_x=32, tile_y=32, k=16, precision="f32_ir", tol=1e-10, inner_tol=1e-4, in_place=1)
    u = to_dev(q.u0, 2, torch.float64)
    out = s.solve(to_dev(q.f, 2, torch.float64), u)
    assert out["status"] == 0
    assert oracle.residual(q.st, q.f, to_host(u, 96)) <= 1e-10 * oracle.residual(q.st, q.f, q.u0) * 1.0001
    s.close()
    p = W.poisson1d_sine(512, seed=0)
    s = gpu_solver(p, tile_x=128, k=32, precision="f64", tol=1e-6, in_place=1)
    u = to_dev(p.u0, 1, torch.float64)
    out = s.solve(to_dev(p.f, 1, torch.float64), u)
    assert out["status"] == 0
    assert oracle.residual(p.st, p.f, to_host(u, 512)) <= 1e-6 * oracle.residual(p.st, p.f, p.u0) * 1.0001
    s.close()


def test_one_call_solve_equals_solver():
    """hj.solve (create, solve, destroy) gives the Solver's iterate."""
    import paper_2006_16465_gb300 as hj
    torch = _torch()
    p = W.random_bc_problem(2, 70, 45, seed=31, sigma_kind="const", asym=True)
    f = to_dev(p.f, 2, torch.float64)
    u1 = to_dev(p.u0, 2, torch.float64)
    out = hj.solve(p.st, f, u1, precision="f64", tile_x=32, tile_y=32, k=8, tol=1e-9, max_cycles=100000)
    s = gpu_solver(p, precision="f64", tile_x=32, tile_y=32, k=8, tol=1e-9, max_cycles=100000)
    u2 = to_dev(p.u0, 2, torch.float64)
    out2 = s.solve(f, u2)
    s.close()
    assert out["status"] == 0 and out["cycles"] == out2["cycles"]
    assert torch.equal(u1, u2)


def test_batched_steps_replay_one_graph_and_log_batch_cycles():
    """The batched scheduler runs every refinement step as a replay of one
    captured graph, feeds the persistent launch from the device work queue
    (the results equal per-problem solves, test above) and records each
    batch cycle's duration with the interior points still active in it."""
    torch = _torch()
    import ctypes as C
    import paper_2006_16465_gb300 as hj
    probs = _batch()
    s = gpu_solver(probs[0], tile_x=32, tile_y=32, k=16, precision="f32_ir", tol=1e-8, inner_tol=1e-4)
    fs = [to_dev(q.f, 2, torch.float64) for q in probs]
    us = [to_dev(q.u0, 2, torch.float64) for q in probs]
    descs = [hj.make_desc(2, q.st.nx, q.st.ny, f.shape[1], q.st.cW, q.st.cE, q.st.cS, q.st.cN, q.st.cD,
                          q.st.sigma_const) for q, f in zip(probs, fs)]
    cap = 1 << 16
    ms = (C.c_double * cap)()
    pts = (C.c_longlong * cap)()
    st = hj.hj_stats()
    st.cycle_ms = C.cast(ms, C.POINTER(C.c_double))
    st.cycle_points = C.cast(pts, C.POINTER(C.c_longlong))
    st.cycle_cap = cap
    cyc = (C.c_longlong * len(probs))()
    code = hj.hj_solve_batched(s.h, descs, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], 0, st, cyc)
    assert code == 0, hj.hj_last_error()
    assert st.graphed == 1
    n = st.cycle_len
    sizes = [q.st.nx * q.st.ny for q in probs]
    # one entry per batch cycle: as many as the longest problem's inner cycles
    # in every refinement step together, at least as many as any one problem's
    assert max(cyc) <= n <= sum(cyc)
    assert pts[0] == sum(sizes)
    assert all(0 < pts[i] <= sum(sizes) for i in range(n))
    assert all(ms[i] > 0 for i in range(n))
    # the active points only shrink within a step and start afresh with the next
    drops = sum(1 for i in range(1, n) if pts[i] < pts[i - 1])
    assert drops >= 1
    s.close()


@pytest.mark.parametrize("prec", ["f32", "bf16corr_ir"])
def test_every_threads_variant_gives_the_same_iterates(prec):
    """A subdomain swept by one, two, four or eight warps (band edges through
    shared memory) computes the same values: every built (tile, threads)
    variant equals the default one bit for bit, in graph launches (with and
    without overlapping subdomains) and in the persistent engine's solve.
    (Binary64 builds one threads variant per 2D shape; the bfloat16-stored
    correction family shares the binary32 kernels' shapes and is run here in
    its refinement.)"""
    torch = _torch()
    import paper_2006_16465_gb300 as hj
    dt = torch.float32 if prec == "f32" else torch.float64
    shapes = {}
    for tx, ty, th in hj.hj_tile_variants(2, hj.PRECISIONS[prec]):
        shapes.setdefault((tx, ty), []).append(th)
    checked = 0
    for (tx, ty), threads in shapes.items():
        if len(threads) < 2:
            continue
        p = W.random_bc_problem(2, 150, 97, seed=tx + ty, sigma_kind="field", asym=True)
        if prec != "f32":
            # refinement: binary64 iterate, inner cycles on bfloat16-stored corrections
            outs = []
            for th in threads:
                s = gpu_solver(p, tile_x=tx, tile_y=ty, k=6, precision=prec, tol=1e-8, inner_tol=1e-2,
                               tile_threads=th, persistent=1, pipeline=0)
                u = to_dev(p.u0, 2, dt)
                out = s.solve(to_dev(p.f, 2, dt), u)
                assert out["status"] == 0
                outs.append((out["inner_cycles"], to_host(u, 150)))
                s.close()
            for th, (c, u) in zip(threads[1:], outs[1:]):
                assert c == outs[0][0] and np.array_equal(u, outs[0][1]), (tx, ty, th)
            checked += 1
            continue
        for extra in (dict(), dict(overlap_x=4, overlap_y=2)):
            outs = []
            for th in threads:
                s = gpu_solver(p, tile_x=tx, tile_y=ty, k=5, precision=prec, fixed_cycles=4, tile_threads=th,
                               pipeline=0, **extra)
                u = to_dev(p.u0, 2, dt)
                s.solve(to_dev(p.f, 2, dt), u)
                outs.append(to_host(u, 150))
                s.close()
            for th, o in zip(threads[1:], outs[1:]):
                assert np.array_equal(o, outs[0]), (tx, ty, th, extra)
        sols = []
        for th in threads:
            s = gpu_solver(p, tile_x=tx, tile_y=ty, k=6, precision=prec, tol=1e-5, check_every=8, tile_threads=th,
                           persistent=1, pipeline=0)
            u = to_dev(p.u0, 2, dt)
            out = s.solve(to_dev(p.f, 2, dt), u)
            assert out["status"] == 0 and out["persistent"] == 1
            sols.append((out["cycles"], to_host(u, 150)))
            s.close()
        for th, (c, u) in zip(threads[1:], sols[1:]):
            assert c == sols[0][0] and np.array_equal(u, sols[0][1]), (tx, ty, th)
        checked += 1
    assert checked >= 1

"""Implicit-adjoint autograd (HJSolve) against the oracle's adjoint and
against central finite differences of the same GPU solve."""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32_ir", 1e-11)])
def test_autograd_matches_oracle_adjoint(prec, tol):
    import torch
    import paper_2006_16465_gb300 as hj
    from paper_2006_16465_gb300.autograd import solve_screened
    nx, ny, B = 72, 56, 3
    sig = W.fourier_sigma(nx, seed=5)[: ny + 2, :]           # a (ny+2, nx+2) slice of the field
    st = W.poisson_stencil(2, nx, ny, sigma=sig)
    fs = [W.uniform(40 + b, nx * ny, -1, 1).reshape(ny, nx) for b in range(B)]
    ustar = W.uniform(99, nx * ny, -1, 1).reshape(ny, nx) * 1e-3
    f = torch.stack([to_dev(np.pad(x, 1), 2, torch.float64) for x in fs]).requires_grad_(True)
    sigma = to_dev(sig, 2, torch.float64).requires_grad_(True)
    target = to_dev(np.pad(ustar, 1), 2, torch.float64)
    u = solve_screened(f, sigma, st, tile_x=32, tile_y=32, k=16, precision=prec, tol=tol)
    loss = 0.5 * ((u - target)[:, 1:ny + 1, 1:nx + 1] ** 2).sum()
    loss.backward()
    dsig_o = np.zeros((ny + 2, nx + 2))
    for b in range(B):
        fo = np.pad(fs[b], 1)
        uo, _, status, _ = oracle.solve(st, fo, np.zeros_like(fo), 1e-13, 10 ** 7, 32, 32, 16)
        assert status == 0
        g = np.zeros_like(fo)
        g[1:-1, 1:-1] = uo[1:-1, 1:-1] - ustar
        lam, ds, status = oracle.adjoint(st, g, uo, tol=1e-13)
        assert status == 0
        got = to_host(f.grad[b], nx)
        assert np.abs(got - lam).max() <= 1e-6 * np.abs(lam).max()
        dsig_o += ds
    got = to_host(sigma.grad, nx)
    assert np.abs(got[1:-1, 1:-1] - dsig_o[1:-1, 1:-1]).max() <= 1e-6 * np.abs(dsig_o).max()


def test_autograd_matches_finite_differences():
    """Central differences of the GPU solve itself (binary64, tight tol)."""
    import torch
    from paper_2006_16465_gb300.autograd import solve_screened
    nx = ny = 48
    sig = W.fourier_sigma(nx, seed=6)
    st = W.poisson_stencil(2, nx, ny, sigma=sig)
    f = to_dev(np.pad(W.uniform(7, nx * ny, -1, 1).reshape(ny, nx), 1), 2, torch.float64)
    target = to_dev(np.pad(W.uniform(8, nx * ny, -1, 1).reshape(ny, nx) * 1e-3, 1), 2, torch.float64)
    params = dict(tile_x=32, tile_y=32, k=16, precision="f64", tol=1e-13)

    def loss_of(sig_np):
        s = to_dev(sig_np, 2, torch.float64)
        u = solve_screened(f, s, W.poisson_stencil(2, nx, ny, sigma=sig_np), **params)
        return float(0.5 * ((u - target)[1:ny + 1, 1:nx + 1] ** 2).sum())

    sigma = to_dev(sig, 2, torch.float64).requires_grad_(True)
    u = solve_screened(f, sigma, st, **params)
    loss = 0.5 * ((u - target)[1:ny + 1, 1:nx + 1] ** 2).sum()
    loss.backward()
    grad = to_host(sigma.grad, nx)
    # interior points (near the Dirichlet ring the gradient is ~1e-13, below
    # what differences of two tolerance-limited solves resolve); relative step
    # 1e-2 (a dense-solve dry run gives <= 1e-8 relative truncation error here)
    for (j, i) in [(20, 30), (10, 40), (30, 12), (25, 25)]:
        eps = 1e-2 * sig[j, i]
        sp = sig.copy(); sp[j, i] += eps
        sm = sig.copy(); sm[j, i] -= eps
        fd = (loss_of(sp) - loss_of(sm)) / (2 * eps)
        assert grad[j, i] == pytest.approx(fd, rel=1e-4, abs=1e-14)


def test_central_differences_at_many_entries_agree_with_the_adjoint():
    """The differentiation workload's recipe at 256^2: central differences of
    L(sigma) with a relative step of 1e-6 at 8 random entries (perturbed
    solutions u + du, du the warm-started correction solved to 1e-9) against
    the implicit-adjoint gradient: within 1e-5 relative."""
    import sys
    import torch
    import paper_2006_16465_gb300 as hj
    sys.path.insert(0, str(__import__("pathlib").Path(__file__).resolve().parents[1]))
    import bench
    r = bench.fd_check(torch, hj, W, n=256, entries=8)
    assert r["status"] == 0, r
    assert r["max_rel_err"] <= 1e-5, (r["max_rel_err"], r["fd"], r["adjoint"])

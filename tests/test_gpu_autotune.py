"""Autotuner: picks a built tile shape and a k from the candidate set by
measurement, caches the choice (per process and in a file), and the handle
created with autotune=1 solves to tolerance."""
import os
import subprocess
import sys

import pytest

import workloads as W
from helpers import gpu_solver, to_dev

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_autotune_picks_a_built_configuration_and_caches_it():
    import paper_2006_16465_gb300 as hj
    st = W.poisson_stencil(2, 192, 160)
    d = hj.make_desc(2, 192, 160, hj.padded_ld(192, None), st.cW, st.cE, st.cS, st.cN, st.cD, dtype=hj.HJ_F32)
    p = hj.make_params(precision="f32", tol=1e-5)
    ms = hj.hj_autotune(d, p)
    assert ms > 0
    assert (p.tile_x, p.tile_y) in hj.hj_tile_shapes(2, hj.HJ_PREC_F32)
    assert p.k in (4, 8, 16, 32, 64)
    assert p.overlap_x in (0, 2, 4, 8) and p.overlap_y == p.overlap_x and 2 * p.overlap_x < min(p.tile_x, p.tile_y)
    q = hj.make_params(precision="f32", tol=1e-5)
    assert hj.hj_autotune(d, q) == -1.0          # cache hit
    assert (q.tile_x, q.tile_y, q.k, q.overlap_x) == (p.tile_x, p.tile_y, p.k, p.overlap_x)


def test_autotuned_handle_solves_to_tolerance():
    import torch
    p = W.poisson2d_uniform(256, 200, seed=3)
    s = gpu_solver(p, precision="f32_ir", tol=1e-8, autotune=1)
    u = to_dev(p.u0, 2, torch.float64)
    out = s.solve(to_dev(p.f, 2, torch.float64), u)
    assert out["status"] == 0 and out["rel_final"] <= 1e-8
    s.close()


_CACHE_SCRIPT = r"""
import os, sys
sys.path.insert(0, os.getcwd())
import paper_2006_16465_gb300 as hj
import workloads as W
st = W.poisson_stencil(2, 128, 96, sigma_const=5.0)
d = hj.make_desc(2, 128, 96, hj.padded_ld(128, None), st.cW, st.cE, st.cS, st.cN, st.cD, 5.0, dtype=hj.HJ_F32)
p = hj.make_params(precision="f32", tol=1e-5)
ms = hj.hj_autotune(d, p)
print("RESULT", ms, p.tile_x, p.tile_y, p.k)
"""


def test_autotune_cache_file_persists_across_processes(tmp_path):
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, HJ_AUTOTUNE_CACHE=str(cache))
    outs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _CACHE_SCRIPT], cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stderr
        outs.append([ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")][0].split())
    assert float(outs[0][1]) > 0 and float(outs[1][1]) == -1.0
    assert outs[0][2:] == outs[1][2:]
    assert cache.read_text().count("\n") == 1


def test_batched_autotune_converges():
    import torch
    import paper_2006_16465_gb300 as hj
    probs = W.batched_screened(6, seed=9)
    s = gpu_solver(probs[0], tile_x=32, tile_y=32, k=16, precision="f32_ir", tol=1e-8, autotune=1)
    fs = [to_dev(q.f, 2, torch.float64) for q in probs]
    us = [to_dev(q.u0, 2, torch.float64) for q in probs]
    descs = [hj.make_desc(2, q.st.nx, q.st.ny, f.shape[1], q.st.cW, q.st.cE, q.st.cS, q.st.cN, q.st.cD,
                          q.st.sigma_const) for q, f in zip(probs, fs)]
    st = hj.hj_stats()
    code = hj.hj_solve_batched(s.h, descs, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], 0, st)
    assert code == 0, hj.hj_last_error()
    assert st.rel_final <= 1e-8
    for q, f, u in zip(probs, fs, us):
        a = hj.Solver(q.st, precision="f64")
        _, rel = a.residual(f, u)
        assert rel <= 1e-8 * 1.0001
        a.close()
    s.close()


def test_launch_tuning_keeps_subdomain_and_k_and_the_iterates():
    """autotune = 3 measures the pipelined kernel's launch shapes (threads per
    subdomain, copy stages, CTAs per SM) and keeps tile and k; the arithmetic
    per point is the same in every launch shape, so the iterates are too."""
    import numpy as np
    import torch
    p = W.poisson2d_uniform(640, 512, seed=5)
    base = dict(tile_x=32, tile_y=32, k=4, precision="f32", tol=1e-5, check_every=12, pipeline=1, persistent=0)
    outs = []
    for extra in ({}, {"autotune": 3}):
        s = gpu_solver(p, **base, **extra)
        u = to_dev(p.u0, 2, torch.float32)
        out = s.solve(to_dev(p.f, 2, torch.float32), u)
        outs.append((out, u.cpu().numpy()))
        s.close()
    (a, ua), (b, ub) = outs
    assert a["status"] == 0 and b["status"] == 0
    assert (b["tile_x"], b["tile_y"], b["k"]) == (32, 32, 4)
    assert b["pipeline_stages"] in (1, 2) and b["tile_threads"] in (32, 64) and b["ctas_per_sm"] >= 0
    assert a["pipeline_stages"] == 1 and a["ctas_per_sm"] == 0
    assert a["cycles"] == b["cycles"]
    assert np.array_equal(ua, ub)

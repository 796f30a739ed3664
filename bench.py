"""Benchmark of the hierarchical Jacobi hot path on GB300.

Workload (one step): 2D Poisson -Lap u = f on the unit square, 8192 x 8192
interior grid, zero Dirichlet data, f ~ U[-1,1] (seeded), binary32, 32 x 32
subdomains, k subiterations, 1000 hierarchical cycles with the fused residual
reduction and device-side convergence control on (tol = 0, so every cycle
runs).  Arrays are 270 MB each, larger than the 129 MB L2, so every cycle
streams from HBM (no flush needed).

value  = inner lattice-update rate, GLUP/s = 8192^2 * k * cycles / time
         (every Jacobi point update counts, as in stencil practice);
roofline = the cycle kernel against measured HBM copy bandwidth: algorithmic
         traffic 12 B per point per cycle (read u, read f, write u); the
         measured DRAM traffic comes from the committed ncu record while the
         kernel's sources are unchanged;
The pipelined kernel's launch shape (threads per subdomain, copy stages,
CTAs per SM) is measured when the solver is created (autotune = 3) and
reported in config.launch; --launch pins it instead.
e2e    = the same metric through hj_solve with HOST buffers (f, u copied in
         and u copied out inside the call, every step).
Also reported beside it: plain global-memory Jacobi on the same grid, and the
time to a 1e-8 relative residual on the 512 x 512 problem (binary32 inner
cycles with binary64 refinement) against global-memory Jacobi in binary64.

N > 1 GPUs: the path runs one problem per GPU (replicas only, no data-path
collective); value is the aggregate over ranks, timed max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D Poisson time-to-1e-8 residual, GLUP/s vs global-mem Jacobi; % HBM roofline"
N_BENCH = 8192
BYTES_PER_POINT_CYCLE = 12  # read u, read f, write u (binary32)
EXTRAS_OUT = os.path.join(ROOT, "bench_extras.json")   # full record of the extra legs (not tracked)


def _r(x, digits=4):
    """x rounded to a few significant digits (keeps the JSON line short)."""
    if isinstance(x, float) and math.isfinite(x) and x != 0.0:
        return float(f"{x:.{digits}g}")
    return x


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def host_rel_residual(st, f, u) -> float:
    """||f - A u|| / ||f|| over interior points, recomputed on the host in
    binary64 numpy (constant five-point stencil, ghost ring = Dirichlet data;
    with u0 = 0 this is the solver's relative residual)."""
    import numpy as np
    f = np.asarray(f, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    au = (st.cD + st.sigma_const) * u[1:-1, 1:-1] + st.cW * u[1:-1, :-2] + st.cE * u[1:-1, 2:] \
        + st.cS * u[:-2, 1:-1] + st.cN * u[2:, 1:-1]
    r = f[1:-1, 1:-1] - au
    return float(np.linalg.norm(r) / np.linalg.norm(f[1:-1, 1:-1]))


def dst_solution(st, f):
    """The exact solution of the discrete 2D Poisson system (constant
    stencil, zero Dirichlet data) by the type-I sine transform, which
    diagonalises the five-point operator."""
    import numpy as np
    import scipy.fft
    nx, ny = st.nx, st.ny
    p = np.arange(1, nx + 1)
    q = np.arange(1, ny + 1)
    lam = (st.cD + st.sigma_const) + 2 * st.cW * np.cos(np.pi * p / (nx + 1))[None, :] \
        + 2 * st.cS * np.cos(np.pi * q / (ny + 1))[:, None]
    fh = scipy.fft.dstn(np.asarray(f, dtype=np.float64)[1:-1, 1:-1], type=1)
    u = np.zeros((ny + 2, nx + 2))
    u[1:-1, 1:-1] = scipy.fft.idstn(fh / lam, type=1)
    return u


# Sources that define the cycle kernel; the DRAM traffic recorded under
# profiles/ counts only while their hash matches the one recorded with it.
KERNEL_SOURCES = ["paper_2006_16465_gb300/csrc/hj_tma.cuh", "paper_2006_16465_gb300/csrc/hj_cycle.cuh",
                  "paper_2006_16465_gb300/csrc/hj_internal.cuh"]
TRAFFIC_RECORD = "profiles/ppc2d_kernel_f32_32x32_k4_poisson8192_dram.md"


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(n):
    """DRAM bytes (read + write) per launch of the cycle kernel from the
    committed ncu record, or None if the kernel changed since, or the record
    is for another grid size."""
    try:
        rec = {}
        with open(os.path.join(ROOT, TRAFFIC_RECORD)) as fh:
            for line in fh:
                if ":" in line and line.split(":")[0].strip() in ("traffic_bytes_per_launch", "kernel_source_hash",
                                                                   "grid"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip().strip("`")
        if rec.get("kernel_source_hash") != kernel_source_hash() or int(rec.get("grid", 0)) != n:
            return None
        return float(rec["traffic_bytes_per_launch"])
    except Exception:
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, device) -> float:
    """Largest x over all ranks (a no-op without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_problem(n, seed=1):
    import torch
    import paper_2006_16465_gb300 as hj
    import workloads as W
    st = W.poisson_stencil(2, n, n)
    f = hj.alloc_grid(2, n, n, torch.float32)
    # seeded U[-1,1] from the shared generator, filled in row blocks to bound host memory
    rows = 512
    for j0 in range(0, n, rows):
        r = min(rows, n - j0)
        blk = W.uniform(seed, r * n, -1.0, 1.0, offset=j0 * n).reshape(r, n)
        f[1 + j0:1 + j0 + r, 1:n + 1].copy_(torch.from_numpy(blk).float())
    u0 = hj.alloc_grid(2, n, n, torch.float32)
    return st, f, u0


def _oracle_rhs_8192(W, n):
    st = W.poisson_stencil(2, n, n)
    f = W.zeros_grid(st)
    rows = 512
    for j0 in range(0, n, rows):
        r = min(rows, n - j0)
        f[1 + j0:1 + j0 + r, 1:n + 1] = W.uniform(1, r * n, -1.0, 1.0, offset=j0 * n).reshape(r, n)
    return st, f


def run_reference(args):
    """The oracle (plain C, binary64; its subdomain loop on every host core
    through OpenMP, bitwise the single-thread result) timed on the host on a
    bounded sample of the same workload: one hierarchical cycle of the
    n x n grid per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import workloads as W
    n = args.n
    st, f = _oracle_rhs_8192(W, n)
    u = W.zeros_grid(st)
    cores = oracle.set_threads(host_cores())
    for _ in range(args.warmup):
        u = oracle.run_fixed(st, f, u, 1, 32, 32, args.k)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = oracle.run_fixed(st, f, u, 1, 32, 32, args.k)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    glups = n * n * args.k * args.steps / dt / 1e9
    sample = (f"{args.steps} hierarchical cycles (k={args.k}, 32x32 subdomains) of the {n}x{n} grid, binary64, "
              f"{cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": glups, "unit": "GLUP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args, world),
            "cpu_baseline": {"value": glups, "unit": "GLUP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": glups, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config(args, world):
    n = getattr(args, "n", N_BENCH)
    return {"workload": f"2D Poisson {n}x{n} binary32, hierarchical Jacobi, 32x32 subdomains, "
                        f"k={args.k}, {args.cycles} cycles per step, fused residual on",
            "grid": [n, n], "tile": [32, 32], "k": args.k, "cycles_per_step": args.cycles,
            "l2": f"inputs larger than L2 (u, f and two more iterate buffers, {4 * (n + 2) * (n + 32) / 1e6:.0f} MB each)",
            "parallelism": f"replicas x{world}"}


def _oracle_rate(oracle, st, f, k, seconds):
    u = f * 0.0
    t0 = time.perf_counter()
    cyc = 0
    while True:
        u = oracle.run_fixed(st, f, u, 1, 32, 32, k)
        cyc += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return st.nx * st.ny * k * cyc / (time.perf_counter() - t0) / 1e9, cyc


def cpu_baseline(k, gpu_counts=None):
    """The oracle on the host cores, bounded (about 30 s in all):
      * value: hierarchical cycles of the full 8192^2 grid (binary64, k, 32x32
        subdomains), subdomains spread over every host core by OpenMP (the
        result is bitwise the single-thread one), and on one core;
      * time to a 1e-6 residual reduction: the 1D workload (N = 512, sum of
        8 sine modes, 128-point subdomains, k = 32, and classic sweeps) run
        to the end; the 2D 512^2 binary64 workload (f ~ U[-1,1]) projected
        from a bounded sample of cycles (the per-cycle time includes the
        residual check the oracle's solve makes every cycle) times the sweep
        count: classic from the closed form of Jacobi's decay on the sine
        modes, hierarchical (32x32, k = 16) from the GPU's binary64 solve,
        whose cycles are bitwise the oracle's."""
    import numpy as np
    import oracle
    import workloads as W
    cores = host_cores()
    st, f = _oracle_rhs_8192(W, N_BENCH)
    used = oracle.set_threads(cores)
    glups_all, cyc_all = _oracle_rate(oracle, st, f, k, 6.0)
    oracle.set_threads(1)
    glups_one, cyc_one = _oracle_rate(oracle, st, f, k, 4.0)
    del f
    out = {"value": glups_all, "unit": "GLUP/s", "cores": used, "kind": "oracle",
           "sample": f"{cyc_all} hierarchical cycles (k={k}, 32x32) of the 8192^2 grid, binary64, {used} threads",
           "single_core_glups": glups_one}
    oracle.set_threads(used)
    try:
        q = W.poisson1d_sine(512, seed=0)
        ttr = {}
        for name, kw in (("hier_128_k32", dict(tx=128, ty=1, k=32)), ("classic", dict(classic=True))):
            t0 = time.perf_counter()
            _, c, status, _ = oracle.solve(q.st, q.f, q.u0, 1e-6, 10 ** 7, **kw)
            ttr[name] = {"s": time.perf_counter() - t0, "cycles": c, "status": status}
        out["cfg1_1d_to_1e-6"] = ttr
        p = W.poisson2d_uniform(512, 512, seed=1)
        proj = {}
        # classic: per-sweep time over a bounded sample, sweeps from the closed form
        t0 = time.perf_counter()
        oracle.solve(p.st, p.f, p.u0, 1e-6, 3000, classic=True)
        per = (time.perf_counter() - t0) / 3000
        n_cl = classic_sweeps_closed_form(p.st, p.f, 1e-6)
        proj["classic"] = {"s_projected": per * n_cl, "sweeps_closed_form": n_cl, "s_per_sweep": per}
        t0 = time.perf_counter()
        oracle.solve(p.st, p.f, p.u0, 1e-6, 200, 32, 32, 16)
        per = (time.perf_counter() - t0) / 200
        n_h = (gpu_counts or {}).get("f64_k16")
        proj["hier_32x32_k16"] = {"s_per_cycle": per, "cycles_gpu_f64": n_h,
                                  "s_projected": per * n_h if n_h else None}
        out["cfg2_512_f64_to_1e-6"] = proj
    finally:
        oracle.set_threads(1)
    return out


def classic_sweeps_closed_form(st, f, factor):
    """Classic Jacobi sweeps from u0 = 0 until ||r_n|| <= factor ||r_0|| for a
    constant five-point stencil with zero Dirichlet data: in the sine basis
    every mode decays by mu = 1 - lam / d per sweep, so the residual norm
    after n sweeps is a closed-form sum over the transformed right-hand side."""
    import numpy as np
    import scipy.fft
    nx, ny = st.nx, st.ny
    d = st.cD + st.sigma_const
    lam = d + 2 * st.cW * np.cos(np.pi * np.arange(1, nx + 1) / (nx + 1))[None, :] \
        + 2 * st.cS * np.cos(np.pi * np.arange(1, ny + 1) / (ny + 1))[:, None]
    mu = np.abs(1.0 - lam / d).ravel()
    w = (scipy.fft.dstn(np.asarray(f, dtype=np.float64)[1:-1, 1:-1], type=1) ** 2).ravel()
    w0 = w.sum()
    lmu = np.log(np.maximum(mu, 1e-300))

    def ratio2(n):
        return float((w * np.exp(2 * n * lmu)).sum() / w0)

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


def _timed_solve(torch, hj, st, f, u0, dim=2, warm=True, **kw):
    """Create, warm (graphs, caches, tuning), solve from u0 and time it; the
    relative residual of the returned u is recomputed on the host."""
    dt_ = torch.float32 if kw.get("precision") == "f32" else torch.float64
    s = hj.Solver(st, **kw)
    fd = hj.grid_from(f, dim, dt_)
    if warm:
        s.solve(fd, hj.grid_from(u0, dim, dt_), check=False)
    u = hj.grid_from(u0, dim, dt_)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = s.solve(fd, u, check=False)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    s.close()
    uh = u[..., :st.nx + 2].double().cpu().numpy()
    out = {"s": sec, "cycles": r["cycles"], "outer": r["outer_steps"], "inner": r["inner_cycles"],
           "status": r["status"], "tile": [r["tile_x"], r["tile_y"]], "k": r["k"],
           "overlap": [r["overlap_x"], r["overlap_y"]]}
    if dim == 2:
        out["rel"] = host_rel_residual(st, f, uh)
    return out, uh


def time_to_residual(torch, hj, W, tol=1e-8):
    """The metric's first clause: 512^2 Poisson, f ~ U[-1,1], u0 = 0, to a
    1e-8 relative residual.  Hierarchical cycles in binary32 with binary64
    refinement (autotuned; 32x32, k = 32; and with 4 overlapping points)
    against the fastest of three binary64 global-memory Jacobi variants
    (one launch per sweep in graphs, one grid-synchronised persistent launch,
    the tile kernel with k = 1, which is one classic sweep bit for bit).
    'rel' is the relative residual of the returned u recomputed on the host."""
    p = W.poisson2d_uniform(512, 512, seed=1)
    out = {}
    runs = [("hj_f32ir_autotuned", dict(precision="f32_ir", inner_tol=1e-4, autotune=1, check_every=256)),
            ("hj_f32ir_32x32_k32", dict(tile_x=32, tile_y=32, k=32, precision="f32_ir", inner_tol=1e-4,
                                        check_every=256)),
            ("hj_f32ir_32x32_k32_o4", dict(tile_x=32, tile_y=32, k=32, overlap_x=4, overlap_y=4,
                                           precision="f32_ir", inner_tol=1e-4, check_every=256)),
            ("classic_f64_graphs", dict(method="classic", precision="f64", check_every=1024, persistent=0)),
            ("classic_f64_gridsync", dict(method="classic", precision="f64", persistent=1)),
            ("classic_f64_tile_k1", dict(tile_x=32, tile_y=32, k=1, precision="f64", check_every=1024))]
    for name, kw in runs:
        out[name], _ = _timed_solve(torch, hj, p.st, p.f, p.u0, tol=tol, max_cycles=5_000_000, **kw)
    classic = min((k for k in out if k.startswith("classic")), key=lambda k: out[k]["s"])
    out["classic_best"] = classic
    out["speedup_autotuned_vs_classic"] = out[classic]["s"] / out["hj_f32ir_autotuned"]["s"]
    out["speedup_32x32_k32_vs_classic"] = out[classic]["s"] / out["hj_f32ir_32x32_k32"]["s"]
    return out


def cfg2_k_sweep(torch, hj, W):
    """The k sweep on the 512^2 Poisson problem (f ~ U[-1,1], u0 = 0, 32x32
    subdomains): binary64 to a 1e-6 relative residual and binary32 to 1e-5
    (binary32 storage floors near 2e-6 here), k in {1, 4, 16, 64}, beside
    classic Jacobi in the same precision.  Inner GLUP/s = points x k x cycles
    / time (the analogue of the paper's k tables)."""
    p = W.poisson2d_uniform(512, 512, seed=1)
    n2 = 512 * 512
    out = {}
    for prec, tol in (("f64", 1e-6), ("f32", 1e-5)):
        row = {}
        for k in (1, 4, 16, 64):
            r, _ = _timed_solve(torch, hj, p.st, p.f, p.u0, warm=False, tile_x=32, tile_y=32, k=k, precision=prec,
                                tol=tol, max_cycles=10_000_000, check_every=1024 if k == 1 else 256)
            r["inner_glups"] = n2 * k * r["cycles"] / r["s"] / 1e9
            row[f"k{k}"] = r
        r, _ = _timed_solve(torch, hj, p.st, p.f, p.u0, warm=False, method="classic", precision=prec, tol=tol,
                            max_cycles=10_000_000, check_every=1024, persistent=0)
        row["classic"] = r
        out[f"{prec}_to_{tol:g}"] = row
    return out


def cfg3_precision(torch, hj, W):
    """Mixed precision on 512^2 Poisson with f = sin(pi x) sin(pi y) + 1e-3
    U[-1,1]: refinement to a 1e-10 relative residual with binary32 inner
    cycles and with a bfloat16-stored correction, beside all-binary64
    hierarchical cycles to the same tolerance.  Each result's error is
    measured against the exact discrete solution (sine-transform solve) and
    against the binary64 result."""
    import numpy as np
    p = W.poisson2d_sin_noise(512, seed=2)
    ue = dst_solution(p.st, p.f)
    out = {}
    sols = {}
    runs = [("f32_ir", dict(precision="f32_ir", tile_x=32, tile_y=32, k=32, inner_tol=1e-4, check_every=256)),
            ("bf16corr_ir", dict(precision="bf16corr_ir", tile_x=32, tile_y=32, k=32, inner_tol=1e-4,
                                 check_every=256)),
            ("f64", dict(precision="f64", tile_x=32, tile_y=32, k=32, check_every=256))]
    for name, kw in runs:
        r, uh = _timed_solve(torch, hj, p.st, p.f, p.u0, warm=False, tol=1e-10, max_cycles=10_000_000,
                             max_outer=200, **kw)
        r["err_vs_exact"] = float(np.linalg.norm(uh - ue) / np.linalg.norm(ue))
        out[name] = r
        sols[name] = uh
    for name in ("f32_ir", "bf16corr_ir"):
        out[name]["err_vs_f64"] = float(np.linalg.norm(sols[name] - sols["f64"]) / np.linalg.norm(sols["f64"]))
    return out


def fd_check(torch, hj, W, n=1024, entries=32, rel_step=1e-6, seed=7, tol=1e-12, du_tol=1e-9):
    """Central differences of L(sigma) = 0.5 ||u(sigma) - u*||^2 against the
    implicit-adjoint gradient dL/dsigma_p = -lambda_p u_p, at `entries`
    random interior points of the differentiation workload (Fourier sigma
    field, first right-hand side), binary64 solutions.

    With step delta = rel_step * sigma_p, the loss changes by ~1e-14 of itself
    at 1024^2: two losses of separately re-solved problems cannot resolve
    that.  So each perturbed solution is u + du, with du the correction a
    solve warm-started from u computes: A(sigma +- delta e_p) du = -+ delta u_p
    e_p (the base residual, common to both and near rounding level, left
    out), solved to a relative residual of du_tol by binary32 cycles with
    binary64 refinement, all 2 x entries corrections in one batched call.
    Then L(u + du) - L(u) = sum du (u - u*) + 0.5 sum du^2, exactly.  The
    base solve and the adjoint run to tol (binary64 refinement)."""
    import numpy as np
    st, fs, ustar = W.differentiation_problem(n, 1, seed=seed)
    sig = st.sigma
    f = hj.grid_from(fs[0], 2, torch.float64)
    sigma = hj.grid_from(sig, 2, torch.float64)
    target = hj.grid_from(ustar, 2, torch.float64)
    prm = dict(tile_x=64, tile_y=64, k=32, precision="f32_ir", inner_tol=1e-4)
    t0 = time.perf_counter()
    s = hj.Solver(st, sigma=sigma, tol=tol, **prm)
    u = hj.alloc_grid(2, n, n, torch.float64)
    s.solve(f, u)
    g = u - target
    g[0, :] = 0
    g[-1, :] = 0
    g[:, 0] = 0
    g[:, n + 1:] = 0
    dl_df = torch.zeros_like(u)
    dl_dsig = torch.zeros_like(u)
    s.adjoint(g, u, dl_df, dl_dsig)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    s.close()
    idx = (W.uniform01(seed + 1000, 2 * entries) * n).astype(np.int64) + 1
    pts = [(int(idx[2 * e]), int(idx[2 * e + 1])) for e in range(entries)]   # (row j, column i)
    # 2 x entries perturbed problems, one batched refinement solve
    sigs, rhs, dus, descs = [], [], [], []
    for (j, i) in pts:
        for sgn in (1.0, -1.0):
            dlt = rel_step * float(sig[j, i])
            sp = sigma.clone()
            sp[j, i] += sgn * dlt
            b = torch.zeros_like(u)
            b[j, i] = -sgn * dlt * u[j, i]
            sigs.append(sp)
            rhs.append(b)
            dus.append(torch.zeros_like(u))
            descs.append(hj.make_desc(2, n, n, u.shape[1], st.cW, st.cE, st.cS, st.cN, st.cD, 0.0, sp))
    sb = hj.Solver(st, sigma=sigma, tol=du_tol, **prm)
    stats = hj.hj_stats()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    code = hj.hj_solve_batched(sb.h, descs, [b.data_ptr() for b in rhs], [d.data_ptr() for d in dus],
                               hj._stream_handle(None), stats)
    torch.cuda.synchronize()
    t_fd = time.perf_counter() - t1
    sb.close()
    w = (u - target)[1:n + 1, 1:n + 1]
    fd, adj, rel = [], [], []
    for e, (j, i) in enumerate(pts):
        dp, dm = dus[2 * e][1:n + 1, 1:n + 1], dus[2 * e + 1][1:n + 1, 1:n + 1]
        lp = float((dp * w).sum() + 0.5 * (dp * dp).sum())
        lm = float((dm * w).sum() + 0.5 * (dm * dm).sum())
        dlt = rel_step * float(sig[j, i])
        fd.append((lp - lm) / (2 * dlt))
        adj.append(float(dl_dsig[j, i]))
        rel.append(abs(fd[-1] - adj[-1]) / abs(adj[-1]))
    scale = max(abs(a) for a in adj)
    return {"grid": [n, n], "entries": entries, "rel_step": rel_step, "status": code,
            "batched_rel_final": stats.rel_final, "max_rel_err": max(rel), "median_rel_err": float(np.median(rel)),
            "max_err_over_max_grad": max(abs(a - b) for a, b in zip(fd, adj)) / scale,
            "forward_adjoint_s": t_adj, "fd_solves_s": t_fd, "points": pts, "fd": fd, "adjoint": adj}


def classic_rate(torch, hj, n, cycles=200):
    """Plain global-memory Jacobi (Section 3.2) on the n x n bench grid,
    binary32: the sweep kernel alone (fixed sweeps) against its 12 B per
    point (read u and f, write u), and with the fused residual every sweep."""
    st, f, u0 = make_problem(n)
    uc = u0.clone()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rates = {}
    for name, kw in (("sweep", dict(fixed_cycles=cycles)),
                     ("sweep_and_residual", dict(tol=0.0, max_cycles=cycles, check_every=100))):
        cl = hj.Solver(st, method="classic", precision="f32", **kw)
        cl.solve(f, uc, check=False)
        torch.cuda.synchronize()
        e0.record(stream)
        cl.solve(f, uc, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        rates[name] = e0.elapsed_time(e1) / cycles
        cl.close()
    hbm_peak, _ = _peaks()
    cms = rates["sweep"]
    return {"glups": n * n / (cms / 1e3) / 1e9, "us_per_sweep": cms * 1e3,
            "hbm_gbs": 12 * n * n / (cms / 1e3) / 1e9, "hbm_frac": 12 * n * n / (cms / 1e3) / 1e9 / hbm_peak,
            "us_per_sweep_with_fused_residual": rates["sweep_and_residual"] * 1e3}


def inner_roofline(torch, hj, W, n, k=16, cycles=100):
    """Inner sweeps bound by the binary32 FMA pipe: 4 FMAs per point update, so
    peak = SMs x 128 lanes x max SM clock / 4 point updates per second."""
    st, f, u0 = make_problem(n)
    s = hj.Solver(st, tile_x=32, tile_y=32, k=k, precision="f32", fixed_cycles=cycles, check_every=cycles)
    u = u0.clone()
    s.solve(f, u)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    s.solve(f, u)
    e1.record()
    torch.cuda.synchronize()
    s.close()
    ms = e0.elapsed_time(e1)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_max_mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            sm_max_mhz = float(json.load(fh).get("sm_max_mhz", sm_max_mhz))
    except Exception:
        pass
    peak = props.multi_processor_count * 128 * sm_max_mhz * 1e6 / 4 / 1e9
    achieved = n * n * k * cycles / (ms / 1e3) / 1e9
    # the on-chip data path of the sweeps: their east/west neighbours and band
    # edges move by warp shuffle, which goes through the SM's shared-memory
    # data pipe at one warp-wide shuffle per clock; a 32x32 subdomain (one
    # warp, two bands of 16 rows, two columns per lane) issues 2 x 16 row
    # shuffles and 2 band-exchange shuffles per subiteration
    smem_bound = props.multi_processor_count * sm_max_mhz * 1e6 * 1024 / 34 / 1e9
    return {"bound": "alu", "k": k, "achieved": achieved, "peak": peak, "unit": "GLUP/s", "frac": achieved / peak,
            "peak_basis": "SMs x 128 FP32 lanes x max SM clock / 4 FMA per point update",
            "smem_path_bound": smem_bound, "smem_path_frac": achieved / smem_bound,
            "smem_path_basis": "SMs x max SM clock x 1024 point updates / 34 warp shuffles (shared-memory data pipe, "
                               "one warp-wide shuffle per clock)"}


def variable_coefficients(torch, hj, W, n=4096, hbm_peak=None):
    """Per-point neighbour coefficients (heterogeneous diffusion, kappa
    contrast 10): the thread-per-point kernel's cycle rate and its roofline
    at n^2, and time to a 1e-6 residual reduction at 256^2, hierarchical vs
    classic (both binary64).  Algorithmic bytes per point and cycle: binary32
    u in/out, f, four -c/d planes and 1/d = 32 B; binary64 u in/out, f, four
    coefficient planes and 1/d = 64 B.  Binary64 is bound by the FP64 pipe:
    9 separately rounded operations per point update against the part's
    nominal 1.25 TFLOP/s FP64 = 0.625 T operations/s."""
    out = {}
    p = W.variable_coef_problem(2, n, n, seed=5, contrast=10.0)
    st = p.st
    ld = hj.padded_ld(n, torch.float32)
    planes = torch.zeros((4, n + 2, ld), dtype=torch.float64, device="cuda")
    planes[:, :, :n + 2] = torch.as_tensor(st.coef)
    sig = hj.grid_from(st.sigma, 2, torch.float64)
    runs = [("f32", (32, 32), 4), ("f32", (32, 8), 1), ("f32", (32, 8), 4), ("f32", (32, 8), 16),
            ("f64", (32, 8), 1), ("f64", (32, 8), 4)]
    for prec, tile, k in runs:
        dt = torch.float32 if prec == "f32" else torch.float64
        bpp = 32 if prec == "f32" else 64
        f = hj.grid_from(p.f, 2, dt)
        t = []
        for ncyc in (4, 24):
            s = hj.Solver(st, sigma=sig, coef=planes, tile_x=tile[0], tile_y=tile[1], k=k, precision=prec,
                          fixed_cycles=ncyc)
            u = hj.grid_from(p.u0, 2, dt)
            s.solve(f, u)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            s.solve(f, u)
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
            s.close()
        us = (t[1] - t[0]) / 20 * 1e3
        gbs = bpp * n * n / (us / 1e6) / 1e9
        row = {"us_per_cycle": us, "glups": n * n / (us / 1e6) / 1e9, "hbm_gbs": gbs,
               "hbm_frac": gbs / hbm_peak if hbm_peak else None, "bytes_per_point": bpp}
        if prec == "f64":
            row["fp64_ops_per_s"] = 9.0 * k * n * n / (us / 1e6)
            row["fp64_frac"] = row["fp64_ops_per_s"] / 0.625e12
        out[f"{prec}_{tile[0]}x{tile[1]}_k{k}"] = row
        del f
    del planes, sig
    q = W.variable_coef_problem(2, 256, 256, seed=6, contrast=10.0)
    qpl = torch.zeros((4, 258, hj.padded_ld(256, torch.float64)), dtype=torch.float64, device="cuda")
    qpl[:, :, :258] = torch.as_tensor(q.st.coef)
    qsig = hj.grid_from(q.st.sigma, 2, torch.float64)
    f = hj.grid_from(q.f, 2, torch.float64)
    ttr = {}
    for name, kw in [("hier_f64_32x32_k16", dict(tile_x=32, tile_y=32, k=16, check_every=64)),
                     ("hier_f64_32x32_k64", dict(tile_x=32, tile_y=32, k=64, check_every=64)),
                     ("classic_f64", dict(method="classic", check_every=1024))]:
        s = hj.Solver(q.st, sigma=qsig, coef=qpl, precision="f64", tol=1e-6, max_cycles=20_000_000, **kw)
        u = hj.grid_from(q.u0, 2, torch.float64)
        s.solve(f, u.clone())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = s.solve(f, u)
        torch.cuda.synchronize()
        ttr[name] = {"seconds": time.perf_counter() - t0, "cycles": r["cycles"], "status": r["status"]}
        s.close()
    for name in ("hier_f64_32x32_k16", "hier_f64_32x32_k64"):
        ttr[f"speedup_{name}_vs_classic"] = ttr["classic_f64"]["seconds"] / ttr[name]["seconds"]
    out["time_to_1e-6_256_kappa10"] = ttr
    return out


def three_d(torch, hj, W, n=512, hbm_peak=None):
    """3D seven-point extension: cycle rate and HBM roofline of the
    subdomain kernels (binary32 at this size: the TMA-pipelined kernel) and of
    the classic sweep at n^3 (binary32: 12 B
    per point and cycle, u in/out and f; binary64 is bound by the FP64 pipe,
    13 separately rounded operations per update), and time to a 1e-5
    residual reduction at 128^3 (binary32), hierarchical vs classic."""
    out = {}
    st = W.poisson_stencil3d(n, n, n)
    runs = [("f32", (16, 8, 4), 1), ("f32", (16, 8, 4), 4), ("f32", (16, 8, 8), 4), ("f32", (32, 4, 8), 1),
            ("f32", (32, 4, 8), 4), ("f32", None, 1), ("f64", (16, 4, 8), 1), ("f64", (16, 4, 8), 4)]
    for prec, tile, k in runs:
        dt = torch.float32 if prec == "f32" else torch.float64
        bpp = 12 if prec == "f32" else 24
        f = hj.alloc_grid(3, n, n, dt, nz=n, fill=1.0)
        t = []
        for ncyc in (4, 24):
            kw = dict(method="classic") if tile is None else dict(tile_x=tile[0], tile_y=tile[1], tile_z=tile[2], k=k)
            s = hj.Solver(st, precision=prec, fixed_cycles=ncyc, **kw)
            u = hj.alloc_grid(3, n, n, dt, nz=n)
            s.solve(f, u)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            s.solve(f, u)
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
            s.close()
            del u
        us = (t[1] - t[0]) / 20 * 1e3
        gbs = bpp * n ** 3 / (us / 1e6) / 1e9
        row = {"us_per_cycle": us, "glups": n ** 3 / (us / 1e6) / 1e9, "hbm_gbs": gbs,
               "hbm_frac": gbs / hbm_peak if hbm_peak else None}
        if prec == "f64":
            row["fp64_frac"] = 13.0 * k * n ** 3 / (us / 1e6) / 0.625e12
        name = "classic" if tile is None else f"{tile[0]}x{tile[1]}x{tile[2]}_k{k}"
        out[f"{prec}_{name}"] = row
        del f
    q = W.poisson3d_uniform(128, seed=4)
    f = hj.grid_from(q.f, 3, torch.float32)
    ttr = {}
    for name, kw in [("hier_16x8x8_k8", dict(tile_x=16, tile_y=8, tile_z=8, k=8, check_every=64)),
                     ("hier_16x8x8_k16", dict(tile_x=16, tile_y=8, tile_z=8, k=16, check_every=64)),
                     ("hier_16x8x4_k8", dict(tile_x=16, tile_y=8, tile_z=4, k=8, check_every=64)),
                     ("classic", dict(method="classic", check_every=1024))]:
        s = hj.Solver(q.st, precision="f32", tol=1e-5, max_cycles=10_000_000, **kw)
        u = hj.grid_from(q.u0, 3, torch.float32)
        s.solve(f, u.clone())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = s.solve(f, u)
        torch.cuda.synchronize()
        ttr[name] = {"seconds": time.perf_counter() - t0, "cycles": r["cycles"], "status": r["status"]}
        s.close()
    for name in list(ttr):
        if name != "classic":
            ttr[f"speedup_{name}_vs_classic"] = ttr["classic"]["seconds"] / ttr[name]["seconds"]
    out["time_to_1e-5_128_f32"] = ttr
    return out


def multigrid(torch, hj, W, n=4095, hbm_peak=None):
    """Hierarchical Jacobi as a multigrid smoother (V-cycles, damped
    subiterations, full weighting, bilinear prolongation): per-V-cycle time
    at n^2 with its algorithmic bytes, time to 1e-10 (binary64) at n^2, and
    time to 1e-8 at 511^2 against the hierarchical Jacobi solver alone
    (binary32 inner cycles, binary64 refinement).

    Algorithmic bytes per V(pre, post)-cycle, binary32, per fine point: each
    level moves 12 (pre + post) + 19 B per own point (smoothing 12 B a cycle;
    restriction reads u, f and writes the coarse f and correction; the
    prolongation reads and writes u and reads the correction), and levels add
    up to 4/3 of the fine level.  The per-V-cycle rows are fixed-cycle runs,
    whose V-cycles carry no residual check (converging runs add one binary64
    residual of the fine level per V-cycle)."""
    out = {}
    q = W.poisson2d_uniform(n, n, seed=1)
    for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
        f = hj.grid_from(q.f, 2, dt)
        for pre, post, k, tile in ((1, 1, 2, (32, 8)), (2, 2, 2, (32, 32))):
            s = hj.Solver(q.st, method="mg", precision=prec, tile_x=tile[0], tile_y=tile[1], k=k, mg_pre=pre,
                          mg_post=post, fixed_cycles=10)
            u = hj.grid_from(q.u0, 2, dt)
            s.solve(f, u)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            s.solve(f, u)
            e1.record()
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) / 10 * 1e3
            s.close()
            row = {"us_per_vcycle": us}
            if prec == "f32":
                bpp = (12 * (pre + post) + 19) * 4.0 / 3.0
                row["algorithmic_bytes_per_point"] = bpp
                row["hbm_gbs"] = bpp * n * n / (us / 1e6) / 1e9
                row["hbm_frac"] = row["hbm_gbs"] / hbm_peak if hbm_peak else None
            out[f"{prec}_V{pre}{post}_k{k}_{tile[0]}x{tile[1]}"] = row
        if prec == "f64":
            s = hj.Solver(q.st, method="mg", precision="f64", tile_x=32, tile_y=8, k=2, tol=1e-10, max_cycles=100)
            u = hj.grid_from(q.u0, 2, dt)
            s.solve(f, u.clone())
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = s.solve(f, u)
            torch.cuda.synchronize()
            out["f64_to_1e-10"] = {"seconds": time.perf_counter() - t0, "vcycles": r["cycles"],
                                   "rel_final": r["rel_final"], "status": r["status"]}
            s.close()
        del f
    p = W.poisson2d_uniform(511, 511, seed=1)
    f = hj.grid_from(p.f, 2, torch.float64)
    ttr = {}
    for name, kw in [("mg_f64_V11_k2", dict(method="mg", precision="f64", tile_x=32, tile_y=8, k=2, max_cycles=100)),
                     ("hier_f32_ir_32x32_k32", dict(tile_x=32, tile_y=32, k=32, precision="f32_ir", inner_tol=1e-4,
                                                    check_every=256))]:
        s = hj.Solver(p.st, tol=1e-8, **kw)
        u = hj.grid_from(p.u0, 2, torch.float64)
        s.solve(f, u.clone())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = s.solve(f, u)
        torch.cuda.synchronize()
        ttr[name] = {"seconds": time.perf_counter() - t0, "cycles": r["cycles"], "status": r["status"]}
        s.close()
    ttr["speedup_mg_vs_hier"] = ttr["hier_f32_ir_32x32_k32"]["seconds"] / ttr["mg_f64_V11_k2"]["seconds"]
    out["time_to_1e-8_511"] = ttr
    return out


def paper_replicas(torch, hj, W, precision="f64"):
    """Context: the paper's timing problems (Sections 3.5 and 4.2), residual
    reduced by 1e-4 from x0 = 1 with b = 1: best classic vs hierarchical
    (tpb 32 / 32x32) for each k of Tables 1 and 3, and with the overlap the
    paper found best for that k (Sections 3.4, 4.3).  The paper runs them in
    binary64; precision="f32" runs the same problems in binary32, where a
    hierarchical cycle's subiterations are cheap on this part."""
    out = {}
    dt = torch.float64 if precision == "f64" else torch.float32
    for dim, tile in ((1, (32, 1)), (2, (32, 32))):
        p = W.paper_replica(dim, 1024, copies=1024)
        f = hj.grid_from(p.f, dim, dt)
        res = {}
        # overlap that Tables 2 (1D) and 4 (2D) report as best for each k
        best_o = {1: {4: 2, 8: 4, 16: 4, 32: 8, 64: 10, 128: 12}, 2: {4: 0, 8: 2, 16: 2, 32: 4, 64: 6, 128: 8}}[dim]
        runs = [("classic_graphs", dict(method="classic", persistent=0, check_every=1024)),
                ("classic_gridsync", dict(method="classic", persistent=1)),
                ("classic_tile_k1", dict(tile_x=tile[0], tile_y=tile[1], k=1, check_every=1024))]
        runs += [(f"hier_k{k}", dict(tile_x=tile[0], tile_y=tile[1], k=k)) for k in (4, 8, 16, 32, 64, 128)]
        runs += [(f"hier_k{k}_o{best_o[k]}", dict(tile_x=tile[0], tile_y=tile[1], k=k, overlap_x=best_o[k],
                                                  overlap_y=best_o[k] if dim == 2 else 0, persistent=0))
                 for k in (4, 8, 16, 32, 64, 128) if best_o[k] > 0]
        # one global array (Appendix A taken literally): convergence and speed
        runs += [(f"hier_k{k}_in_place", dict(tile_x=tile[0], tile_y=tile[1], k=k, in_place=1)) for k in (4, 16, 64)]
        for name, kw in runs:
            s = hj.Solver(p.st, precision=precision, tol=1e-4, **kw)
            u = hj.grid_from(p.u0, dim, dt)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = s.solve(f, u)
            torch.cuda.synchronize()
            res[name] = {"seconds": time.perf_counter() - t0, "cycles": r["cycles"], "status": r["status"]}
            s.close()
        best = min(res[k]["seconds"] for k in ("classic_graphs", "classic_gridsync", "classic_tile_k1"))
        res["speedup_vs_best_classic"] = {k: best / v["seconds"] for k, v in res.items() if k.startswith("hier")}
        out[f"{dim}d"] = res
    return out


def time_1d(torch, hj, W):
    """cfg1: 1D Poisson N = 512, f = sum of 8 sine modes, binary64, to 1e-6:
    hierarchical (128-point subdomains, k = 32) vs classic."""
    q = W.poisson1d_sine(512, seed=0)
    f = hj.grid_from(q.f, 1, torch.float64)
    out = {}
    for name, kw in [("hier_f64", dict(tile_x=128, k=32)), ("classic_f64", dict(method="classic")),
                     ("classic_f64_tile_k1", dict(tile_x=128, k=1))]:
        s = hj.Solver(q.st, precision="f64", tol=1e-6, check_every=512, **kw)
        u = hj.grid_from(q.u0, 1, torch.float64)
        s.solve(f, u.clone())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = s.solve(f, u)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "cycles": r["cycles"], "status": r["status"]}
        s.close()
    out["speedup"] = min(out["classic_f64"]["seconds"], out["classic_f64_tile_k1"]["seconds"]) / \
        out["hier_f64"]["seconds"]
    return out


def time_batched(torch, hj, W):
    """cfg4: 256 screened problems, sides from {64..512}, binary32 inner cycles
    with binary64 refinement to 1e-8: every refinement step one replay of a
    captured graph around one persistent launch fed by the device work queue;
    autotuned tile and per-size-class k (second call timed: tuning is cached).
    The per-batch-cycle log gives the time against the points still active:
    inner point updates per second against the binary32 FMA bound (SMs x 128
    lanes x max SM clock / 4 FMA per update), and the time of the cycles with
    fewer than 1M active points (the tail)."""
    import ctypes as C
    import numpy as np
    probs = W.batched_screened(256, seed=3)
    s = hj.Solver(probs[0].st, tile_x=32, tile_y=32, k=16, precision="f32_ir", tol=1e-8, autotune=1)
    fs = [hj.grid_from(q.f, 2, torch.float64) for q in probs]
    descs = [hj.make_desc(2, q.st.nx, q.st.ny, f.shape[1], q.st.cW, q.st.cE, q.st.cS, q.st.cN, q.st.cD,
                          q.st.sigma_const) for q, f in zip(probs, fs)]
    cap = 1 << 20
    ms = (C.c_double * cap)()
    pts = (C.c_longlong * cap)()
    res = {}
    for rep in range(2):
        us = [hj.grid_from(q.u0, 2, torch.float64) for q in probs]
        st = hj.hj_stats()
        st.cycle_ms = C.cast(ms, C.POINTER(C.c_double))
        st.cycle_points = C.cast(pts, C.POINTER(C.c_longlong))
        st.cycle_cap = cap
        cyc = (hj.C.c_longlong * len(probs))()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code = hj.hj_solve_batched(s.h, descs, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], 0, st, cyc)
        torch.cuda.synchronize()
        n = st.cycle_len
        m = np.array(ms[:n]) * 1e-3   # seconds per batch cycle
        p = np.array(pts[:n], dtype=np.float64)
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        alu_peak = props.multi_processor_count * 128 * 2070e6 / 4
        upd = float((p * st.k).sum()) if st.k else 0.0
        res = {"seconds": time.perf_counter() - t0, "status": code, "graphed": st.graphed,
               "worst_rel_residual": st.rel_final, "outer_steps": st.outer_steps,
               "inner_cycles_total": st.inner_cycles, "inner_cycles_max": max(cyc),
               "unknowns": sum(q.st.nx * q.st.ny for q in probs), "tile": [st.tile_x, st.tile_y], "k_max": st.k,
               "batch_cycles": n, "batch_cycle_seconds": float(m.sum()),
               "us_per_cycle_all_active": float(m[p >= p.max()].mean() * 1e6) if n else None,
               "us_per_cycle_tail": float(m[p < 1e6].mean() * 1e6) if (p < 1e6).any() else None,
               "tail_cycles_lt_1M_points": int((p < 1e6).sum()), "tail_seconds": float(m[p < 1e6].sum()),
               "inner_updates_per_s_at_k_max": upd / float(m.sum()) if n else None,
               "inner_alu_frac_at_k_max": upd / float(m.sum()) / alu_peak if n else None}
    s.close()
    return res


def time_differentiation(torch, hj, W):
    """cfg5: screened Poisson 1024^2, Fourier sigma field, 16 RHS, loss
    0.5 ||u - u*||^2; forward solves and implicit-adjoint backward (binary32
    inner cycles, binary64 refinement to 1e-10)."""
    from paper_2006_16465_gb300.autograd import solve_screened
    st, fs, ustar = W.differentiation_problem(1024, 16, seed=7)
    f = torch.stack([hj.grid_from(x, 2, torch.float64) for x in fs]).requires_grad_(True)
    sigma = hj.grid_from(st.sigma, 2, torch.float64).requires_grad_(True)
    target = hj.grid_from(ustar, 2, torch.float64)
    params = dict(tile_x=64, tile_y=64, k=32, precision="f32_ir", tol=1e-10)

    def loss_of(u):
        return 0.5 * ((u - target)[:, 1:-1, 1:1025] ** 2).sum()

    # PyTorch loads (and may JIT) its own elementwise / reduction kernels on
    # first use: run the loss expression once on a small slice first
    w = torch.zeros(2, 10, 16, dtype=torch.float64, device=target.device)
    (0.5 * ((w - w[0])[:, 1:-1, 1:9] ** 2).sum()).item()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u = solve_screened(f, sigma, st, **params)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss = loss_of(u)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    return {"forward_seconds": t1 - t0, "loss_seconds": t2 - t1, "backward_seconds": t3 - t2, "rhs": 16,
            "grid": [1024, 1024],
            "loss": float(loss.detach()), "grad_sigma_norm": float(sigma.grad.norm()),
            "grad_f_norm": float(f.grad.norm())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hj", choices=["hj", "reference"])
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--cycles", type=int, default=1000)
    ap.add_argument("--n", type=int, default=N_BENCH, help="grid side (profiling runs use a smaller grid)")
    ap.add_argument("--no-extras", action="store_true", help="skip classic / time-to-residual / cpu legs")
    ap.add_argument("--launch", default="",
                    help="pin the pipelined kernel's launch as THREADS,STAGES,CTAS_PER_SM instead of tuning it "
                         "(profiling runs: keeps the tuner's launches out of the capture)")
    ap.add_argument("--paper-replicas", action="store_true",
                    help="also time the paper's Section 3.5 / 4.2 problems (binary64, minutes)")
    ap.add_argument("--only", default="", choices=["", "variable_coefficients", "three_d", "multigrid",
                                                    "time_to_residual", "cfg2_k_sweep", "cfg3_precision",
                                                    "fd_check", "cpu_baseline", "classic", "batched",
                                                    "differentiation"],
                    help="run one extras section alone and print its JSON (profiling runs)")
    ap.add_argument("--fd-n", type=int, default=1024, help="grid side of the finite-difference check")
    ap.add_argument("--fd-entries", type=int, default=32, help="sigma entries the finite-difference check perturbs")
    ap.add_argument("--extras-out", default=EXTRAS_OUT, help="where the full record of the extra legs goes")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        import torch
        import paper_2006_16465_gb300 as hj
        import workloads as W
        torch.cuda.set_device(0)
        hbm_peak, _ = _peaks()
        section = {"variable_coefficients": lambda: variable_coefficients(torch, hj, W, hbm_peak=hbm_peak),
                   "three_d": lambda: three_d(torch, hj, W, hbm_peak=hbm_peak),
                   "multigrid": lambda: multigrid(torch, hj, W, hbm_peak=hbm_peak),
                   "time_to_residual": lambda: time_to_residual(torch, hj, W),
                   "cfg2_k_sweep": lambda: cfg2_k_sweep(torch, hj, W),
                   "cfg3_precision": lambda: cfg3_precision(torch, hj, W),
                   "fd_check": lambda: fd_check(torch, hj, W, n=args.fd_n, entries=args.fd_entries),
                   "cpu_baseline": lambda: cpu_baseline(args.k),
                   "classic": lambda: classic_rate(torch, hj, args.n),
                   "batched": lambda: time_batched(torch, hj, W),
                   "differentiation": lambda: time_differentiation(torch, hj, W)}
        print(json.dumps({args.only: section[args.only]()}), flush=True)
        return 0

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2006_16465_gb300 as hj
    import workloads as W

    n, k, C = args.n, args.k, args.cycles
    st, f, u0 = make_problem(n)
    # 32x32 subdomains and k are the workload; the launch shape of the pipelined
    # kernel (threads per subdomain, copy stages, CTAs per SM) is measured at
    # creation (autotune = 3), or pinned with --launch
    if args.launch:
        th, stg, cps = (int(x) for x in args.launch.split(","))
        launch_kw = dict(tile_threads=th, pipeline_stages=stg, ctas_per_sm=cps)
    else:
        launch_kw = dict(autotune=3)
    solver = hj.Solver(st, tile_x=32, tile_y=32, k=k, precision="f32", tol=0.0, max_cycles=C, check_every=100,
                       **launch_kw)
    u = u0.clone()
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        solver.solve(f, u, check=False)
    launches = 0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            r = solver.solve(f, u, check=False)
            launches += r["cycles_launched"]
        ev1.record(stream)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), torch.device("cuda", local))
    launch_used = {"threads_per_subdomain": r["tile_threads"], "copy_stages": r["pipeline_stages"],
                   "ctas_per_sm": r["ctas_per_sm"], "tuned": not args.launch}
    cycles_done = args.steps * C
    glups = job_rate(n * n * k * cycles_done, world, ms) / 1e9
    per_launch_ms = ms / cycles_done
    hbm_peak, peak_kind = _peaks()
    achieved = BYTES_PER_POINT_CYCLE * n * n / (per_launch_ms / 1e3) / 1e9

    # e2e through the C ABI with host buffers (copies inside the timed region)
    fh = f.cpu().pin_memory()
    uh = u0.cpu().pin_memory()
    solver.solve(fh, uh, check=False)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.solve(fh, uh, check=False)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, torch.device("cuda", local))
    e2e = {"value": job_rate(n * n * k * cycles_done, world, e2e_s * 1e3) / 1e9, "unit": "GLUP/s",
           "h2d_bytes_per_step": 2 * f.numel() * 4, "d2h_bytes_per_step": u.numel() * 4}

    extras = {}
    if not args.no_extras and rank == 0:
        # plain global-memory Jacobi on the same grid: the sweep kernel alone
        # (fixed sweeps: its HBM roofline) and with the fused residual every
        # sweep (as the converging solves run it)
        extras["classic_global_jacobi"] = classic_rate(torch, hj, n, cycles=1000)
        uc = u0.clone()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        # the same sweep through the tile kernels (a hierarchical cycle with k = 1 is one
        # classic sweep, bitwise), launch shape tuned like the headline's
        cl = hj.Solver(st, tile_x=32, tile_y=32, k=1, precision="f32", tol=0.0, max_cycles=1000, check_every=100,
                       autotune=3)
        cl.solve(f, uc, check=False)
        torch.cuda.synchronize()
        e0.record(stream)
        cl.solve(f, uc, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        tms = e0.elapsed_time(e1) / 1000
        extras["classic_jacobi_tile_kernel_k1"] = {"glups": n * n / (tms / 1e3) / 1e9, "us_per_sweep": tms * 1e3,
                                                   "hbm_gbs": 12 * n * n / (tms / 1e3) / 1e9}
        cl.close()
        del uc
        extras["hier_global_cycle_rate_gdofs"] = n * n / (per_launch_ms / 1e3) / 1e9
        extras["time_to_1e-8_512"] = time_to_residual(torch, hj, W)
        extras["cfg2_k_sweep_512"] = cfg2_k_sweep(torch, hj, W)
        extras["cfg3_precision_512"] = cfg3_precision(torch, hj, W)
        extras["cfg1_1d_to_1e-6"] = time_1d(torch, hj, W)
        extras["cfg4_batched_256_to_1e-8"] = time_batched(torch, hj, W)
        extras["cfg5_differentiation_1024"] = time_differentiation(torch, hj, W)
        extras["cfg5_fd_check"] = fd_check(torch, hj, W, n=args.fd_n, entries=args.fd_entries)
        extras["inner_sweep_roofline_k16"] = inner_roofline(torch, hj, W, n)
        extras["variable_coefficients_4096"] = variable_coefficients(torch, hj, W, hbm_peak=hbm_peak)
        extras["three_d_512"] = three_d(torch, hj, W, hbm_peak=hbm_peak)
        extras["multigrid_4095"] = multigrid(torch, hj, W, hbm_peak=hbm_peak)
    if args.paper_replicas and rank == 0:
        extras["paper_replicas"] = paper_replicas(torch, hj, W)
        extras["paper_replicas_f32"] = paper_replicas(torch, hj, W, "f32")
    launches += args.steps  # one residual launch per step (the final iterate is not converged: tol = 0)
    ntiles = ((n + 31) // 32) ** 2
    pipelined = ntiles >= 8 * torch.cuda.get_device_properties(local).multi_processor_count
    kernel_name = ("ppc2d_kernel" if pipelined else "hier2d_kernel") + "<float,32x32>"
    line = {"metric": METRIC, "value": _r(glups), "unit": "GLUP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": _r(ms / args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(_config(args, world), launch=launch_used),
            "roofline": {"bound": "hbm", "achieved": _r(achieved), "peak": hbm_peak, "unit": "GB/s",
                         "frac": _r(achieved / hbm_peak), "traffic": recorded_traffic(n),
                         "algorithmic_bytes_per_launch": BYTES_PER_POINT_CYCLE * n * n,
                         "kernel": kernel_name, "peak_kind": peak_kind},
            "e2e": {k: _r(v) for k, v in e2e.items()}, "gpu_launches": int(launches), "clocks": clk.summary()}
    if rank == 0 and not args.no_extras:
        cpu = cpu_baseline(k, gpu_counts={"f64_k16": extras["cfg2_k_sweep_512"]["f64_to_1e-06"]["k16"]["cycles"]})
        extras["cpu_baseline"] = cpu
        line["cpu_baseline"] = {"value": _r(cpu["value"]), "unit": "GLUP/s", "cores": cpu["cores"], "kind": "oracle",
                                "sample": cpu["sample"], "single_core": _r(cpu["single_core_glups"]),
                                "cfg1_to_1e-6_s": {a: _r(b["s"], 3) for a, b in cpu["cfg1_1d_to_1e-6"].items()},
                                "cfg2_f64_to_1e-6_s_projected": {
                                    a: _r(b["s_projected"], 3) for a, b in cpu["cfg2_512_f64_to_1e-6"].items()}}
        line.update(compact_summary(extras))
        try:
            os.makedirs(os.path.dirname(args.extras_out), exist_ok=True)
            with open(args.extras_out, "w") as fh:
                json.dump(dict(line, extras=extras), fh, indent=1)
        except OSError:
            pass
    solver.close()
    if rank == 0:
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def compact_summary(x):
    """The legs' key numbers for the JSON line (the full record goes to the
    extras file): [seconds, cycles, outer steps, host-recomputed relative
    residual] per solve, errors against the exact discrete solution."""
    t = x["time_to_1e-8_512"]

    def solve_row(r, err=False):
        row = [_r(r["s"], 3), r["cycles"], r["outer"], _r(r.get("rel", 0.0), 2)]
        if err:
            row.append(_r(r["err_vs_exact"], 2))
        return row

    out = {"time_to_1e-8_512": {"fields": "s,cycles,outer,rel",
                                "hj_f32ir_autotuned": solve_row(t["hj_f32ir_autotuned"]),
                                "hj_f32ir_32x32_k32": solve_row(t["hj_f32ir_32x32_k32"]),
                                "classic_f64_best": solve_row(t[t["classic_best"]]),
                                "classic_variant": t["classic_best"][12:],
                                "speedup": _r(t["speedup_autotuned_vs_classic"], 3)}}
    c3 = x["cfg3_precision_512"]
    out["cfg3_ir_to_1e-10_512"] = {"fields": "s,cycles,outer,rel,err_vs_exact",
                                   **{k: solve_row(v, True) for k, v in c3.items()}}
    sw = x["cfg2_k_sweep_512"]
    out["cfg2_k_sweep_512"] = {"fields": "s,cycles", **{p: {k: [_r(v["s"], 3), v["cycles"]] for k, v in row.items()}
                                                         for p, row in sw.items()}}
    fd = x["cfg5_fd_check"]
    out["cfg5_fd"] = {"grid": fd["grid"][0], "entries": fd["entries"], "step": fd["rel_step"],
                      "max_rel_err": _r(fd["max_rel_err"], 2), "s": _r(fd["fd_solves_s"], 3)}
    out["legs"] = {"classic_kernel_hbm_frac": _r(x["classic_global_jacobi"]["hbm_frac"], 3),
                   "inner_k16_alu_frac": _r(x["inner_sweep_roofline_k16"]["frac"], 3),
                   "inner_k16_smem_frac": _r(x["inner_sweep_roofline_k16"]["smem_path_frac"], 3),
                   "cfg1_gpu_speedup": _r(x["cfg1_1d_to_1e-6"]["speedup"], 3),
                   "cfg4_s": _r(x["cfg4_batched_256_to_1e-8"]["seconds"], 3),
                   "cfg4_graphed": x["cfg4_batched_256_to_1e-8"]["graphed"],
                   "cfg4_tail_s": _r(x["cfg4_batched_256_to_1e-8"]["tail_seconds"], 3),
                   "cfg5_fwd_bwd_s": [_r(x["cfg5_differentiation_1024"]["forward_seconds"], 3),
                                      _r(x["cfg5_differentiation_1024"]["backward_seconds"], 3)]}
    return out


if __name__ == "__main__":
    sys.exit(main())

"""Host-side logic of bench.py: the multi-rank timing reduction (gloo, two
ranks on the CPU), the whole-job rate, and the reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms = bench.max_over_ranks(10.0 * (rank + 1), "cpu")
    out.put((rank, ms, bench.job_rate(100.0, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the rate counts both ranks' units
    assert [r[1] for r in res] == [20.0, 20.0]
    assert res[0][2] == pytest.approx(2 * 100.0 / 0.020)


def test_reference_arm_prints_its_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--n", "1024"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GLUP/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_closed_form_sweep_count_and_sine_solve_of_the_bench():
    """The bench's classic sweep count (closed form in the sine basis) equals
    the oracle's count, and its sine-transform solution makes the host
    residual vanish."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import oracle
    import workloads as W
    p = W.poisson2d_uniform(40, 28, seed=3)
    n = bench.classic_sweeps_closed_form(p.st, p.f, 1e-3)
    _, c, status, _ = oracle.solve(p.st, p.f, p.u0, 1e-3, 10 ** 6, classic=True)
    assert status == 0 and n == c
    u = bench.dst_solution(p.st, p.f)
    assert bench.host_rel_residual(p.st, p.f, u) < 1e-12
    assert bench.host_rel_residual(p.st, p.f, p.u0) == 1.0
    assert np.allclose(bench.host_rel_residual(p.st, p.f, u * 0.5), 0.5)

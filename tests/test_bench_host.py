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


def test_compact_summary_fits_the_line_and_carries_every_leg():
    """The JSON line's summary of the extra legs, from a synthetic record with
    the keys the legs write: every leg present, rows rounded, and the whole
    line well inside the few kilobytes the bench's output tail keeps."""
    sys.path.insert(0, ROOT)
    import bench
    row = {"s": 0.123456, "cycles": 1234, "outer": 3, "rel": 2.5e-10, "err_vs_exact": 6.4e-12}
    sweep = {"k1": {"s": 1.0, "cycles": 10}, "k4": {"s": 0.5, "cycles": 5}, "classic": {"s": 2.0, "cycles": 20}}
    x = {"time_to_1e-8_512": {"hj_f32ir_autotuned": row, "hj_f32ir_32x32_k32": row, "classic_f64_tile_k1": row,
                              "classic_best": "classic_f64_tile_k1", "speedup_autotuned_vs_classic": 46.8},
         "cfg3_precision_512": {"f32_ir": row, "bf16corr_ir": row, "f64": row},
         "cfg2_k_sweep_512": {"f64_to_1e-06": sweep, "f32_to_1e-05": sweep},
         "cfg5_fd_check": {"grid": [1024, 1024], "entries": 32, "rel_step": 1e-6, "max_rel_err": 5.4e-6,
                           "fd_solves_s": 36.2},
         "classic_global_jacobi": {"hbm_frac": 0.9123},
         "inner_sweep_roofline_k16": {"frac": 0.4834, "smem_path_frac": 0.5118},
         "cfg1_1d_to_1e-6": {"speedup": 9.37},
         "cfg4_batched_256_to_1e-8": {"seconds": 2.66, "graphed": 1, "tail_seconds": 0.544},
         "cfg5_differentiation_1024": {"forward_seconds": 14.1, "backward_seconds": 14.6}}
    out = bench.compact_summary(x)
    assert out["time_to_1e-8_512"]["hj_f32ir_autotuned"] == [0.123, 1234, 3, 2.5e-10]
    assert out["cfg3_ir_to_1e-10_512"]["f32_ir"] == [0.123, 1234, 3, 2.5e-10, 6.4e-12]
    assert out["legs"]["inner_k16_smem_frac"] == 0.512 and out["legs"]["inner_k16_alu_frac"] == 0.483
    assert out["cfg5_fd"]["entries"] == 32 and out["cfg2_k_sweep_512"]["f32_to_1e-05"]["k4"] == [0.5, 5]
    assert len(json.dumps(out, separators=(",", ":"))) < 1500

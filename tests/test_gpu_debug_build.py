"""The debug build (libhj_debug.so: index checks in the kernels, guard bands
around device allocations) as a stand-in for a memory checker.

The library is compiled with -DHJ_DEBUG, its self-test must catch a planted
out-of-range index (checked, never accessed) and a host-written guard byte,
and then the tile-walk parity tests, the classic sweeps, the persistent and
batched engines and the refinement run against it in a child process, each
test followed by hj_debug_check (tests/conftest.py)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def debug_env():
    sys.path.insert(0, ROOT)
    from paper_2006_16465_gb300 import _build
    _build.build(debug=True)
    import __graft_entry__
    __graft_entry__.build()
    return dict(os.environ, HJ_LIBRARY="debug")


def test_debug_build_catches_what_it_checks(debug_env):
    code = ("import paper_2006_16465_gb300 as hj; assert hj.LIB_PATH.name == 'libhj_debug.so'; "
            "st = hj.hj_debug_selftest(); print('SELFTEST', st, hj.hj_last_error()); "
            "c, s, i = hj.hj_debug_check(); print('CLEAN', c, s, i)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=debug_env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    sel = [ln for ln in r.stdout.splitlines() if ln.startswith("SELFTEST")][0].split()
    assert sel[1] == "0", r.stdout
    clean = [ln for ln in r.stdout.splitlines() if ln.startswith("CLEAN")][0].split()
    assert clean[1:3] == ["0", "0"], r.stdout


def test_3d_and_multigrid_suites_pass_the_debug_checks(debug_env):
    """The 3D kernels (binary64 one column per lane, binary32 two columns per
    lane with the halo folded into f/d, the prefetching variant) and the
    multigrid V-cycles (smoothing launches that form the coarse RHS or stage
    the prolongation themselves) under the guard bands of every device
    allocation, checked after each test."""
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_gpu_3d.py", "tests/test_gpu_mg.py",
                        "-m", "gpu", "-q", "-p", "no:cacheprovider", "-x"],
                       cwd=ROOT, env=debug_env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join(r.stdout.splitlines()[-15:])
    assert r.returncode == 0, tail + r.stderr[-2000:]
    assert " passed" in tail


def test_parity_suites_pass_the_debug_checks(debug_env):
    sel = ("tile_walk or classic or batched or pipelined or persistent or refinement or f64_cycles_match_oracle_1d "
           "or launch_shapes")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_gpu_tilewalk.py", "tests/test_gpu_parity.py",
                        "-m", "gpu", "-k", sel, "-q", "-p", "no:cacheprovider", "-x"],
                       cwd=ROOT, env=debug_env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join(r.stdout.splitlines()[-15:])
    assert r.returncode == 0, tail + r.stderr[-2000:]
    assert " passed" in tail

"""The C-ABI library loads and exports every entry point include/hj.h
declares; host-only entry points answer without a GPU."""
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def hj():
    from paper_2006_16465_gb300 import _build
    _build.build()
    import paper_2006_16465_gb300 as hj
    hj.lib()
    return hj


def declared_symbols():
    text = (ROOT / "include" / "hj.h").read_text()
    return sorted(set(re.findall(r"HJ_API[^;(]*?\b(hj_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["hj_create", "hj_solve", "hj_residual", "hj_solve_adjoint", "hj_solve_batched", "hj_destroy",
              "hj_error_string", "hj_last_error", "hj_default_params", "hj_tile_shapes"]:
        assert n in names


def test_library_exports_every_declared_symbol(hj):
    import ctypes
    lib = ctypes.CDLL(str(hj.LIB_PATH))
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_binding_has_same_names(hj):
    for n in declared_symbols():
        assert callable(getattr(hj, n)), n


def test_default_params_and_strings(hj):
    p = hj.hj_default_params()
    assert (p.tile_x, p.tile_y, p.k, p.precision, p.check_every) == (32, 32, 16, hj.HJ_PREC_F64, 64)
    assert p.tol == 1e-6 and p.max_outer == 60 and p.persistent == -1
    for code in range(0, 10):
        assert hj.hj_error_string(code) != "unknown status"
    assert hj.hj_error_string(99) == "unknown status"


def test_tile_shapes(hj):
    s64 = hj.hj_tile_shapes(2, hj.HJ_PREC_F64)
    s32 = hj.hj_tile_shapes(2, hj.HJ_PREC_F32)
    assert (32, 32) in s64 and (32, 32) in s32 and (64, 64) in s32
    assert (128, 1) in hj.hj_tile_shapes(1, hj.HJ_PREC_F64)
    assert hj.hj_tile_shapes(2, hj.HJ_PREC_BF16CORR_IR) == s32


def test_create_rejects_bad_descriptors_without_touching_the_gpu(hj):
    # argument validation happens before any CUDA call
    d = hj.make_desc(4, 10, 10, 32, -1, -1, -1, -1, 4)
    with pytest.raises(hj.HJError) as e:
        hj.hj_create(d, hj.make_params())
    assert e.value.code == hj.HJ_ERR_INVALID_ARG
    # 3D seven-point extension: planes, dominance over six neighbours, scope
    for kw, prm, code in [(dict(nz=0), {}, hj.HJ_ERR_INVALID_ARG),
                          (dict(nz=5, cB=-1, cT=-1), {}, hj.HJ_ERR_NOT_DIAG_DOMINANT),
                          (dict(nz=5, cB=-1, cT=-1, cD=6.0), dict(precision="f32_ir"), hj.HJ_ERR_UNSUPPORTED),
                          (dict(nz=5, cB=-1, cT=-1, cD=6.0), dict(overlap_x=2), hj.HJ_ERR_UNSUPPORTED),
                          (dict(nz=5, cB=-1, cT=-1, cD=6.0), dict(persistent=1), hj.HJ_ERR_UNSUPPORTED),
                          (dict(nz=5, cB=-1, cT=-1, cD=6.0), dict(tile_x=32, tile_y=32, tile_z=32),
                           hj.HJ_ERR_UNSUPPORTED)]:
        cD = kw.pop("cD", 4.0)
        d = hj.make_desc(3, 10, 10, 32, -1, -1, -1, -1, cD, **kw)
        with pytest.raises(hj.HJError) as e:
            hj.hj_create(d, hj.make_params(**prm))
        assert e.value.code == code, (kw, prm)
    d = hj.make_desc(2, 10, 10, 11, -1, -1, -1, -1, 4)     # ld < nx + 2
    with pytest.raises(hj.HJError) as e:
        hj.hj_create(d, hj.make_params())
    assert e.value.code == hj.HJ_ERR_INVALID_ARG
    d = hj.make_desc(2, 10, 10, 32, -1, -1, -1, -1, 3.9)   # not diagonally dominant
    with pytest.raises(hj.HJError) as e:
        hj.hj_create(d, hj.make_params())
    assert e.value.code == hj.HJ_ERR_NOT_DIAG_DOMINANT
    d = hj.make_desc(2, 10, 10, 32, -1, -1, -1, -1, 4, dtype=hj.HJ_F32)   # f32 data with f64 precision
    with pytest.raises(hj.HJError) as e:
        hj.hj_create(d, hj.make_params())
    assert e.value.code == hj.HJ_ERR_INVALID_ARG


def test_no_cpu_fallback(tmp_path, monkeypatch, hj):
    # with the library absent, the binding raises instead of computing anything
    import importlib
    monkeypatch.setattr(hj, "LIB_PATH", tmp_path / "missing.so")
    monkeypatch.setattr(hj, "_lib", None)
    with pytest.raises(RuntimeError):
        hj.lib()


def test_struct_layouts_match_the_header(tmp_path, hj):
    """Every field of hj_desc, hj_params and hj_stats sits at the same offset
    (and every struct has the same size) in the ctypes mirrors as in
    include/hj.h compiled by the C compiler."""
    import ctypes as C
    import subprocess
    from pathlib import Path
    root = Path(__file__).resolve().parents[1]
    structs = [hj.hj_desc, hj.hj_params, hj.hj_stats]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hj.h"', "int main(void) {"]
    for S in structs:
        lines.append(f'printf("{S.__name__} size %zu\\n", sizeof({S.__name__}));')
        for name, _ in S._fields_:
            lines.append(f'printf("{S.__name__} {name} %zu\\n", offsetof({S.__name__}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", str(root / "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            s, f, v = line.split()
            got[(s, f)] = int(v)
    for S in structs:
        assert got[(S.__name__, "size")] == C.sizeof(S), S.__name__
        for name, _ in S._fields_:
            assert got[(S.__name__, name)] == getattr(S, name).offset, (S.__name__, name)


def test_autotune_refuses_what_it_does_not_tune(hj):
    """3D descriptors, per-point coefficients and multigrid are refused
    before any GPU work."""
    import ctypes as C
    d3 = hj.make_desc(3, 16, 16, 32, -1, -1, -1, -1, 6.0, nz=8, cB=-1, cT=-1)
    dc = hj.make_desc(2, 16, 16, 32, -1, -1, -1, -1, 4.0)
    dc.coef = 4096   # never dereferenced: the refusal comes first
    d2 = hj.make_desc(2, 15, 15, 32, -1, -1, -1, -1, 4.0)
    for d, prm in [(d3, hj.make_params(autotune=1)), (dc, hj.make_params(autotune=1)),
                   (d2, hj.make_params(autotune=1, method="mg"))]:
        assert hj.lib().hj_autotune(C.byref(d), C.byref(prm), None) == hj.HJ_ERR_UNSUPPORTED


def test_noalloc_refuses_engines_that_need_workspace(hj):
    """hj_cycles_noalloc refuses in-place, persistent, pipelined and autotuned
    runs instead of ignoring them (the refusal comes before any CUDA call, so
    the fake pointers are never used)."""
    import ctypes as C
    st_d = hj.make_desc(2, 64, 64, 96, -1, -1, -1, -1, 4.0)
    for kw in (dict(in_place=1), dict(persistent=1), dict(pipeline=1), dict(autotune=1), dict(overlap_x=2)):
        prm = hj.make_params(fixed_cycles=1, precision="f64", **kw)
        code = hj.lib().hj_cycles_noalloc(C.byref(st_d), C.byref(prm), C.c_void_p(4096), C.c_void_p(8192), None)
        assert code == hj.HJ_ERR_UNSUPPORTED, kw


def test_release_build_reports_no_debug_checks(hj):
    """The release library compiles the memory checks away: hj_debug_check
    says so (site -1) and the self-test is refused; no GPU work either way."""
    code, site, _ = hj.hj_debug_check()
    assert code == hj.HJ_OK and site == -1
    assert hj.hj_debug_selftest() == hj.HJ_ERR_UNSUPPORTED

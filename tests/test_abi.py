"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h (CPU only: no compute call is made without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(mpml_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2602_07853_gb300 import build
    return build.build()


def test_header_declares_the_three_step_calls():
    names = declared_symbols()
    for n in ("mpml_create", "mpml_resample", "mpml_newton_step", "mpml_g2p", "mpml_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_library_loads_and_binding_matches_header(lib_path):
    lib = ctypes.CDLL(lib_path)
    for n in declared_symbols():
        assert hasattr(lib, n)
    import paper_2602_07853_gb300.mpml as m
    m.load()
    assert set(declared_symbols()) == set(m.EXPORTS), "binding and header disagree"
    # a pure host call: status strings
    assert m.load().mpml_status_str(m.ERR_OUT_OF_DOMAIN).decode().startswith("particle")


def test_struct_layouts_match_header(tmp_path):
    """Compile a tiny C program against include/mpml.h and compare sizeof/offsets with ctypes."""
    import paper_2602_07853_gb300.mpml as m
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "mpml.h"
int main(void){
 printf("%zu %zu %zu %zu %zu %zu\n", sizeof(mpml_scene_desc), sizeof(mpml_material), sizeof(mpml_particles),
        sizeof(mpml_solver_opts), sizeof(mpml_solve_stats), sizeof(mpml_pcg_config));
 printf("%zu %zu %zu %zu %zu\n", offsetof(mpml_scene_desc, plate_vel), offsetof(mpml_particles, perm),
        offsetof(mpml_solve_stats, g0_norm), offsetof(mpml_solve_stats, n_bricks),
        offsetof(mpml_solver_opts, cg_forcing));
 return 0;}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    lines = subprocess.check_output([str(exe)], text=True).split("\n")
    sizes = [int(v) for v in lines[0].split()]
    offs = [int(v) for v in lines[1].split()]
    assert sizes == [ctypes.sizeof(t) for t in (m.mpml_scene_desc, m.mpml_material, m.mpml_particles,
                                                 m.mpml_solver_opts, m.mpml_solve_stats, m.mpml_pcg_config)]
    assert offs == [m.mpml_scene_desc.plate_vel.offset, m.mpml_particles.perm.offset,
                    m.mpml_solve_stats.g0_norm.offset, m.mpml_solve_stats.n_bricks.offset,
                    m.mpml_solver_opts.cg_forcing.offset]


def test_noalloc_sort_rejects_on_the_host(lib_path):
    """Argument and capacity checks of mpml_sort_particles_noalloc run before any CUDA call."""
    import paper_2602_07853_gb300.mpml as m
    lib = m.load()
    f = lib.mpml_sort_particles_noalloc
    dummy = ctypes.c_void_p(256)  # never dereferenced: every case below returns before any launch
    n_ok, n_big = (ctypes.c_int * 3)(127, 127, 127), (ctypes.c_int * 3)(128, 127, 127)
    assert f(n_big, 128.0, m.FP32, dummy, 10, dummy, None, None) == m.ERR_TOO_LARGE
    assert f(n_ok, 128.0, m.FP32, dummy, 0, None, None, None) == m.OK
    assert f(n_ok, 128.0, m.FP32, None, 10, dummy, None, None) == m.ERR_ARG
    assert f(n_ok, 128.0, m.FP32, dummy, 10, None, None, None) == m.ERR_ARG
    assert f(n_ok, 128.0, 7, dummy, 10, dummy, None, None) == m.ERR_ARG
    assert f(n_ok, 0.0, m.FP32, dummy, 10, dummy, None, None) == m.ERR_ARG
    assert f(n_ok, 128.0, m.FP32, dummy, 1 << 31, dummy, None, None) == m.ERR_ARG
    assert f((ctypes.c_int * 3)(1, 8, 8), 128.0, m.FP32, dummy, 10, dummy, None, None) == m.ERR_ARG
    assert lib.mpml_status_str(m.ERR_TOO_LARGE).decode().startswith("size above")


def test_lame_parameters_in_the_library(lib_path):
    """mpml_lame_parameters (host code): the pair it returns gives back E and nu through the
    inverse relations E = mu (3 lambda + 2 mu) / (lambda + mu), nu = lambda / (2 (lambda + mu));
    invalid moduli are rejected."""
    import paper_2602_07853_gb300.mpml as m
    for E, nu in ((1e5, 0.3), (1e8, 0.33), (5e5, 0.0), (1e6, 0.45), (2e3, -0.2)):
        mu, lam = m.mpml_lame_parameters(E, nu)
        assert abs(mu * (3 * lam + 2 * mu) / (lam + mu) - E) <= 1e-12 * E
        assert abs(lam / (2 * (lam + mu)) - nu) <= 1e-12
    for E, nu in ((0.0, 0.3), (1e5, 0.5), (1e5, -1.0), (float("nan"), 0.3)):
        with pytest.raises(m.MPMLError) as e:
            m.mpml_lame_parameters(E, nu)
        assert e.value.code == m.ERR_ARG


def test_pcg_config_rejects_on_the_host(lib_path):
    import paper_2602_07853_gb300.mpml as m
    lib = m.load()
    cfg = m.mpml_pcg_config()
    assert lib.mpml_set_pcg_config(None, ctypes.byref(cfg)) == m.ERR_ARG
    assert lib.mpml_get_pcg_config(None, ctypes.byref(cfg), None, None) == m.ERR_ARG
    assert lib.mpml_autotune_pcg(None, 10, 1, None, None) == m.ERR_ARG

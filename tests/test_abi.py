"""The C-ABI library builds, loads and exports every symbol include/swof.h
declares; the Python structs mirror the header's layout (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1307_4839_gb300 as sw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swof.h")


@pytest.fixture(scope="module")
def lib():
    sw.build()
    return sw.load()


def header_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"SWOF_API\s+[\w\s\*]*?\b(swof_\w+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = header_functions()
    for must in ("swof_create", "swof_set_state", "swof_step", "swof_get_state", "swof_destroy",
                 "swof_set_dt_sequence", "swof_get_diagnostics", "swof_set_state_device",
                 "swof_get_state_device", "swof_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    so = sw.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(swof_\w+)", out))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing
    # the binding declares the same set
    assert set(sw.declared_symbols()) == set(header_functions())
    for n in header_functions():
        assert hasattr(lib, n)


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "swof.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(swof_params), offsetof(swof_params, bc),
         offsetof(swof_params, friction_map), offsetof(swof_params, ks_map),
         offsetof(swof_params, dt_fixed), offsetof(swof_params, stream), offsetof(swof_params, friction_coef),
         offsetof(swof_params, order), offsetof(swof_params, bc_h), offsetof(swof_params, bc_q));
  printf("%zu %zu\\n", sizeof(swof_step_info), offsetof(swof_step_info, status));
  printf("%zu %zu %zu\\n", sizeof(swof_diag), offsetof(swof_diag, min_h), offsetof(swof_diag, cfl_viol));
  printf("%zu %zu %zu\\n", sizeof(swof_scenario), offsetof(swof_scenario, manning_n), offsetof(swof_scenario, bc));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [list(map(int, l.split())) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                               check=True).stdout.strip().splitlines()]
    P = sw.SwofParams
    assert vals[0] == [ctypes.sizeof(P), P.bc.offset, P.friction_map.offset, P.ks_map.offset,
                       P.dt_fixed.offset, P.stream.offset, P.friction_coef.offset, P.order.offset,
                       P.bc_h.offset, P.bc_q.offset]
    assert vals[1] == [ctypes.sizeof(sw.SwofStepInfo), sw.SwofStepInfo.status.offset]
    assert vals[2] == [ctypes.sizeof(sw.SwofDiag), sw.SwofDiag.min_h.offset, sw.SwofDiag.cfl_viol.offset]
    assert vals[3] == [ctypes.sizeof(sw.SwofScenario), sw.SwofScenario.manning_n.offset, sw.SwofScenario.bc.offset]


def test_host_only_calls(lib):
    p = sw.default_params()
    assert p.g == 9.81 and p.cfl == 0.5 and p.h_dry == 1e-6 and p.precision == sw.FP64
    assert lib.swof_strerror(-7) == b"replayed dt sequence exhausted"
    assert b"sm_103a" in lib.swof_version()
    lib.swof_destroy(None)   # NULL-safe


def test_create_rejects_bad_arguments_before_touching_a_device(lib):
    import numpy as np
    z = np.zeros((4, 4))
    p = sw.default_params()
    ctx = ctypes.c_void_p()
    zp = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.swof_create(1, 4, 1.0, 1.0, zp, ctypes.byref(p), ctypes.byref(ctx)) == sw.EINVAL
    assert lib.swof_create(4, 4, -1.0, 1.0, zp, ctypes.byref(p), ctypes.byref(ctx)) == sw.EINVAL
    p.bc[2] = 7
    assert lib.swof_create(4, 4, 1.0, 1.0, zp, ctypes.byref(p), ctypes.byref(ctx)) == sw.EINVAL
    p = sw.default_params(bc=(sw.BC_IMPOSED_Q, 0, 0, 0), bc_q=(-1.0, 0, 0, 0))     # inflow only
    assert lib.swof_create(4, 4, 1.0, 1.0, zp, ctypes.byref(p), ctypes.byref(ctx)) == sw.EINVAL
    p = sw.default_params(friction=sw.FRIC_CHEZY, friction_coef=0.0)              # C = 0
    assert lib.swof_create(4, 4, 1.0, 1.0, zp, ctypes.byref(p), ctypes.byref(ctx)) == sw.EINVAL
    p = sw.default_params(friction=5)
    assert lib.swof_create(4, 4, 1.0, 1.0, zp, ctypes.byref(p), ctypes.byref(ctx)) == sw.EINVAL
    p = sw.default_params(order=3)
    assert lib.swof_create(4, 4, 1.0, 1.0, zp, ctypes.byref(p), ctypes.byref(ctx)) == sw.EINVAL
    assert lib.swof_flow_directions(None, 4, 4, None, None, None) == sw.EINVAL
    p = sw.default_params(precision=3)
    assert lib.swof_create(4, 4, 1.0, 1.0, zp, ctypes.byref(p), ctypes.byref(ctx)) == sw.EINVAL
    zn = np.full((4, 4), np.nan)
    p = sw.default_params()
    assert lib.swof_create(4, 4, 1.0, 1.0, zn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           ctypes.byref(p), ctypes.byref(ctx)) == sw.ENONFINITE
    assert lib.swof_create(4, 4, 1.0, 1.0, zp, ctypes.byref(p), None) == sw.EINVAL


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1307_4839_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                code = re.sub(r"(#|//).*", "", txt)
                assert not re.search(r"\b(import|from)\s+oracle\b|liboracle|oracle_\w+\(|swof_oracle", code), f

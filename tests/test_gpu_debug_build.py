"""The index-checking debug build (libswof_debug.so, compiled with
SWOF_BOUNDS_CHECK): every padded-array index the stencil kernels form, every
ring slot the stage kernels read and every tensor-copy origin is checked on
the device, and a failed check latches SWOF_EBOUNDS (the access itself is
clamped to a valid element).  Small grids through that build must give the
oracle's results bit for bit (FP64) with no check failing, across the
stage-kernel forms (TMA ring with the dry fast path, register prefetch),
imposed edges, the first-order step and dry-tile skipping; and a failed
check must be reported (a probe that forms an out-of-range index through
the checked path).  Runs in a child process that loads the debug build."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
sys.path.insert(0, ROOT)
import numpy as np
import oracle
import paper_1307_4839_gb300 as sw
import swof_inputs as si

L = sw.load()
assert L.swof_debug_build() == 1, "not the debug build"
out = {"cases": 0}

def same(s, o, dts):
    assert np.array_equal(s.dt_history(), dts)
    for a, b in zip(s.state(), o.state()):
        assert np.array_equal(a, b)
    out["cases"] += 1

# ragged grid, wet/dry, outflow edges: ring shapes, register shapes, mixed
w = si.random_state(131, 77, seed=3, dry_frac=0.3)
w.bc = (0, 1, 0, 1)
o = oracle.Oracle.from_workload(w)
dts = o.step(10)
for shapes in ((0, 4), (5, 9), (2, 7), (3, 1)):
    s = sw.Solver.from_workload(w, sw.FP64)
    s.set_tile_shape(*shapes)
    assert s.step(10).status == 0
    same(s, o, dts)
    s.close()

# a mostly dry valley: the dry fast path of the ring kernels, and skipping
wv = si.valley(n=200, dx=2.0, seed=1)
ov = oracle.Oracle.from_workload(wv)
dv = ov.step(25)
for skip in (False, True):
    s = sw.Solver.from_workload(wv, sw.FP64)
    s.set_tile_shape(1, 1)
    s.set_dry_tile_skip(skip)
    assert s.step(25).status == 0
    same(s, ov, dv)
    s.close()

# imposed edges, Darcy-Weisbach, first order
over = dict(order=sw.ORDER_1, cfl=1.0, bc=(3, 2, 0, 1), bc_h=(0, 0.9, 0, 0), bc_q=(0.4, 0, 0, 0),
            friction=sw.FRIC_DARCY, friction_coef=0.5)
o1 = oracle.Oracle.from_workload(w, **over)
d1 = o1.step(8)
s = sw.Solver.from_workload(w, sw.FP64, **over)
assert s.step(8).status == 0
same(s, o1, d1)
s.close()

# FP32 through every form: no check fails
for shapes in ((0, 4), (5, 9)):
    s = sw.Solver.from_workload(wv, sw.FP32)
    s.set_tile_shape(*shapes)
    assert s.step(25).status == 0
    out["cases"] += 1
    s.close()

# the probe: an in-range cell passes, an out-of-range one latches EBOUNDS
s = sw.Solver.from_workload(w, sw.FP64)
out["probe_in"] = s.debug_probe_index(5, 7)
s2 = sw.Solver.from_workload(w, sw.FP64)
out["probe_out"] = s2.debug_probe_index(w.nx + 50, 3)
try:                                     # the status stays latched: the next step reports it
    s2.step(1)
    out["status_after"] = 0
except sw.SwofError as e:
    out["status_after"] = e.code
print(json.dumps(out))
'''


def test_debug_build_matches_oracle_and_reports_failed_checks():
    import paper_1307_4839_gb300 as sw
    sw.build(debug=True)
    env = dict(os.environ, SWOF_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["cases"] == 9
    assert out["probe_in"] == sw.OK
    assert out["probe_out"] == sw.EBOUNDS and out["status_after"] == sw.EBOUNDS

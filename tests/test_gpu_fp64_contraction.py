"""FP64 with multiply-add contraction (swof_set_fp64_contraction) against the
FP64 oracle (needs a GPU).

The contracted kernels round each fused a*b+c once instead of twice, so
they cannot equal the oracle bit for bit; the bar is relative L-inf <= 1e-12
per field after the same steps under an identical dt sequence (the oracle's
own, replayed).  Run on its own CFL dt, the contracted solver's dt sequence
and states stay within the same bar on the dam break to t = 1 s.
"""
import numpy as np
import pytest

import oracle
import paper_1307_4839_gb300 as sw
import swof_inputs as si

pytestmark = pytest.mark.gpu
BAR = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sw.build()
    sw.load()
    oracle.build()


def rel_linf(a, b):
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (s if s > 0 else 1.0))


def assert_close(s, o, bar=BAR):
    errs = [rel_linf(a, b) for a, b in zip(s.state(), o.state())]
    assert max(errs) <= bar, errs
    return errs


def replay_pair(w, steps=None, t_end=None, shapes=None, **over):
    """The oracle takes its own dt; the contracted solver replays it."""
    o = oracle.Oracle.from_workload(w, **over)
    dts = o.run_to(t_end) if t_end is not None else o.step(steps)
    s = sw.Solver.from_workload(w, sw.FP64, **over)
    s.set_fp64_contraction(True)
    if shapes is not None:
        s.set_tile_shape(*shapes)
    s.set_dt_sequence(dts)
    info = s.step(len(dts))
    assert info.status == 0 and info.steps == len(dts)
    assert np.array_equal(s.dt_history(), dts)
    return o, s, dts


def test_contracted_dam_break_200_to_t1_replayed_dt():
    o, s, _ = replay_pair(si.dam_break(200), t_end=1.0)
    assert s.diagnostics()["t"] == 1.0
    assert_close(s, o)


def test_contracted_dam_break_200_to_t1_own_dt():
    """Its own CFL dt: the sequence differs from the oracle's only in the
    last bits and the states stay within the bar."""
    w = si.dam_break(200)
    o = oracle.Oracle.from_workload(w)
    dts = o.run_to(1.0)
    s = sw.Solver.from_workload(w, sw.FP64)
    s.set_fp64_contraction(True)
    info = s.step(len(dts))
    assert info.t == 1.0 and info.status == 0
    assert np.max(np.abs(s.dt_history() - dts) / dts) <= BAR
    assert_close(s, o)


@pytest.mark.parametrize("seed,nx,ny,bc", [(1, 100, 77, (0, 1, 0, 1)), (2, 67, 41, (1, 0, 1, 0)),
                                           (3, 33, 9, (1, 1, 1, 1)), (4, 130, 17, (0, 0, 0, 0))])
def test_contracted_ragged_random_wet_dry_60_steps(seed, nx, ny, bc):
    w = si.random_state(nx, ny, seed=seed, dry_frac=0.25, vel=0.8)
    w.bc = bc
    o, s, _ = replay_pair(w, 60)
    assert_close(s, o)
    d, od = s.diagnostics(), o.diag()
    assert abs(d["volume"] - od["volume"]) <= BAR * od["volume"]


def test_contracted_rain_green_ampt_ks_map():
    w = si.hillslope(n=96, dx=1.0, rain_mm_h=120.0, rain_s=40.0, t_end=80.0)
    w.bc = (0, 1, 0, 1)
    o, s, _ = replay_pair(w, t_end=80.0)
    assert_close(s, o)
    assert rel_linf(s.infiltrated(), o.vinf()) <= BAR
    d, od = s.diagnostics(), o.diag()
    for k in ("volume", "rain_in", "infiltrated", "outflow"):
        assert abs(d[k] - od[k]) <= BAR * max(abs(od[k]), 1e-30), k


def test_contracted_valley_256_150_steps():
    o, s, _ = replay_pair(si.valley(n=256, dx=2.0, seed=5, reservoir=20.0), 150)
    assert_close(s, o)


def test_contracted_first_order_imposed_edges():
    w = si.random_state(100, 77, seed=41, dry_frac=0.25, vel=0.8)
    o, s, _ = replay_pair(w, 70, order=sw.ORDER_1, cfl=1.0, bc=(3, 2, 1, 0), bc_h=(0, 0.9, 0, 0),
                          bc_q=(0.4, 0, 0, 0))
    assert_close(s, o)


@pytest.mark.parametrize("shape", range(10))
def test_contracted_every_tile_shape(shape):
    w = si.random_state(300, 150, seed=40 + shape, dry_frac=0.2)
    w.bc = (1, 0, 0, 1)
    o, s, _ = replay_pair(w, 12, shapes=(shape, (shape + 3) % 10))
    assert_close(s, o)


def test_contracted_full_size_valley_4096_first_steps():
    o, s, _ = replay_pair(si.valley(4096), 3)
    assert_close(s, o)


def test_contraction_switches_back_to_bitwise_and_rejects_fp32():
    """Switched on and off again before stepping, the solver is the
    bit-exact one; an FP32 context has no FP64 kernels to switch."""
    w = si.random_state(70, 50, seed=9, dry_frac=0.1)
    o = oracle.Oracle.from_workload(w)
    dts = o.step(20)
    s = sw.Solver.from_workload(w, sw.FP64)
    s.set_fp64_contraction(True)
    s.set_fp64_contraction(False)
    s.step(20)
    assert np.array_equal(s.dt_history(), dts)
    for a, b in zip(s.state(), o.state()):
        assert np.array_equal(a, b)
    f = sw.Solver.from_workload(w, sw.FP32)
    with pytest.raises(sw.SwofError) as e:
        f.set_fp64_contraction(True)
    assert e.value.code == sw.EINVAL

"""CUDA path vs the FP64 oracle for the extensions (needs a GPU), through the
C ABI: the friction laws of Sec. 2.1, the imposed (Riemann-invariant)
edges of Sec. 2.2, the first-order variant of Sec. 3.3, gauges and the
maximum depth, dry-tile skipping, and the D8 flow direction of Sec. 5.2.

FP64 states, dt sequences, gauge records and maximum depths must agree with
the oracle bit for bit; FP32 by relative L1 (<= 1e-5 on depths); D8 codes
exactly.  Grids span several tiles with ragged tails.
"""
import numpy as np
import pytest

import oracle
import paper_1307_4839_gb300 as sw
import swof_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sw.build()
    sw.load()
    oracle.build()


def rel_l1(a, b):
    s = np.sum(np.abs(b))
    return np.sum(np.abs(a - b)) / (s if s > 0 else 1.0)


def pair(w, steps, precision=sw.FP64, **over):
    o = oracle.Oracle.from_workload(w, **over)
    s = sw.Solver.from_workload(w, precision, **over)
    dts = o.step(steps)
    if precision == sw.FP32:
        s.set_dt_sequence(dts)
    info = s.step(steps)
    assert info.status == 0 and info.steps == steps
    return o, s, dts


def assert_bitwise(o, s, dts):
    assert np.array_equal(s.dt_history(), dts)
    for a, b, name in zip(s.state(), o.state(), ("h", "qx", "qy")):
        assert np.array_equal(a, b), f"{name}: max |diff| {np.max(np.abs(a - b)):.3e}"


# ------------------------------------------------------------------ friction laws

@pytest.mark.parametrize("law,coef", [(sw.FRIC_STRICKLER, 30.0), (sw.FRIC_DARCY, 0.6),
                                      (sw.FRIC_CHEZY, 12.0), (sw.FRIC_MANNING, 0.05)])
def test_fp64_friction_laws_bitwise(law, coef):
    w = si.random_state(77, 45, seed=21, dry_frac=0.25, vel=0.9)
    o, s, dts = pair(w, 60, friction=law, friction_coef=coef)
    assert_bitwise(o, s, dts)


def test_fp64_friction_coefficient_map_bitwise():
    w = si.random_state(66, 38, seed=22, dry_frac=0.2, vel=0.8)
    fmap = 0.2 + np.random.default_rng(5).random((w.ny, w.nx))
    o = oracle.Oracle.from_workload(w, friction=sw.FRIC_DARCY, friction_coef=0.0, n_map=fmap)
    s = sw.Solver.from_workload(w, sw.FP64, friction=sw.FRIC_DARCY, friction_coef=0.0, friction_map=fmap)
    dts = o.step(50)
    assert s.step(50).status == 0
    assert_bitwise(o, s, dts)


def test_fp32_friction_laws_rel_l1():
    w = si.random_state(96, 64, seed=23, dry_frac=0.15, vel=0.7)
    for law, coef in ((sw.FRIC_DARCY, 0.6), (sw.FRIC_CHEZY, 12.0), (sw.FRIC_STRICKLER, 30.0)):
        o, s, _ = pair(w, 40, sw.FP32, friction=law, friction_coef=coef)
        (h, qx, qy), (ho, qxo, qyo) = s.state(), o.state()
        assert rel_l1(h, ho) <= 1e-5 and rel_l1(qx, qxo) <= 1e-4 and rel_l1(qy, qyo) <= 1e-4


# ------------------------------------------------------------------ imposed edges

IMPOSED = [
    ((3, 2, 0, 1), (0, 0.9, 0, 0), (0.4, 0, 0, 0)),
    ((2, 3, 4, 0), (1.1, 0, 0.6, 0), (0, 0.3, 4.0, 0)),
    ((0, 1, 3, 2), (0, 0, 0, 0.8), (0, 0, 0.5, 0)),
    ((4, 1, 1, 3), (0.5, 0, 0, 0), (5.0, 0, 0, 0.2)),
]


@pytest.mark.parametrize("bc,bc_h,bc_q", IMPOSED)
def test_fp64_imposed_edges_bitwise(bc, bc_h, bc_q):
    w = si.random_state(69, 43, seed=31, dry_frac=0.2, vel=0.6)
    o, s, dts = pair(w, 80, bc=bc, bc_h=bc_h, bc_q=bc_q)
    assert_bitwise(o, s, dts)
    d, od = s.diagnostics(), o.diag()
    assert abs(d["volume"] - od["volume"]) <= 1e-12 * od["volume"]
    assert abs(d["outflow"] - od["outflow"]) <= 1e-11 * max(abs(od["outflow"]), 1e-12)


def test_fp64_torrential_inflow_fills_dry_channel_bitwise():
    nx, ny = 140, 10
    z = np.zeros((ny, nx))
    o = oracle.Oracle(nx, ny, 1.0, 1.0, z, bc=(4, 1, 0, 0), bc_h=(0.5, 0, 0, 0), bc_q=(5.0, 0, 0, 0),
                      dt_max=1.0)
    s = sw.Solver(nx, ny, 1.0, 1.0, z, bc=(4, 1, 0, 0), bc_h=(0.5, 0, 0, 0), bc_q=(5.0, 0, 0, 0),
                  dt_max=1.0)
    zero = np.zeros((ny, nx))
    o.set_state(zero, zero, zero)
    s.set_state(zero, zero, zero)
    dts = o.step(120)
    assert s.step(120).status == 0
    assert_bitwise(o, s, dts)
    assert dts[0] < 0.1                      # the boundary state set the first dt


def test_fp32_imposed_edges_rel_l1():
    bc, bc_h, bc_q = IMPOSED[1]
    w = si.random_state(96, 70, seed=32, dry_frac=0.1, vel=0.5)
    o, s, _ = pair(w, 60, sw.FP32, bc=bc, bc_h=bc_h, bc_q=bc_q)
    (h, qx, qy), (ho, qxo, qyo) = s.state(), o.state()
    assert rel_l1(h, ho) <= 1e-5 and rel_l1(qx, qxo) <= 2e-4 and rel_l1(qy, qyo) <= 2e-4


# ------------------------------------------------------------------ first order

@pytest.mark.parametrize("nx,ny,bc", [(100, 77, (0, 1, 0, 1)), (67, 130, (3, 2, 1, 0)), (33, 9, (1, 1, 1, 1))])
def test_fp64_first_order_bitwise(nx, ny, bc):
    w = si.random_state(nx, ny, seed=41, dry_frac=0.25, vel=0.8)
    o, s, dts = pair(w, 70, order=sw.ORDER_1, cfl=1.0, bc=bc, bc_h=(0, 0.9, 0, 0), bc_q=(0.4, 0, 0, 0))
    assert_bitwise(o, s, dts)
    d, od = s.diagnostics(), o.diag()
    assert abs(d["volume"] - od["volume"]) <= 1e-12 * od["volume"]
    assert abs(d["outflow"] - od["outflow"]) <= 1e-11 * max(abs(od["outflow"]), 1e-12)


def test_fp64_first_order_rain_green_ampt_and_cfl_check_bitwise():
    w = si.hillslope(n=96, dx=1.0)
    over = dict(order=sw.ORDER_1, cfl=1.0, check_cfl=1, friction=sw.FRIC_CHEZY, friction_coef=20.0)
    o = oracle.Oracle.from_workload(w, **over)
    s = sw.Solver.from_workload(w, sw.FP64, **over)
    dts = o.step(150)
    assert s.step(150).status == 0
    assert_bitwise(o, s, dts)
    assert np.array_equal(s.infiltrated(), o.vinf())
    d, od = s.diagnostics(), o.diag()
    assert d["cfl_viol"] == od["cfl_viol"]
    assert abs(d["infiltrated"] - od["infiltrated"]) <= 1e-10 * max(od["infiltrated"], 1e-30)
    assert d["rain_in"] == pytest.approx(od["rain_in"], rel=1e-13)


def test_fp32_first_order_dam_break_rel_l1():
    w = si.dam_break(200)
    o, s, _ = pair(w, 150, sw.FP32, order=sw.ORDER_1, cfl=1.0)
    (h, qx, _), (ho, qxo, _) = s.state(), o.state()
    assert rel_l1(h, ho) <= 1e-5 and rel_l1(qx, qxo) <= 1e-4


def test_first_order_graph_replay_equals_stream_launches():
    w = si.random_state(80, 60, seed=43, dry_frac=0.2)
    res = []
    for graph in (False, True):
        s = sw.Solver.from_workload(w, sw.FP64, order=sw.ORDER_1, cfl=1.0)
        s.use_graph(graph)
        for _ in range(3):
            s.step(20)
        res.append((s.state(), s.dt_history()))
    for a, b in zip(res[0][0], res[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(res[0][1], res[1][1])


# ------------------------------------------------------------------ gauges and maximum depth

@pytest.mark.parametrize("order", [sw.ORDER_2, sw.ORDER_1])
def test_fp64_gauges_and_max_depth_bitwise(order):
    w = si.random_state(90, 70, seed=51, dry_frac=0.2, vel=1.0)
    cells = [(0, 0), (89, 69), (45, 33), (12, 60), (45, 33)]
    cfl = 1.0 if order == sw.ORDER_1 else 0.5
    o = oracle.Oracle.from_workload(w, order=order, cfl=cfl)
    s = sw.Solver.from_workload(w, sw.FP64, order=order, cfl=cfl)
    o.track_max(True)
    s.track_max_depth(True)
    o.set_gauges(cells, 40)
    s.set_gauges(cells, 40)
    o.step(55)
    s.use_graph(True)
    for _ in range(5):
        assert s.step(11).status == 0
    g, og = s.gauges(), o.gauges()
    assert g.shape == og.shape == (40, 1 + 3 * len(cells))
    assert np.array_equal(g, og)
    assert np.array_equal(s.max_depth(), o.max_depth())


def test_fp32_gauges_follow_state():
    w = si.random_state(64, 48, seed=52, dry_frac=0.1)
    s = sw.Solver.from_workload(w, sw.FP32)
    cells = [(3, 4), (60, 40)]
    s.set_gauges(cells, 100)
    s.track_max_depth(True)
    hm = s.state()[0].copy()
    for k in range(5):
        s.step(1)
        h, qx, qy = s.state()
        hm = np.maximum(hm, h)
        r = s.gauges()[k]
        assert r[1] == h[4, 3] and r[2] == qx[4, 3] and r[6] == qy[40, 60]
        assert r[0] == s.diagnostics()["t"]
    assert np.array_equal(s.max_depth(), hm)


def test_rejected_gauges_keep_the_earlier_ones():
    """A gauge set with a cell outside the grid is rejected before anything
    changes: the earlier gauges go on recording."""
    w = si.random_state(40, 30, seed=62, dry_frac=0.2)
    s = sw.Solver.from_workload(w, sw.FP64)
    s.set_gauges([(3, 4)], 10)
    with pytest.raises(sw.SwofError) as e:
        s.set_gauges([(3, 4), (40, 0)], 10)          # i = nx: outside
    assert e.value.code == sw.EINVAL
    for _ in range(3):
        s.step(1)
    g = s.gauges()
    h, qx, qy = s.state()
    assert g.shape == (3, 4)
    assert g[-1][1] == h[4, 3] and g[-1][2] == qx[4, 3] and g[-1][3] == qy[4, 3]


def test_rejected_dt_sequence_keeps_the_previous_replay():
    """A replay rejected for a non-finite value changes nothing: the steps
    that follow take the earlier sequence (the oracle's, so the state is
    bit for bit the oracle's), and running past its end latches
    SWOF_EDTSEQ."""
    w = si.random_state(40, 30, seed=61, dry_frac=0.2)
    o = oracle.Oracle.from_workload(w)
    dts = o.step(4)
    s = sw.Solver.from_workload(w, sw.FP64)
    s.set_dt_sequence(dts)
    with pytest.raises(sw.SwofError) as e:
        s.set_dt_sequence([1e-3, float("nan")])
    assert e.value.code == sw.ENONFINITE
    assert s.step(4).status == 0
    assert_bitwise(o, s, dts)
    with pytest.raises(sw.SwofError) as e:
        s.step(1)
    assert e.value.code == sw.EDTSEQ


# ------------------------------------------------------------------ dry-tile skipping

@pytest.mark.parametrize("precision", [sw.FP64, sw.FP32])
def test_dry_tile_skip_is_bitwise_the_full_step(precision):
    """A mostly dry valley (pool behind a dam): with skipping on, states, dt
    and maximum depth equal the full step's bit for bit, while most tiles
    are skipped; FP64 also equals the oracle."""
    w = si.valley(n=768, dx=2.0, seed=1)
    runs = []
    for skip in (False, True):
        s = sw.Solver.from_workload(w, precision)
        s.set_tile_shape(1)
        s.track_max_depth(True)
        if skip:
            s.set_dry_tile_skip(True)
        for _ in range(4):
            assert s.step(40).status == 0
        runs.append((s.state(), s.dt_history(), s.max_depth(), s.tile_activity() if skip else None))
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][2], runs[1][2])
    live, total = runs[1][3]
    assert 0 < live < 0.6 * total
    if precision == sw.FP64:
        o = oracle.Oracle.from_workload(w)
        o.step(160)
        for a, b in zip(runs[1][0], o.state()):
            assert np.array_equal(a, b)


def test_dry_tile_skip_with_rain_spell_inflow_and_outflow():
    """Rain that stops, an imposed inflow into a dry corner, Green-Ampt and
    an outflow edge: skipping stays exact through tiles that wet, dry and
    turn live again (FP64 vs the oracle, bit for bit)."""
    w = si.hillslope(n=200, dx=1.0)
    h0 = np.zeros_like(w.h)
    h0[150:170, 20:60] = 0.3
    over = dict(rain_t_on=0.0, rain_t_off=3.0, bc=(3, 0, 0, 1), bc_q=(0.2, 0, 0, 0), dt_max=0.05)
    o = oracle.Oracle.from_workload(w, **over)
    o.set_state(h0, 0 * h0, 0 * h0)
    s = sw.Solver.from_workload(w, sw.FP64, **over)
    s.set_state(h0, 0 * h0, 0 * h0)
    s.set_dry_tile_skip(True)
    dts = o.step(200)
    for _ in range(4):
        assert s.step(50).status == 0
    assert_bitwise(o, s, dts)
    assert np.array_equal(s.infiltrated(), o.vinf())


# ------------------------------------------------------------------ D8 flow direction

@pytest.mark.parametrize("nx,ny", [(128, 64), (516, 257), (260, 70), (37, 21), (130, 7), (1, 5), (4, 1), (12, 3)])
def test_d8_matches_oracle_exactly(nx, ny):
    import torch
    for quantum, frac in ((0.0, 0.0), (0.25, 0.05)):
        z = si.dem(nx, ny, seed=nx + ny, quantum=quantum, nodata_frac=frac)
        zt = torch.from_numpy(z).cuda()
        for nodata in (None, -9999.0, 0.5):
            got = sw.flow_directions(zt, nodata=nodata).cpu().numpy()
            assert np.array_equal(got, oracle.d8(z, nodata)), (quantum, nodata)
    zi = si.dem(nx, ny, seed=3)
    zi.flat[:: 7] = -np.inf
    zi.flat[3:: 11] = np.nan
    got = sw.flow_directions(torch.from_numpy(zi).cuda()).cpu().numpy()
    assert np.array_equal(got, oracle.d8(zi))


def test_d8_full_size_sampled_rows():
    """The 16384 x 16384 DEM of the benchmark: every row band's first and
    last rows and a sample of interior rows against the oracle on those rows
    (the oracle takes the rows with their neighbours)."""
    import torch
    n = 16384
    z = si.dem(n, n, seed=7, quantum=0.01)
    zt = torch.from_numpy(z).cuda()
    d = sw.flow_directions(zt).cpu().numpy()
    rng = np.random.default_rng(0)
    rows = sorted(set([0, 1, 63, 64, 65, n - 2, n - 1] + list(rng.integers(0, n, 24))))
    for j in rows:
        a, b = max(j - 1, 0), min(j + 2, n)      # the row with all of its neighbour rows
        assert np.array_equal(d[j], oracle.d8(z[a:b])[j - a]), j


# ------------------------------------------------------------------ the bench's size

def test_fp64_full_size_first_order_with_imposed_edge_bitwise():
    """The 4096^2 valley at first order (n_CFL 1) with an imposed inflow on
    the west edge and an imposed depth on the east edge, against the oracle
    over its first 3 steps (whole grid, bit for bit)."""
    w = si.valley(4096)
    over = dict(order=sw.ORDER_1, cfl=1.0, bc=(3, 2, 0, 1), bc_q=(0.5, 0, 0, 0), bc_h=(0, 0.2, 0, 0))
    o, s, dts = pair(w, 3, **over)
    assert_bitwise(o, s, dts)


def test_fp32_full_size_first_order_against_oracle_dt():
    """The first-order FP32 variant the benchmark times, on the oracle's dt:
    relative L1 of h <= 1e-5 and of the down-valley discharge <= 1e-4."""
    w = si.valley(4096)
    o, s, _ = pair(w, 6, sw.FP32, order=sw.ORDER_1, cfl=1.0)
    (h, qx, qy), (oh, oqx, oqy) = s.state(), o.state()
    assert rel_l1(h, oh) <= 1e-5 and rel_l1(qy, oqy) <= 1e-4
    assert h.min() >= 0.0


def test_full_size_dry_tile_skip_equals_full_step():
    """Dry-tile skipping on the benchmark's 4096^2 valley (FP32, the shape
    skipping selects): 60 steps give the full step's state and dt sequence
    bit for bit."""
    w = si.valley(4096)
    res = []
    for skip in (False, True):
        s = sw.Solver.from_workload(w, sw.FP32)
        if skip:
            s.set_dry_tile_skip(True)
        for _ in range(3):
            assert s.step(20).status == 0
        res.append((s.state(), s.dt_history(), s.tile_activity() if skip else None))
        s.close()
    for a, b in zip(res[0][0], res[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(res[0][1], res[1][1])
    live, total = res[1][2]
    assert 0 < live < 0.2 * total

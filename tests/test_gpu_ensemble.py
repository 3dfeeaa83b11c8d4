"""Batched ensemble (one persistent launch over many grids) vs its members
stepped one by one and vs the FP64 oracle (needs a GPU).

FP64 members are compiled without contraction, so the ensemble must equal
both the single-grid path and the oracle bit for bit.  FP32 members may be
contracted differently in the two kernels (the arithmetic is inlined in
different places), so they are compared to rounding.
"""
import numpy as np
import pytest

import oracle
import paper_1307_4839_gb300 as sw
import swof_inputs as si

pytestmark = pytest.mark.gpu

SIDES = [32, 48, 64, 96, 130, 160, 40, 72]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    sw.build()
    sw.load()
    oracle.build()


def members(seed=4, sides=SIDES):
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate(sides):
        spec = si.Scenario(side=n, reservoir=float(rng.uniform(5, 40)), manning_n=float(rng.uniform(0.02, 0.06)),
                           rain_mm_h=float(rng.uniform(0, 80)), seed=500 + k)
        out.append(si.ensemble_member(spec))
    return out


def test_fp64_ensemble_equals_members_and_oracle():
    ws = members()
    ens = sw.Ensemble(ws, precision=sw.FP64)
    assert ens.step(25) == 0
    for k, w in enumerate(ws):
        m = ens.member(k)
        solo = sw.Solver.from_workload(w, sw.FP64)
        solo.step(25)
        for a, b in zip(m.state(), solo.state()):
            assert np.array_equal(a, b), k
        assert np.array_equal(m.dt_history(), solo.dt_history()), k
        if k in (0, 4, 5):
            o = oracle.Oracle.from_workload(w)
            dts = o.step(25)
            assert np.array_equal(m.dt_history(), dts), k
            for a, b in zip(m.state(), o.state()):
                assert np.array_equal(a, b), k


def test_fp32_ensemble_matches_members_and_graph_replay():
    ws = members(seed=9)
    ens = sw.Ensemble(ws, precision=sw.FP32)
    for _ in range(3):
        assert ens.step(10) == 0       # the second and third calls replay the graph
    for k, w in enumerate(ws):
        m = ens.member(k)
        solo = sw.Solver.from_workload(w, sw.FP32)
        solo.step(30)
        d1, d2 = m.diagnostics(), solo.diagnostics()
        assert d1["steps"] == d2["steps"] == 30
        assert abs(d1["t"] - d2["t"]) <= 1e-6 * d2["t"]
        for a, b in zip(m.state(), solo.state()):
            scale = max(np.max(np.abs(b)), 1e-30)
            assert np.max(np.abs(a - b)) / scale <= 1e-4, k


def test_ensemble_autotune_restores_members():
    ws = members(seed=11, sides=[64, 130, 96])
    a = sw.Ensemble(ws, precision=sw.FP64)
    b = sw.Ensemble(ws, precision=sw.FP64)
    a.step(5)
    b.step(5)
    rec = b.autotune(steps=2)
    assert 0 <= rec["shape"] < len(sw.ensemble_shapes())
    a.set_member_shapes(rec["member_shapes"])
    a.step(7)
    b.step(7)
    for k in range(len(ws)):
        for x, y in zip(a.member(k).state(), b.member(k).state()):
            assert np.array_equal(x, y)
        assert a.member(k).diagnostics() == b.member(k).diagnostics()


def test_ensemble_bounded_wait_reports_timeout():
    """A member whose waits can never succeed (test hook): the bounded wait
    runs out, every CTA stops, and the host reads SWOF_ETIMEOUT."""
    ws = members(seed=13, sides=[48, 64, 80])
    ens = sw.Ensemble(ws, precision=sw.FP32)
    assert ens.step(2) == 0
    ens.set_wait_limit(2000, block_member=1)
    with pytest.raises(sw.SwofError) as e:
        ens.step(3)
    assert e.value.code == sw.ETIMEOUT
    with pytest.raises(sw.SwofError):
        ens.step(1)                     # latched
    # the context is still usable: an unrelated solver runs fine
    s = sw.Solver.from_workload(ws[0], sw.FP32)
    assert s.step(3).status == 0


def test_fp32_ensemble_members_against_fp64_oracle():
    """FP32 bulk members with the oracle's dt replayed: relative L1 of
    (h, hu, hv) per member after 60 steps within 1e-5 (the discharges also
    printed against the discharge vector's L1 norm)."""
    ws = members(seed=21, sides=[64, 96, 130, 48])
    ens = sw.Ensemble(ws, precision=sw.FP32)
    refs = []
    for k, w in enumerate(ws):
        o = oracle.Oracle.from_workload(w)
        dts = o.step(60)
        ens.member(k).set_dt_sequence(dts)
        refs.append(o.state())
    assert ens.step(60) == 0
    for k in range(len(ws)):
        got = ens.member(k).state()
        errs = [np.sum(np.abs(a - b)) / max(np.sum(np.abs(b)), 1e-30) for a, b in zip(got, refs[k])]
        qn = max(np.sum(np.hypot(refs[k][1], refs[k][2])), 1e-30)
        eq = [np.sum(np.abs(a - b)) / qn for a, b in zip(got[1:], refs[k][1:])]
        print(f"member {k} ({ws[k].nx}^2): rel L1 h {errs[0]:.2e} hu {errs[1]:.2e} hv {errs[2]:.2e}; "
              f"vs |q| {eq[0]:.2e} {eq[1]:.2e}")
        assert max(errs) <= 1e-5, errs


def test_fp64_ensemble_mixed_tile_heights_equal_members():
    """One launch width, members on different tile heights (64 x 64 and
    64 x 16): each FP64 member still equals its own single-grid run and the
    oracle bit for bit."""
    ws = members(seed=31, sides=[64, 130, 96, 48])
    ens = sw.Ensemble(ws, precision=sw.FP64)
    shp = sw.ensemble_shapes()
    narrow = [k for k, (ntx, _) in enumerate(shp) if ntx == 64]
    ens.set_member_shapes([narrow[k % len(narrow)] for k in range(len(ws))])
    assert len(set(ens.member_shapes())) == 2
    assert ens.step(9) == 0
    for k, w in enumerate(ws):
        o = oracle.Oracle.from_workload(w, dt_max=0.1)
        dts = o.step(9)
        m = ens.member(k)
        assert np.array_equal(m.dt_history(), dts), k
        for a, b in zip(m.state(), o.state()):
            assert np.array_equal(a, b), k


def test_fp64_ensemble_members_with_imposed_edges_equal_oracle():
    """Members with Riemann-invariant imposed edges (Sec. 2.2: depth,
    discharge, both) beside walls and outflow: FP64 bit for bit the oracle's
    states and dt sequences, the CFL maximum seeing each boundary state."""
    ws = members(seed=41, sides=[64, 96, 80])
    edges = [((2, 1, 0, 3), (1.2, 0, 0, 0), (0, 0, 0, 0.6)),
             ((3, 0, 4, 1), (0, 0, 0.8, 0), (0.5, 0, 0.9, 0)),
             ((4, 2, 1, 0), (1.0, 0.7, 0, 0), (2.0, 0, 0, 0))]
    for w, (bc, bh, bq) in zip(ws, edges):
        w.bc, w.bc_h, w.bc_q = bc, bh, bq
    ens = sw.Ensemble(ws, precision=sw.FP64)
    assert ens.step(12) == 0
    for k, (w, (bc, bh, bq)) in enumerate(zip(ws, edges)):
        o = oracle.Oracle.from_workload(w, dt_max=0.1, bc=bc, bc_h=bh, bc_q=bq)
        dts = o.step(12)
        m = ens.member(k)
        assert np.array_equal(m.dt_history(), dts), k
        for a, b in zip(m.state(), o.state()):
            assert np.array_equal(a, b), k


def test_fp32_ensemble_bench_members_over_1000_steps():
    """Every 8th member of the 256-member benchmark ensemble (sides 128-1024,
    reservoirs of 5-40 m under rain), FP32 against the FP64 ensemble (bit for
    bit the oracle's members) on each member's FP64 dt sequence over the full
    1000 steps: h and hv within 1e-5 relative L1 per member; the cross-valley
    discharge hu, ~0 in the pools, within 1e-5 of the discharge vector's L1
    norm (its own relative L1 is printed)."""
    specs = si.ensemble_specs(256, seed=4)
    ws = [si.ensemble_member(specs[k]) for k in range(0, len(specs), 8)]
    e64 = sw.Ensemble(ws, precision=sw.FP64)
    assert e64.step(1000) == 0
    ref = [(e64.member(k).state(), e64.member(k).dt_history(1000)) for k in range(len(ws))]
    e64.close()
    e32 = sw.Ensemble(ws, precision=sw.FP32)
    for k in range(len(ws)):
        e32.member(k).set_dt_sequence(ref[k][1])
    assert e32.step(1000) == 0
    for k in range(len(ws)):
        (h, hu, hv), got = ref[k][0], e32.member(k).state()
        rel = [np.sum(np.abs(a - b)) / max(np.sum(np.abs(b)), 1e-300) for a, b in zip(got, (h, hu, hv))]
        hu_q = np.sum(np.abs(got[1] - hu)) / max(np.sum(np.hypot(hu, hv)), 1e-300)
        print(f"member {8 * k} ({ws[k].nx}^2): h {rel[0]:.2e} hu {rel[1]:.2e} hv {rel[2]:.2e} hu/|q| {hu_q:.2e}")
        assert rel[0] <= 1e-5 and rel[2] <= 1e-5 and hu_q <= 1e-5, (8 * k, rel, hu_q)
    e32.close()

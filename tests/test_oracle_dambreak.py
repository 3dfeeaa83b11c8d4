"""Pins of the oracle against the dam-break closed forms (no GPU).

The paper validates FullSWOF on SWASHES analytic solutions (Sec. 4.1); the
two dam breaks below are the textbook Riemann solutions restated in
tests/swe_closed_forms.py.  Strips uniform in y (walls all round) reduce the
2-D scheme to the 1-D one.  Thresholds: the 200-cell L1 errors were
calibrated once on the oracle and frozen with margin; the observed
convergence order is fixed by the theory (a second-order scheme drops to
first order at a shock / dry front in L1).
"""
import math

import numpy as np
import pytest

import oracle
from swe_closed_forms import dam_break_profile, stoker_state


def _strip(n, h_r, t_end, length=10.0, ny=4):
    dx = length / n
    x = (np.arange(n) + 0.5) * dx
    h0 = np.where(x < 0.5 * length, 1.0, h_r)
    H = np.tile(h0, (ny, 1))
    o = oracle.Oracle(n, ny, dx, dx, np.zeros_like(H), t_end=t_end, dt_max=0.1)
    o.set_state(H, np.zeros_like(H), np.zeros_like(H))
    o.run_to(t_end)
    h, qx, qy = o.state()
    assert np.all(h == h[0:1]) and np.all(qy == 0.0)
    return x, h[0], qx[0], o.diag()


def _l1(a, b):
    return np.sum(np.abs(a - b)) / np.sum(np.abs(b))


def test_stoker_intermediate_state():
    hm, um, s = stoker_state(1.0, 0.5)
    g = 9.81
    # Riemann invariant across the rarefaction and Rankine-Hugoniot mass/momentum
    assert math.isclose(um + 2 * math.sqrt(g * hm), 2 * math.sqrt(g * 1.0), rel_tol=1e-12)
    mass = s * (hm - 0.5) - hm * um
    mom = s * hm * um - (hm * um * um + 0.5 * g * (hm * hm - 0.25))
    assert abs(mass) < 1e-12 and abs(mom) < 1e-12


def test_stoker_wet_bed_dam_break_config0():
    """The 200 x 200, dx = 0.05 m dam break (h = 1 | 0.5) at t = 1 s."""
    x, h, q, d = _strip(200, 0.5, 1.0)
    he, ue = dam_break_profile(x, 1.0, 5.0, 1.0, 0.5)
    assert _l1(h, he) < 5e-3
    assert _l1(q, he * ue) < 3e-2
    assert d["volume"] == pytest.approx(0.75 * 10.0 * 0.2, rel=1e-14)
    # the waves are still inside the domain at t = 1 s
    assert abs(h[0] - 1.0) < 1e-12 and abs(h[-1] - 0.5) < 1e-12


def test_stoker_convergence_order():
    errs = []
    for n in (100, 200, 400, 800):
        x, h, q, _ = _strip(n, 0.5, 1.0)
        errs.append(_l1(h, dam_break_profile(x, 1.0, 5.0, 1.0, 0.5)[0]))
    order = math.log2(errs[0] / errs[-1]) / 3
    assert order >= 0.8, errs


def test_ritter_dry_bed_dam_break():
    t = 0.6
    errs = []
    for n in (100, 200, 400, 800):
        x, h, q, _ = _strip(n, 0.0, t)
        he, _ = dam_break_profile(x, t, 5.0, 1.0, 0.0)
        errs.append(_l1(h, he))
        front = 5.0 + 2.0 * math.sqrt(9.81) * t
        wet_edge = x[h > 1e-6].max()
        dx = 10.0 / n
        assert wet_edge <= front + dx           # never ahead of the exact front
        assert front - wet_edge <= 0.5          # the dry threshold lags it a little
        assert h.min() >= 0.0
    assert errs[1] < 7e-3
    assert math.log2(errs[0] / errs[-1]) / 3 >= 0.5, errs

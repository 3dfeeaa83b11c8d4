"""Pins of the oracle's extensions against what the paper and the mathematics
fix (no GPU):

* the friction laws of Sec. 2.1 (Manning, Strickler, Darcy-Weisbach, Chezy)
  through the closed-form solution of the friction ODE on a uniform flow,
* the imposed boundaries of Sec. 2.2: the Riemann invariant leaving the
  domain is kept, the imposed variable is met, uniform flows stay uniform
  (in x, in y, in both directions, with a tangential component), a lake at
  rest stays at rest, a torrential inflow fills a dry channel to the imposed
  state, a fluvial channel relaxes to the imposed discharge, the volume
  budget closes,
* the first-order variant of Sec. 3.3: one step is the textbook 1-D HLL
  finite-volume update on a flat bed, lake at rest, the dam-break closed
  form with first-order convergence, and the CFL speed of the cell values,
* gauges and the running maximum depth against brute force over single
  steps,
* the D8 flow direction (Sec. 5.2) against a brute-force restatement on small
  DEMs with ties, a cone and a tilted plane.
"""
import math

import mpmath as mp

import numpy as np
import pytest

import oracle
import swof_inputs as si
from mp_scheme import MPScheme
from swe_closed_forms import dam_break_profile

G = 9.81


# ---------------------------------------------------------------- friction

@pytest.mark.parametrize("law,coef,power", [(1, 0.15, 4.0 / 3.0), (2, 1.0 / 0.15, 4.0 / 3.0),
                                            (3, 1.2, 1.0), (4, 8.0, 1.0)])
def test_friction_law_decay_matches_ode(law, coef, power):
    """Uniform flow on a flat bed, outflow all round: the convective step is
    the identity and q follows dq/dt = -g C_f |q| q / h^(p+1), whose solution
    is |q|(t) = |q0| / (1 + k |q0| t), direction fixed, k = g C_f / h^(p+1)
    (S_f of Sec. 2.1: C_f = n^2, 1/K^2, f/(8g), 1/C^2; p = 4/3 or 1)."""
    cf = {1: coef ** 2, 2: 1.0 / coef ** 2, 3: coef / (8.0 * G), 4: 1.0 / coef ** 2}[law]
    assert oracle.friction_cf(law, G, coef) == pytest.approx(cf, rel=1e-15)
    n, h0, qx0, qy0, T = 4, 2.0, 1.2, -0.7, 10.0
    k = G * cf / h0 ** (power + 1.0)
    q0 = math.hypot(qx0, qy0)
    qe = q0 / (1.0 + k * q0 * T)
    assert q0 / qe > 1.3                         # friction really acted
    errs = []
    for dt in (0.01, 0.005):
        o = oracle.Oracle(n, n, 1.0, 1.0, np.zeros((n, n)), bc=(1, 1, 1, 1), friction=law,
                          friction_coef=coef, dt_fixed=dt, dt_max=1.0)
        o.set_state(np.full((n, n), h0), np.full((n, n), qx0), np.full((n, n), qy0))
        o.step(int(round(T / dt)))
        h, qx, qy = o.state()
        assert np.all(h == h0)
        assert np.all(qx == qx[0, 0]) and np.all(qy == qy[0, 0])
        assert qx[0, 0] / qy[0, 0] == pytest.approx(qx0 / qy0, rel=1e-12)
        errs.append(abs(math.hypot(qx[0, 0], qy[0, 0]) / qe - 1.0))
    # the semi-implicit splitting converges to the ODE solution at first order in dt
    assert errs[1] < 1e-4 and 1.8 < errs[0] / errs[1] < 2.2, errs


def test_strickler_is_manning_with_inverse_coefficient():
    n = 5
    res = []
    for law, coef in ((1, 0.05), (2, 20.0)):
        o = oracle.Oracle(n, n, 1.0, 1.0, np.zeros((n, n)), bc=(1, 1, 1, 1), friction=law,
                          friction_coef=coef, dt_max=0.1)
        o.set_state(np.full((n, n), 0.7), np.full((n, n), 0.4), np.zeros((n, n)))
        o.step(50)
        res.append(o.state()[1])
    assert np.allclose(res[0], res[1], rtol=1e-14)


def test_friction_map_per_cell():
    """A per-cell coefficient map (Darcy-Weisbach): a map equal to the scalar
    everywhere reproduces the scalar run bit for bit; changing one column
    changes, after one step, that column and nothing farther than the
    4-cell reach of two 2-cell stencils."""
    nx, ny, c0 = 16, 5, 3
    st = (np.full((ny, nx), 1.5), np.zeros((ny, nx)), np.full((ny, nx), 0.9))

    def run(coef, fmap, steps):
        o = oracle.Oracle(nx, ny, 1.0, 1.0, np.zeros((ny, nx)), bc=(1, 1, 1, 1), friction=3,
                          friction_coef=coef, n_map=fmap, dt_fixed=0.02, dt_max=1.0)
        o.set_state(*st)
        o.step(steps)
        return o.state()

    ref = run(0.6, None, 1)
    same = run(0.0, np.full((ny, nx), 0.6), 1)
    assert all(np.array_equal(a, b) for a, b in zip(ref, same))
    fmap = np.full((ny, nx), 0.6)
    fmap[:, c0] = 1.8
    one = run(0.0, fmap, 1)
    far = np.abs(np.arange(nx) - c0) > 4
    assert all(np.array_equal(a[:, far], b[:, far]) for a, b in zip(ref, one))
    assert np.all(one[2][:, c0] < ref[2][:, c0])


# ---------------------------------------------------------------- imposed boundaries

@pytest.mark.parametrize("R,Q", [(-6.0, 4.9), (-0.5, 1e-3), (3.0, 20.0), (0.0, 7.0), (-40.0, 0.02)])
def test_inflow_celerity_is_the_root_of_the_invariant(R, Q):
    c = oracle.inflow_celerity(R, Q)
    roots = np.roots([2.0, R, 0.0, -Q])
    real_pos = [r.real for r in roots if abs(r.imag) < 1e-12 and r.real > 0]
    assert len(real_pos) == 1
    assert c == pytest.approx(real_pos[0], rel=1e-13)
    h = c * c / G
    q = Q / G
    assert q / h - 2.0 * math.sqrt(G * h) == pytest.approx(R, rel=1e-12, abs=1e-12)


def test_inflow_celerity_zero_discharge():
    assert oracle.inflow_celerity(-4.0, 0.0) == 2.0
    assert oracle.inflow_celerity(3.0, 0.0) == 0.0


@pytest.mark.parametrize("h1,qn1,qt1", [(1.0, 0.5, 0.2), (0.3, -0.4, 0.0), (2.0, 0.0, -1.0), (0.0, 0.0, 0.0)])
def test_imposed_states_keep_the_outgoing_invariant(h1, qn1, qt1):
    w1 = qn1 / h1 if h1 > 1e-6 else 0.0
    t1 = qt1 / h1 if h1 > 1e-6 else 0.0
    R = w1 - 2.0 * math.sqrt(G * h1)
    # imposed depth
    hb, qb, tb = oracle.imposed_state(G, 1e-6, 2, 0.8, 0.0, h1, qn1, qt1)
    assert hb == 0.8
    assert qb / hb - 2.0 * math.sqrt(G * hb) == pytest.approx(R, abs=1e-13)
    assert tb == pytest.approx(hb * t1, abs=1e-15)
    # imposed discharge
    hb, qb, tb = oracle.imposed_state(G, 1e-6, 3, 0.0, 0.6, h1, qn1, qt1)
    assert qb == 0.6 and hb > 0
    assert qb / hb - 2.0 * math.sqrt(G * hb) == pytest.approx(R, abs=1e-12)
    assert tb == pytest.approx(hb * t1, abs=1e-15)
    # both imposed: no tangential flow
    assert list(oracle.imposed_state(G, 1e-6, 4, 0.5, 5.0, h1, qn1, qt1)) == [0.5, 5.0, 0.0]


def _channel(axis, nx, ny, bc, bc_h, bc_q, **kw):
    if axis == "y":
        nx, ny = ny, nx
        bc = (bc[2], bc[3], bc[0], bc[1])
        bc_h = (bc_h[2], bc_h[3], bc_h[0], bc_h[1])
        bc_q = (bc_q[2], bc_q[3], bc_q[0], bc_q[1])
    return oracle.Oracle(nx, ny, 1.0, 1.0, np.zeros((ny, nx)), bc=bc, bc_h=bc_h, bc_q=bc_q,
                         dt_max=1.0, **kw)


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("direction", [1, -1])
def test_uniform_fluvial_flow_between_imposed_edges_is_steady(axis, direction):
    """Flat, frictionless channel with a uniform subcritical flow (h0, q0)
    plus a tangential component: imposed discharge where the flow enters,
    imposed depth where it leaves.  Every ghost state equals the interior
    one, so the flow must stay exactly uniform."""
    h0, q0, qt0, L, W = 1.0, 0.5, 0.2, 24, 3
    up, down = (0, 1) if direction == 1 else (1, 0)
    bc = [0, 0, 1, 1]
    bc_h, bc_q = [0.0] * 4, [0.0] * 4
    bc[up], bc[down] = 3, 2
    bc_q[up], bc_h[down] = q0, h0
    o = _channel(axis, L, W, bc, bc_h, bc_q)
    shape = (W, L) if axis == "x" else (L, W)
    qn = np.full(shape, direction * q0)
    qt = np.full(shape, qt0)
    st = (np.full(shape, h0), qn, qt) if axis == "x" else (np.full(shape, h0), qt, qn)
    o.set_state(*st)
    o.step(200)
    for a, b in zip(o.state(), st):
        assert np.max(np.abs(a - b)) <= 1e-14


def test_lake_at_rest_with_imposed_depth_edge():
    """An imposed depth equal to the edge cell's depth at rest keeps a lake
    over uneven topography at rest."""
    w = si.lake_at_rest(n=32, level=1.0)
    ok = w.h[:, 0] > 0.1
    assert ok.all()
    hb = float(w.h[0, 0])
    z = w.z.copy()
    z[:, 0] = z[0, 0]          # flat edge column so one imposed depth fits all its cells
    h = np.maximum(1.0 - z, 0.0)
    o = oracle.Oracle(w.nx, w.ny, w.dx, w.dy, z, bc=(2, 0, 0, 0), bc_h=(1.0 - z[0, 0], 0, 0, 0))
    o.set_state(h, 0 * h, 0 * h)
    o.step(300)
    hn, qx, qy = o.state()
    wet = h > 0
    assert np.max(np.abs((hn + z)[wet] - 1.0)) <= 1e-12
    assert np.max(np.abs(qx)) <= 1e-12 and np.max(np.abs(qy)) <= 1e-12
    assert hb > 0


def test_torrential_inflow_fills_dry_channel_to_imposed_state():
    """Both variables imposed (supercritical inflow, Sec. 2.2) into a dry flat
    channel with free outflow: the channel fills and settles at exactly the
    imposed uniform state; the CFL step sees the boundary state."""
    nx, ny, hb, qb = 24, 3, 0.5, 5.0
    assert qb / hb > math.sqrt(G * hb)
    o = oracle.Oracle(nx, ny, 1.0, 1.0, np.zeros((ny, nx)), bc=(4, 1, 0, 0), bc_h=(hb, 0, 0, 0),
                      bc_q=(qb, 0, 0, 0), dt_max=1.0)
    o.set_state(np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    assert o.lam()[0] == pytest.approx(qb / hb + math.sqrt(G * hb), rel=1e-15)
    o.step(300)
    h, qx, qy = o.state()
    assert np.max(np.abs(h - hb)) <= 1e-12 and np.max(np.abs(qx - qb)) <= 1e-11
    assert np.all(qy == 0.0)


def test_fluvial_channel_relaxes_to_imposed_discharge_and_budget_closes():
    """Lake at rest in a flat channel, imposed discharge q_in upstream and the
    same depth downstream: a flat frictionless steady flow has one q and one
    h everywhere, so the state relaxes to (h0, q_in).  Inflow enters the
    volume budget through the edge fluxes."""
    nx, ny, h0, qin = 24, 3, 1.0, 0.5
    o = oracle.Oracle(nx, ny, 1.0, 1.0, np.zeros((ny, nx)), bc=(3, 2, 0, 0), bc_q=(qin, 0, 0, 0),
                      bc_h=(0, h0, 0, 0), dt_max=1.0)
    o.set_state(np.full((ny, nx), h0), np.zeros((ny, nx)), np.zeros((ny, nx)))
    v0 = o.diag()["volume"]
    o.step(4000)
    h, qx, qy = o.state()
    d = o.diag()
    assert np.max(np.abs(qx - qin)) < 2e-3 and np.max(np.abs(h - h0)) < 1e-3
    assert abs(d["volume"] - v0 + d["outflow"]) <= 1e-12 * v0


# ---------------------------------------------------------------- first order

def _textbook_hll_step(h, q, dx, dt):
    """First-order finite volumes with the 1-D HLL flux (Harten-Lax-van Leer,
    wave speeds min/max of u -+ c over both states), constant extension at
    both ends; flat bed, so no source term."""
    he = np.concatenate([[h[0]], h, [h[-1]]])
    qe = np.concatenate([[q[0]], q, [q[-1]]])
    u = qe / he
    c = np.sqrt(G * he)
    flux = []
    for i in range(len(h) + 1):
        a, b = i, i + 1
        s1 = min(u[a] - c[a], u[b] - c[b])
        s2 = max(u[a] + c[a], u[b] + c[b])
        FL = np.array([qe[a], qe[a] ** 2 / he[a] + 0.5 * G * he[a] ** 2])
        FR = np.array([qe[b], qe[b] ** 2 / he[b] + 0.5 * G * he[b] ** 2])
        if s1 >= 0:
            f = FL
        elif s2 <= 0:
            f = FR
        else:
            f = (s2 * FL - s1 * FR + s1 * s2 * (np.array([he[b], qe[b]]) - np.array([he[a], qe[a]]))) / (s2 - s1)
        flux.append(f)
    flux = np.array(flux)
    return h - dt / dx * (flux[1:, 0] - flux[:-1, 0]), q - dt / dx * (flux[1:, 1] - flux[:-1, 1])


@pytest.mark.parametrize("seed", [0, 1])
def test_first_order_step_is_textbook_hll_on_flat_bed(seed):
    rng = np.random.default_rng(seed)
    n, ny, dx = 16, 3, 0.7
    h = 0.5 + rng.random(n)
    q = 0.8 * rng.standard_normal(n)
    o = oracle.Oracle(n, ny, dx, 1.0, np.zeros((ny, n)), order=1, cfl=1.0, bc=(1, 1, 0, 0),
                      dt_max=10.0)
    o.set_state(np.tile(h, (ny, 1)), np.tile(q, (ny, 1)), np.zeros((ny, n)))
    u = q / h
    c = np.sqrt(G * h)
    lam_x = np.max(np.abs(u) + c)
    assert o.lam()[0] == pytest.approx(lam_x, rel=1e-15)       # cell values (Eq. (cfl), first order)
    dt = o.step(1)[0]
    assert dt == pytest.approx(1.0 / (lam_x / dx + np.max(c) / 1.0), rel=1e-15)
    H, QX, QY = o.state()
    hn, qn = _textbook_hll_step(h, q, dx, dt)
    assert np.max(np.abs(H - hn)) <= 1e-14 and np.max(np.abs(QX - qn)) <= 1e-14
    assert np.all(QY == 0.0)


def test_first_order_lake_at_rest():
    w = si.lake_at_rest(n=40, level=1.0)
    o = oracle.Oracle.from_workload(w, order=1, cfl=1.0)
    o.step(500)
    h, qx, qy = o.state()
    wet = w.h > 0
    assert np.max(np.abs((h + w.z)[wet] - 1.0)) <= 1e-12
    assert np.max(np.abs(qx)) <= 1e-12 and np.max(np.abs(qy)) <= 1e-12


def _strip(n, order, length=10.0, ny=4, t_end=1.0):
    dx = length / n
    x = (np.arange(n) + 0.5) * dx
    H = np.tile(np.where(x < 0.5 * length, 1.0, 0.5), (ny, 1))
    o = oracle.Oracle(n, ny, dx, dx, np.zeros_like(H), t_end=t_end, dt_max=0.1, order=order,
                      cfl=1.0 if order == 1 else 0.5)
    o.set_state(H, 0 * H, 0 * H)
    o.run_to(t_end)
    return x, o.state()[0][0], o.diag()


def test_first_order_dam_break_converges_at_first_order():
    errs = []
    for n in (100, 200, 400, 800):
        x, h, d = _strip(n, 1)
        errs.append(np.sum(np.abs(h - dam_break_profile(x, 1.0, 5.0, 1.0, 0.5)[0]))
                    / np.sum(dam_break_profile(x, 1.0, 5.0, 1.0, 0.5)[0]))
        assert d["volume"] == pytest.approx(0.75 * 10.0 * 4 * (10.0 / n), rel=1e-14)
    order = math.log2(errs[0] / errs[-1]) / 3
    assert 0.6 <= order <= 1.1, errs
    assert errs[1] < 1.2e-2
    # and it is the more diffusive of the two orders
    x, h2, _ = _strip(200, 2)
    e2 = np.sum(np.abs(h2 - dam_break_profile(x, 1.0, 5.0, 1.0, 0.5)[0])) / np.sum(
        dam_break_profile(x, 1.0, 5.0, 1.0, 0.5)[0])
    assert e2 < 0.6 * errs[1]


def test_first_order_positive_and_mass_conserving_on_rough_state():
    w = si.random_state(40, 32, seed=5, dry_frac=0.3, vel=1.5)
    w.bc = (0, 0, 0, 0)
    o = oracle.Oracle.from_workload(w, order=1, cfl=1.0, friction=3, friction_coef=0.5)
    m0 = o.diag()["volume"]
    for _ in range(100):
        o.step(1)
        assert o.diag()["min_h"] >= 0.0
    assert abs(o.diag()["volume"] - m0) <= 1e-13 * m0 * 10


# ---------------------------------------------------------------- gauges and maximum depth

def test_gauges_and_max_depth_match_brute_force():
    w = si.random_state(20, 16, seed=7, dry_frac=0.2, vel=1.0)
    cells = [(0, 0), (19, 15), (7, 3), (7, 3), (12, 9)]
    o = oracle.Oracle.from_workload(w)
    o.track_max(True)
    o.set_gauges(cells, capacity=8)
    ref = oracle.Oracle.from_workload(w)
    hmax = w.h.copy()
    recs = []
    for s in range(10):
        o.step(1)
        ref.step(1)
        h, qx, qy = ref.state()
        hmax = np.maximum(hmax, h)
        r = [ref.diag()["t"]]
        for i, j in cells:
            r += [h[j, i], qx[j, i], qy[j, i]]
        recs.append(r)
    got = o.gauges()
    assert got.shape == (8, 1 + 3 * len(cells))          # capacity reached, later steps dropped
    assert np.array_equal(got, np.array(recs[:8]))
    assert np.array_equal(o.max_depth(), hmax)
    assert (o.max_depth() > ref.state()[0]).any()


def test_gauge_outside_grid_rejected_and_max_requires_tracking():
    o = oracle.Oracle(4, 4, 1.0, 1.0, np.zeros((4, 4)))
    with pytest.raises(oracle.OracleError):
        o.set_gauges([(4, 0)], 2)
    with pytest.raises(oracle.OracleError):
        o.max_depth()


# ---------------------------------------------------------------- D8 flow direction

def _d8_brute(z, nodata=None):
    """Restatement by angles: neighbour (di, dj) has code 1 + (angle of
    (di, dj) from +x, counter-clockwise, in steps of 45 degrees)."""
    ny, nx = z.shape
    out = np.zeros((ny, nx), np.uint8)
    order = sorted([(di, dj) for di in (-1, 0, 1) for dj in (-1, 0, 1) if (di, dj) != (0, 0)],
                   key=lambda d: (math.degrees(math.atan2(d[1], d[0])) + 360.0) % 360.0)
    for j in range(ny):
        for i in range(nx):
            best, code = z[j, i], 0
            for k, (di, dj) in enumerate(order):
                a, b = i + di, j + dj
                if 0 <= a < nx and 0 <= b < ny and (nodata is None or z[b, a] > nodata) and z[b, a] < best:
                    best, code = z[b, a], k + 1
            out[j, i] = code
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_d8_matches_brute_force_with_ties_and_nodata(seed):
    rng = np.random.default_rng(seed)
    z = rng.integers(0, 4, size=(9, 11)).astype(np.float32)     # many ties
    z[rng.random(z.shape) < 0.1] = -9999.0                    # no-data cells
    assert np.array_equal(oracle.d8(z), _d8_brute(z))
    assert np.array_equal(oracle.d8(z, nodata=-9999.0), _d8_brute(z, -9999.0))
    assert np.array_equal(oracle.d8(z, nodata=1.0), _d8_brute(z, 1.0))
    zi = z.copy()
    zi[0, 0], zi[3, 4] = -np.inf, np.nan                     # -inf is a candidate without no-data; NaN never
    assert np.array_equal(oracle.d8(zi), _d8_brute(zi))
    zc = rng.standard_normal((13, 7)).astype(np.float32)
    assert np.array_equal(oracle.d8(zc), _d8_brute(zc))


def test_d8_cone_and_plane():
    n = 9
    y, x = np.mgrid[0:n, 0:n]
    cone = np.hypot(x - 4, y - 4).astype(np.float32)
    d = oracle.d8(cone)
    assert d[4, 4] == 0
    # each cell drains towards the centre: code of the direction (sign(dx), sign(dy))
    code = {(1, 0): 1, (1, 1): 2, (0, 1): 3, (-1, 1): 4, (-1, 0): 5, (-1, -1): 6, (0, -1): 7, (1, -1): 8}
    for j in range(n):
        for i in range(n):
            if (i, j) != (4, 4):
                assert d[j, i] == code[(int(np.sign(4 - i)), int(np.sign(4 - j)))]
    plane = (x + 2.0 * y).astype(np.float32)                # lowest neighbour: south-west
    d = oracle.d8(plane)
    assert np.all(d[1:, 1:] == 6) and np.all(d[0, 1:] == 5) and np.all(d[1:, 0] == 7) and d[0, 0] == 0


# ------------------------------------------------ 50-digit second implementation

# (name, order, friction law, coefficient, bc W E S N, bc_h, bc_q[, Green-Ampt])
MP_CASES = [
    ("first_order", 1, 1, 0.04, (0, 1, 1, 0), (0, 0, 0, 0), (0, 0, 0, 0)),
    ("strickler", 2, 2, 25.0, (0, 1, 1, 0), (0, 0, 0, 0), (0, 0, 0, 0)),
    ("darcy_weisbach", 2, 3, 0.3, (1, 0, 0, 1), (0, 0, 0, 0), (0, 0, 0, 0)),
    ("chezy", 2, 4, 15.0, (0, 0, 1, 1), (0, 0, 0, 0), (0, 0, 0, 0)),
    ("imposed_q_west_h_east", 2, 1, 0.03, (3, 2, 0, 1), (0, 1.3, 0, 0), (0.6, 0, 0, 0)),
    ("imposed_hq_south_first_order", 1, 0, 0.0, (0, 1, 4, 2), (0, 0, 0.8, 1.1), (0, 0, 2.5, 0)),
    # where V_inf = 0 Green-Ampt takes all the water: the clean-up must zero q
    ("green_ampt_dry_out", 2, 1, 0.04, (0, 1, 1, 0), (0, 0, 0, 0), (0, 0, 0, 0), True),
]


def mp_case_errors(case, library=None):
    """(wave speeds agree to 1e-14, largest relative state difference after
    two steps) between the oracle (or a library built from it) and the
    50-digit restatement for one of MP_CASES."""
    name, order, law, coef, bc, bc_h, bc_q = case[:7]
    ga = len(case) > 7 and case[7]
    rng = np.random.default_rng(sum(map(ord, name)))
    nx, ny, dx, dy = 5, 4, 0.3, 0.25
    z = 0.2 * rng.standard_normal((ny, nx))
    h = 0.5 + rng.random((ny, nx))
    h[rng.random((ny, nx)) < 0.2] = 0.0
    qx = h * 0.4 * rng.standard_normal((ny, nx))
    qy = h * 0.4 * rng.standard_normal((ny, nx))
    R, ks, psi, dth = (1e-3, 1e-4, 0.1, 0.3) if ga else (0.0, 0.0, 0.0, 0.0)
    o = oracle.Oracle(nx, ny, dx, dy, z, friction=law, friction_coef=coef, bc=bc, bc_h=bc_h, bc_q=bc_q,
                      order=order, rain_rate=R, rain_t_off=1e9 if ga else 0.0, infiltration=int(ga), ks=ks,
                      psi=psi, dtheta=dth, library=library)
    o.set_state(h, qx, qy)
    m = MPScheme(nx, ny, dx, dy, z, h, qx, qy, bc=bc, friction=law, friction_coef=coef if law else 0.0,
                 order=order, bc_h=bc_h, bc_q=bc_q, rain_rate=R, ks=ks, psi=psi, dtheta=dth,
                 infiltration=ga)
    if ga:
        v0 = 0.01 * (rng.random((ny, nx)) < 0.5)
        o.set_vinf(v0)
        m.vinf = [[mp.mpf(float(v0[j, i])) for i in range(nx)] for j in range(ny)]
    lx, ly = o.lam()
    mlx, mly = m.lam()
    lam_ok = math.isclose(lx, float(mlx), rel_tol=1e-14) and math.isclose(ly, float(mly), rel_tol=1e-14)
    for _ in range(2):
        m.step(o.step(1)[0])
    err = max(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300) for a, b in zip(o.state(), m.state()))
    return lam_ok, err


@pytest.mark.parametrize("case", MP_CASES, ids=[c[0] for c in MP_CASES])
def test_extensions_match_50_digit_second_implementation(case):
    """The first-order step, the Strickler / Darcy-Weisbach / Chezy laws,
    the imposed edges and Green-Ampt emptying cells against the 50-digit
    restatement (tests/mp_scheme.py: exact powers h^p, the imposed-discharge
    celerity from the exact roots of its cubic): wave speeds to 1e-14 and
    two steps to 1e-13 relative on a rough 5 x 4 grid."""
    lam_ok, err = mp_case_errors(case)
    assert lam_ok and err <= 1e-13, err

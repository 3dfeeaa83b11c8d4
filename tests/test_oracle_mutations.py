"""Do the oracle's pins catch plausible mistakes?

Each case plants one slip in a private copy of the oracle's C source (a
dropped term, a wrong sign, a swapped index or operand), builds it into a
temporary library on the CPU and runs a fast battery of the pins used in
test_oracle_*.py against it.  At least one pin must fail for every slip;
the unmodified source must pass them all.
"""
import math
import os
import subprocess

import mpmath
import numpy as np
import pytest

import oracle
import swof_inputs as si
from mp_scheme import MPScheme
from swe_closed_forms import dam_break_profile
from test_oracle_extensions import MP_CASES, _d8_brute, _textbook_hll_step, mp_case_errors

SRC = os.path.join(os.path.dirname(oracle.__file__), "swof_oracle.c")

MUTATIONS = {
    "drop_S_L": ("*f2l = F[1] + 0.5 * g * (hpa * hpa - hL * hL);", "*f2l = F[1];"),
    "drop_S_R": ("*f2r = F[1] + 0.5 * g * (hmb * hmb - hR * hR);", "*f2r = F[1];"),
    "Fc_sign": ("double fcx = hg *", "double fcx = -hg *"),
    "Fc_dropped_y": ("- dtdy * ((o->fy2l[c] - o->fy2r[s]) + fcy);", "- dtdy * (o->fy2l[c] - o->fy2r[s]);"),
    "modvel_swap": ("*unm = un[c] - (hpv * rh) * (0.5 * dun);", "*unm = un[c] - (hmv * rh) * (0.5 * dun);"),
    "modvel_sign": ("*unp = un[c] + (hmv * rh) * (0.5 * dun);", "*unp = un[c] - (hmv * rh) * (0.5 * dun);"),
    "hll_c1c2_swapped": ("F[k] = (c2 * FL[k] - c1 * FR[k]) * r", "F[k] = (c1 * FL[k] - c2 * FR[k]) * r"),
    "hll_diffusion_sign": ("+ w * (UR[k] - UL[k]);", "+ w * (UL[k] - UR[k]);"),
    "hll_c2_uses_minus": ("double c2 = fmax(unL + cL, unR + cR);", "double c2 = fmax(unL + cL, unR - cR);"),
    "minmod_max": ("if (a >= 0.0 && b >= 0.0) return fmin(a, b);", "if (a >= 0.0 && b >= 0.0) return fmax(a, b);"),
    "hydrostatic_min": ("double zmax = fmax(zpa, zmb);", "double zmax = fmin(zpa, zmb);"),
    "eta_not_h": ("double de = oracle_minmod(ec - em, ep - ec);", "double de = oracle_minmod(h[c] - h[cm], h[cp] - h[c]);"),
    "wall_no_negate": ("fill_ghost_x(o, qx, -1.0);", "fill_ghost_x(o, qx, 1.0);"),
    "west_index": ("double hs = h[c] - dtdx * (o->fx1[c] - o->fx1[w])", "double hs = h[c] - dtdx * (o->fx1[c] - o->fx1[s])"),
    "transverse_flux_axis": ("- dtdy * (o->fy3[c] - o->fy3[s]);", "- dtdy * (o->fx3[c] - o->fx3[s]);"),
    "friction_h_power": ("hinv = (y * y) * (y * y);", "hinv = (y * y) * y;"),
    "friction_old_speed_dropped": ("double den = 1.0 + (dt * g * cf) * speed * hinv;", "double den = 1.0 + (dt * g * cf) * hinv;"),
    "heun_no_average": ("h = 0.5 * (o->h[c] + o->h2[c]);", "h = o->h2[c];"),
    "darcy_power_4_3": ("if (o->p.friction <= 2) {", "if (o->p.friction <= 3) {"),
    "darcy_cf_without_g": ("case 3: return coef / (8.0 * g);", "case 3: return coef / 8.0;"),
    "strickler_not_inverse": ("case 2: return 1.0 / (coef * coef);", "case 2: return coef * coef;"),
    "chezy_not_squared": ("case 4: return 1.0 / (coef * coef);", "case 4: return 1.0 / coef;"),
    "riemann_invariant_sign": ("double R = w1 - 2.0 * sqrt(g * h1);", "double R = w1 + 2.0 * sqrt(g * h1);"),
    "imposed_h_velocity_sign": ("double w = R + 2.0 * sqrt(g * hset);", "double w = R - 2.0 * sqrt(g * hset);"),
    "imposed_outward_normal": ("double sgn = (side == 1 || side == 3) ? -1.0 : 1.0;", "double sgn = 1.0;"),
    "imposed_tangent_axis": ("double qt = side < 2 ? qy[c] : qx[c];", "double qt = side < 2 ? qx[c] : qy[c];"),
    "inflow_newton_one_step": ("for (int it = 0; it < 64; ++it) {", "for (int it = 0; it < 1; ++it) {"),
    "cfl_ignores_boundary_state": ("if (o->p.bc[0] >= 2) ax = fmax(ax, fabs(o->xup[w]) + sqrt(g * o->xhp[w]));", ""),
    "first_order_runs_heun": ("const int euler = o->p.order == 1;", "const int euler = 0;"),
    "first_order_outflow_halved": ("o->outflow += dt * b1;", "o->outflow += 0.5 * dt * b1;"),
    "first_order_z_from_h": ("o->xzm[c] = o->xzp[c] = o->yzm[c] = o->yzp[c] = z[c];",
                             "o->xzm[c] = o->xzp[c] = o->yzm[c] = o->yzp[c] = h[c];"),
    "d8_tie_goes_last": ("if ((!use_nodata || v > nodata) && v < best) {", "if ((!use_nodata || v > nodata) && v <= best) {"),
    "d8_nodata_ignored": ("if ((!use_nodata || v > nodata) && v < best) {", "if (v < best) {"),
    "d8_ne_nw_swapped": ("static const int di[8] = {1, 1, 0, -1, -1, -1, 0, 1};",
                         "static const int di[8] = {1, -1, 0, 1, -1, -1, 0, 1};"),
    "gauge_qx_qy_swapped": ("r[2 + 3 * g] = o->qx[c];", "r[2 + 3 * g] = o->qy[c];"),
    "hmax_is_min": ("o->hmax[ci] = fmax(o->hmax[ci], o->h[IDX(o, i, j)]);",
                    "o->hmax[ci] = fmin(o->hmax[ci], o->h[IDX(o, i, j)]);"),
    "ga_psi_sign": ("(1.0 + ((o->p.psi + h) * o->p.dtheta) / vi)", "(1.0 + ((o->p.psi - h) * o->p.dtheta) / vi)"),
    "ga_suction_dropped": ("(1.0 + ((o->p.psi + h) * o->p.dtheta) / vi)", "(1.0 + (h * o->p.dtheta) / vi)"),
    "cfl_dy_as_dx": ("double den = lx / o->dx + ly / o->dy;", "double den = lx / o->dx + ly / o->dx;"),
    "cfl_uses_cell_not_face": ("fabs(o->xup[c]) + sqrt(g * o->xhp[c]));", "fabs(o->xum[c]) + sqrt(g * o->xhm[c]));"),
    "rain_before_dt_scale": ("double rdt = dt * o->p.rain_rate;", "double rdt = o->p.rain_rate;"),
    "icbrt_one_newton_step": ("for (int it = 0; it < 4; ++it) {", "for (int it = 0; it < 1; ++it) {"),
    "imposed_hq_tangent_kept": ("out[0] = hset; out[1] = qset; out[2] = 0.0;",
                                "out[0] = hset; out[1] = qset; out[2] = hset * t1;"),
    "no_dry_cleanup": ("if (h <= hdry) { qx = 0.0; qy = 0.0; }", ""),
    "cfl_min_mode_max": ("double m = fmin(a, b);", "double m = fmax(a, b);"),
    "event_clamp_keeps_dt": ("if (ev[k] > t && ev[k] < t + dt) { dt = ev[k] - t; tn = ev[k]; }",
                             "if (ev[k] > t && ev[k] < t + dt) { tn = ev[k]; }"),
    "cfl_viol_inverted": ("if (dt * (lx / o->dx + ly / o->dy) > o->p.cfl) o->cfl_viol++;",
                          "if (dt * (lx / o->dx + ly / o->dy) <= o->p.cfl) o->cfl_viol++;"),
    "rain_before_t_on": ("int rain = o->p.rain_rate > 0.0 && o->t >= o->p.rain_t_on && o->t < o->p.rain_t_off;",
                         "int rain = o->p.rain_rate > 0.0 && o->t < o->p.rain_t_off;"),
    "dt_max_cap_dropped": ("if (dt > o->p.dt_max) dt = o->p.dt_max;", ""),
    "ks_map_ignored": ("double ks = o->ksmap ? o->ksmap[ci] : o->p.ks;", "double ks = o->p.ks;"),
    "friction_map_ignored": ("double cf = o->cf ? o->cf[(size_t)j * nx + i] : o->p_cf;", "double cf = o->p_cf;"),
    "infiltration_budget_without_area": ("o->infiltrated += infil * o->dx * o->dy;", "o->infiltrated += infil;"),
    "cfl_ignores_east_boundary_state": (
        "if (o->p.bc[1] >= 2) ax = fmax(ax, fabs(o->xum[e]) + sqrt(g * o->xhm[e]));", ""),
    "cfl_ignores_south_boundary_state": (
        "if (o->p.bc[2] >= 2) ay = fmax(ay, fabs(o->yvp[s]) + sqrt(g * o->yhp[s]));", ""),
    "cfl_ignores_north_boundary_state": (
        "if (o->p.bc[3] >= 2) ay = fmax(ay, fabs(o->yvm[n]) + sqrt(g * o->yhm[n]));", ""),
}


def _build_variant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: pattern must occur exactly once"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    str(path), "-o", str(so), "-lm"], check=True)
    return oracle.load_library(str(so))


# ---- the battery: each returns True when the pin holds -------------------

def pin_mp_second_implementation(L):
    rng = np.random.default_rng(3)
    nx, ny = 5, 4
    z = 0.2 * rng.standard_normal((ny, nx))
    h = 0.5 + rng.random((ny, nx))
    h[rng.random((ny, nx)) < 0.2] = 0.0
    qx = h * 0.4 * rng.standard_normal((ny, nx))
    qy = h * 0.4 * rng.standard_normal((ny, nx))
    kw = dict(bc=(0, 1, 1, 0), manning_n=0.04, rain_rate=1e-3, ks=1e-4, psi=0.1, dtheta=0.3)
    o = oracle.Oracle(nx, ny, 0.3, 0.25, z, friction=1, rain_t_off=1e9, infiltration=1,
                      library=L, **kw)
    o.set_state(h, qx, qy)
    o.set_vinf(np.full((ny, nx), 0.01))
    m = MPScheme(nx, ny, 0.3, 0.25, z, h, qx, qy, infiltration=True, **kw)
    m.vinf = [[mpmath.mpf(0.01) for _ in range(nx)] for _ in range(ny)]
    for _ in range(3):
        m.step(o.step(1)[0])
    ok = True
    for a, b in zip(o.state(), m.state()):
        ok &= bool(np.max(np.abs(a - b)) <= 1e-13 * max(np.max(np.abs(b)), 1e-300))
    return ok


def pin_lake_at_rest(L):
    w = si.lake_at_rest(n=24, level=1.0)
    o = oracle.Oracle(w.nx, w.ny, w.dx, w.dy, w.z, library=L)
    o.set_state(w.h, w.qx, w.qy)
    o.step(100)
    h, qx, qy = o.state()
    wet = w.h > 0
    return bool(np.max(np.abs((h + w.z)[wet] - 1.0)) <= 1e-12
                and np.max(np.abs(qx)) <= 1e-12 and np.max(np.abs(qy)) <= 1e-12)


def pin_mass_and_positivity(L):
    w = si.random_state(24, 20, seed=11, dry_frac=0.3, vel=1.2)
    o = oracle.Oracle(w.nx, w.ny, w.dx, w.dy, w.z, library=L, friction=1, manning_n=0.03)
    o.set_state(w.h, w.qx, w.qy)
    m0 = o.diag()["volume"]
    o.step(60)
    d = o.diag()
    return bool(abs(d["volume"] - m0) / m0 <= 1e-12 and d["min_h"] >= 0.0)


def pin_stoker(L):
    n, ny = 200, 4
    dx = 10.0 / n
    x = (np.arange(n) + 0.5) * dx
    H = np.tile(np.where(x < 5.0, 1.0, 0.5), (ny, 1))
    o = oracle.Oracle(n, ny, dx, dx, np.zeros_like(H), t_end=1.0, library=L)
    o.set_state(H, 0 * H, 0 * H)
    o.run_to(1.0)
    h = o.state()[0][0]
    he, _ = dam_break_profile(x, 1.0, 5.0, 1.0, 0.5)
    return bool(np.sum(np.abs(h - he)) / np.sum(he) < 5e-3)


def pin_symmetry(L):
    wx = si.dam_break(n=32, dx=0.3, axis="x")
    wy = si.dam_break(n=32, dx=0.3, axis="y")
    res = []
    for w in (wx, wy):
        o = oracle.Oracle(w.nx, w.ny, w.dx, w.dy, w.z, library=L)
        o.set_state(w.h, w.qx, w.qy)
        o.step(20)
        res.append(o.state())
    return bool(np.array_equal(res[0][0], res[1][0].T) and np.array_equal(res[0][1], res[1][2].T))


def pin_cfl_uniform(L):
    h, u, v, dx, dy, n = 0.7, -0.9, 0.35, 0.4, 0.25, 6
    o = oracle.Oracle(n, n, dx, dy, np.zeros((n, n)), bc=(1, 1, 1, 1), dt_max=10.0, library=L)
    o.set_state(np.full((n, n), h), np.full((n, n), h * u), np.full((n, n), h * v))
    c = math.sqrt(9.81 * h)
    return math.isclose(o.step(1)[0], 0.5 / ((abs(u) + c) / dx + (abs(v) + c) / dy), rel_tol=1e-14)


def pin_cfl_muscl_faces(L):
    """On a smooth, non-uniform flow the CFL speed uses the MUSCL face values:
    compare with the 50-digit second implementation's lambda."""
    rng = np.random.default_rng(5)
    nx, ny = 6, 5
    h = 1.0 + 0.3 * rng.random((ny, nx))
    qx = h * rng.standard_normal((ny, nx))
    qy = h * rng.standard_normal((ny, nx))
    z = 0.1 * rng.standard_normal((ny, nx))
    o = oracle.Oracle(nx, ny, 0.5, 0.5, z, library=L)
    o.set_state(h, qx, qy)
    m = MPScheme(nx, ny, 0.5, 0.5, z, h, qx, qy)
    lx, ly = o.lam()
    mlx, mly = m.lam()
    return math.isclose(lx, float(mlx), rel_tol=1e-14) and math.isclose(ly, float(mly), rel_tol=1e-14)


def pin_friction_uniform(L):
    n, h0, q0, nm = 8, 0.8, 0.6, 0.12
    o = oracle.Oracle(n, n, 1.0, 1.0, np.zeros((n, n)), bc=(1, 1, 1, 1), friction=1,
                      manning_n=nm, dt_max=0.05, library=L)
    o.set_state(np.full((n, n), h0), np.full((n, n), q0), np.zeros((n, n)))
    dts = o.step(30)
    q = q0
    for dt in dts:
        k = dt * 9.81 * nm * nm / h0 ** (7.0 / 3.0)
        q1 = q / (1.0 + k * abs(q))
        q = 0.5 * (q + q1 / (1.0 + k * abs(q1)))
    return bool(np.allclose(o.state()[1], q, rtol=1e-14, atol=0))


def pin_ponding_time(L):
    n = 4
    R, ks, psi, dth = 50.0 * si.RAIN_MM_PER_H, 1e-6, 0.1, 0.3
    o = oracle.Oracle(n, n, 1.0, 1.0, np.zeros((n, n)), bc=(1, 1, 1, 1), dt_max=1.0,
                      rain_rate=R, rain_t_off=600.0, infiltration=1, ks=ks, psi=psi,
                      dtheta=dth, library=L)
    o.set_state(np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n)))
    t = 0.0
    for _ in range(300):
        t += o.step(1)[0]
        if o.state()[0][0, 0] > 0:
            break
    tp = ks * psi * dth / (R * (R - ks))
    return abs(t - tp) <= 2.0 and math.isclose(o.diag()["rain_in"], R * n * n * t, rel_tol=1e-12)


def pin_friction_laws_ode(L):
    n, h0, qx0, qy0, T, dt = 4, 2.0, 1.2, -0.7, 10.0, 0.01
    ok = True
    for law, coef, p in ((2, 1.0 / 0.15, 4.0 / 3.0), (3, 1.2, 1.0), (4, 8.0, 1.0)):
        cf = {2: 1.0 / coef ** 2, 3: coef / (8.0 * 9.81), 4: 1.0 / coef ** 2}[law]
        o = oracle.Oracle(n, n, 1.0, 1.0, np.zeros((n, n)), bc=(1, 1, 1, 1), friction=law,
                          friction_coef=coef, dt_fixed=dt, dt_max=1.0, library=L)
        o.set_state(np.full((n, n), h0), np.full((n, n), qx0), np.full((n, n), qy0))
        o.step(int(round(T / dt)))
        q0 = math.hypot(qx0, qy0)
        qe = q0 / (1.0 + 9.81 * cf / h0 ** (p + 1.0) * q0 * T)
        _, qx, qy = o.state()
        ok &= abs(math.hypot(qx[0, 0], qy[0, 0]) / qe - 1.0) < 3e-4
    return ok


def pin_imposed_uniform_channels(L):
    h0, q0, qt0, n, w = 1.0, 0.5, 0.2, 16, 3
    ok = True
    for up, down, sgn in ((0, 1, 1.0), (1, 0, -1.0)):
        bc, bh, bq = [0, 0, 1, 1], [0.0] * 4, [0.0] * 4
        bc[up], bc[down], bq[up], bh[down] = 3, 2, q0, h0
        o = oracle.Oracle(n, w, 1.0, 1.0, np.zeros((w, n)), bc=bc, bc_h=bh, bc_q=bq, dt_max=1.0, library=L)
        st = (np.full((w, n), h0), np.full((w, n), sgn * q0), np.full((w, n), qt0))
        o.set_state(*st)
        o.step(60)
        ok &= all(np.max(np.abs(a - b)) <= 1e-14 for a, b in zip(o.state(), st))
    o = oracle.Oracle(w, n, 1.0, 1.0, np.zeros((n, w)), bc=(1, 1, 3, 2), bc_q=(0, 0, q0, 0),
                      bc_h=(0, 0, 0, h0), dt_max=1.0, library=L)
    st = (np.full((n, w), h0), np.full((n, w), qt0), np.full((n, w), q0))
    o.set_state(*st)
    o.step(60)
    ok &= all(np.max(np.abs(a - b)) <= 1e-14 for a, b in zip(o.state(), st))
    return ok


def pin_torrential_fill(L):
    nx, ny = 16, 3
    o = oracle.Oracle(nx, ny, 1.0, 1.0, np.zeros((ny, nx)), bc=(4, 1, 0, 0), bc_h=(0.5, 0, 0, 0),
                      bc_q=(5.0, 0, 0, 0), dt_max=1.0, library=L)
    o.set_state(np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    o.step(200)
    h, qx, _ = o.state()
    return bool(np.max(np.abs(h - 0.5)) <= 1e-12 and np.max(np.abs(qx - 5.0)) <= 1e-11)


def pin_first_order_textbook(L):
    rng = np.random.default_rng(0)
    n, ny, dx = 12, 3, 0.7
    h = 0.5 + rng.random(n)
    q = 0.8 * rng.standard_normal(n)
    o = oracle.Oracle(n, ny, dx, 1.0, np.zeros((ny, n)), order=1, cfl=1.0, bc=(1, 1, 0, 0),
                      dt_max=10.0, library=L)
    o.set_state(np.tile(h, (ny, 1)), np.tile(q, (ny, 1)), np.zeros((ny, n)))
    dt = o.step(1)[0]
    H, QX, _ = o.state()
    hn, qn = _textbook_hll_step(h, q, dx, dt)
    return bool(np.max(np.abs(H - hn)) <= 1e-14 and np.max(np.abs(QX - qn)) <= 1e-14)


def pin_first_order_lake_and_budget(L):
    w = si.lake_at_rest(n=24, level=1.0)
    o = oracle.Oracle(w.nx, w.ny, w.dx, w.dy, w.z, order=1, cfl=1.0, library=L)
    o.set_state(w.h, w.qx, w.qy)
    o.step(100)
    h, qx, qy = o.state()
    wet = w.h > 0
    ok = bool(np.max(np.abs((h + w.z)[wet] - 1.0)) <= 1e-12 and np.max(np.abs(qx)) <= 1e-12)
    r = si.random_state(16, 12, seed=2, dry_frac=0.2, vel=1.0)
    o = oracle.Oracle(r.nx, r.ny, r.dx, r.dy, r.z, order=1, cfl=1.0, bc=(3, 1, 0, 1),
                      bc_q=(0.4, 0, 0, 0), library=L)
    o.set_state(r.h, r.qx, r.qy)
    v0 = o.diag()["volume"]
    o.step(40)
    d = o.diag()
    return ok and abs(d["volume"] - v0 + d["outflow"]) <= 1e-12 * v0 and d["outflow"] != 0.0


def pin_d8_brute_force(L):
    rng = np.random.default_rng(1)
    z = rng.integers(0, 4, size=(7, 9)).astype(np.float32)
    z[rng.random(z.shape) < 0.15] = -9999.0
    ok = True
    for nodata in (None, -9999.0):
        out = np.zeros(z.shape, np.uint8)
        L.oracle_d8(z.ctypes.data_as(oracle.ctypes.POINTER(oracle.ctypes.c_float)), z.shape[1], z.shape[0],
                    int(nodata is not None), float(nodata or 0.0),
                    out.ctypes.data_as(oracle.ctypes.POINTER(oracle.ctypes.c_uint8)))
        ok &= bool(np.array_equal(out, _d8_brute(z, nodata)))
    return ok


def pin_gauges_and_max(L):
    w = si.random_state(10, 8, seed=7, dry_frac=0.2, vel=1.0)
    cells = [(0, 0), (9, 7), (4, 3)]
    o = oracle.Oracle(w.nx, w.ny, w.dx, w.dy, w.z, library=L)
    o.set_state(w.h, w.qx, w.qy)
    o.track_max(True)
    o.set_gauges(cells, 16)
    hmax, recs = w.h.copy(), []
    for _ in range(6):
        o.step(1)
        h, qx, qy = o.state()
        hmax = np.maximum(hmax, h)
        recs.append([o.diag()["t"]] + [v for i, j in cells for v in (h[j, i], qx[j, i], qy[j, i])])
    return bool(np.array_equal(o.gauges(), np.array(recs)) and np.array_equal(o.max_depth(), hmax))


def pin_mp_extension_cases(L):
    """50-digit restatement: depth and discharge both imposed (tangential
    discharge 0, Sec. 2.2) at first order; Green-Ampt emptying the cells
    with V_inf = 0 (the clean-up then zeroes their discharge); Darcy-
    Weisbach friction between outflow edges on the west and north."""
    cases = [c for c in MP_CASES if c[0] in ("imposed_hq_south_first_order", "green_ampt_dry_out",
                                              "darcy_weisbach")]
    return all(lam_ok and err <= 1e-13 for lam_ok, err in (mp_case_errors(c, L) for c in cases))


def pin_cfl_min_mode(L):
    """The per-direction form of Eq. (cfl) in 2-D (SWOF_CFL_MIN): on a
    uniform flow dt = n_CFL min(dx / (|u| + c), dy / (|v| + c))."""
    h, u, v, dx, dy, n = 0.7, -0.9, 0.35, 0.4, 0.25, 6
    o = oracle.Oracle(n, n, dx, dy, np.zeros((n, n)), bc=(1, 1, 1, 1), dt_max=10.0, cfl_mode=1, library=L)
    o.set_state(np.full((n, n), h), np.full((n, n), h * u), np.full((n, n), h * v))
    c = math.sqrt(9.81 * h)
    return math.isclose(o.step(1)[0], 0.5 * min(dx / (abs(u) + c), dy / (abs(v) + c)), rel_tol=1e-14)


def pin_event_clamps_and_rain_window(L):
    """Steps land on the rain on/off times and on t_end, and rain falls only
    on steps that start in [t_on, t_off): a lake at rest under rain from
    0.3 to 0.7 s with dt capped at 0.08 s (so both event times and t_end
    fall inside steps)."""
    n, R, dx = 4, 1e-3, 10.0
    o = oracle.Oracle(n, n, dx, dx, np.zeros((n, n)), dt_max=0.08, t_end=1.0, rain_rate=R,
                      rain_t_on=0.3, rain_t_off=0.7, library=L)
    o.set_state(np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
    dts = o.run_to(1.0)
    d = o.diag()
    return (d["t"] == 1.0 and abs(float(np.sum(dts)) - 1.0) <= 1e-12 and float(np.max(dts)) <= 0.08
            and math.isclose(d["rain_in"], R * 0.4 * n * n * dx * dx, rel_tol=1e-12))


def pin_maps_and_infiltration_budget(L):
    """Per-cell maps and the infiltration budget over one step of a uniform
    flow on a flat bed between outflow edges: away from the column where the
    Manning map changes (3 cells, the reach of one step) each cell's
    discharge follows the friction recurrence with its own n (Sec. 3.2);
    where the flow stays uniform the infiltrated depth scales with the
    cell's own K_s (Sec. 3.5); the volume falls by the infiltrated volume
    plus the net outflow (cells of 0.5 x 0.25 m)."""
    nx, ny, dx, dy, h0, q0 = 16, 6, 0.5, 0.25, 0.6, 0.3
    col = np.arange(nx)[None, :] * np.ones((ny, 1), dtype=int)
    nmap = np.where(col < nx // 2, 0.02, 0.07)
    ksmap = np.where(np.arange(ny)[:, None] < ny // 2, 2e-5, 5e-5) * np.ones((ny, nx))
    o = oracle.Oracle(nx, ny, dx, dy, np.zeros((ny, nx)), bc=(1, 1, 1, 1), friction=1, n_map=nmap,
                      infiltration=1, ks_map=ksmap, psi=0.1, dtheta=0.3, dt_max=0.05, library=L)
    o.set_state(np.full((ny, nx), h0), np.full((ny, nx), q0), np.zeros((ny, nx)))
    v0 = 0.01
    o.set_vinf(np.full((ny, nx), v0))
    vol0 = o.diag()["volume"]
    dt = o.step(1)[0]
    _, qx, _ = o.state()
    far = np.abs(col - (nx // 2 - 0.5)) >= 3.5
    ok = True
    for nm in (0.02, 0.07):
        k = dt * 9.81 * nm * nm / h0 ** (7.0 / 3.0)
        q1 = q0 / (1.0 + k * abs(q0))
        qe = 0.5 * (q0 + q1 / (1.0 + k * abs(q1)))
        sel = far & (nmap == nm)
        ok &= bool(np.allclose(qx[sel], qe, rtol=1e-14, atol=0))
    dv = o.vinf()[:, 0] - v0                      # column 0: uniform flow all step
    with np.errstate(divide="ignore", invalid="ignore"):
        ok &= bool(np.allclose(dv[ny // 2:] / dv[: ny // 2], 2.5, rtol=1e-12))
    d = o.diag()
    ok &= math.isclose(vol0 - d["volume"], d["infiltrated"] + d["outflow"], rel_tol=1e-9)
    return ok and d["infiltrated"] > 0


def pin_cfl_violation_counter(L):
    """The CFL check at U* (counted, not corrected): a replayed dt of a
    quarter of the bound counts nothing over 3 steps, three times the
    bound counts its step."""
    w = si.random_state(12, 10, seed=4, dry_frac=0.0, vel=0.3)
    counts = []
    for factor, steps in ((0.25, 3), (3.0, 1)):
        o = oracle.Oracle(w.nx, w.ny, w.dx, w.dy, w.z, check_cfl=1, library=L)
        o.set_state(w.h, w.qx, w.qy)
        lx, ly = o.lam()
        o.set_dt_sequence(np.full(steps, factor * 0.5 / (lx / w.dx + ly / w.dy)))
        o.step(steps)
        counts.append(o.diag()["cfl_viol"])
    return counts == [0.0, 1.0]


def pin_cfl_sees_every_imposed_edge(L):
    """The CFL maximum covers an imposed edge's boundary state (it feeds
    the edge fluxes): a fast inflow, depth 0.5 m and discharge 3 m^2/s both
    imposed, beside a lake at rest 1 m deep, on each side in turn -- the
    wave speed along that side's axis is the ghost's 6 + sqrt(0.5 g), the
    other axis keeps the lake's sqrt(g)."""
    n, g, hb, qb = 6, 9.81, 0.5, 3.0
    ok = True
    for side in range(4):
        bc, bh, bq = [0] * 4, [0.0] * 4, [0.0] * 4
        bc[side], bh[side], bq[side] = 4, hb, qb
        o = oracle.Oracle(n, n, 1.0, 1.0, np.zeros((n, n)), bc=bc, bc_h=bh, bc_q=bq, library=L)
        o.set_state(np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
        lam = o.lam()
        fast, still = (lam[0], lam[1]) if side < 2 else (lam[1], lam[0])
        ok &= math.isclose(fast, qb / hb + math.sqrt(g * hb), rel_tol=1e-14)
        ok &= math.isclose(still, math.sqrt(g), rel_tol=1e-14)
    return ok


BATTERY = [pin_mp_second_implementation, pin_lake_at_rest, pin_mass_and_positivity,
           pin_stoker, pin_symmetry, pin_cfl_uniform, pin_cfl_muscl_faces,
           pin_friction_uniform, pin_ponding_time, pin_friction_laws_ode,
           pin_imposed_uniform_channels, pin_torrential_fill, pin_first_order_textbook,
           pin_first_order_lake_and_budget, pin_d8_brute_force, pin_gauges_and_max,
           pin_mp_extension_cases, pin_cfl_min_mode, pin_event_clamps_and_rain_window,
           pin_cfl_violation_counter, pin_maps_and_infiltration_budget, pin_cfl_sees_every_imposed_edge]


def _run_battery(L):
    out = {}
    for pin in BATTERY:
        try:
            out[pin.__name__] = bool(pin(L))
        except Exception:   # a crash or a raised error counts as a failed pin
            out[pin.__name__] = False
    return out


def test_unmodified_oracle_passes_battery(tmp_path):
    L = _build_variant(tmp_path, "unmodified", "double oracle_minmod", "double oracle_minmod")
    res = _run_battery(L)
    assert all(res.values()), res


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    L = _build_variant(tmp_path, name, old, new)
    res = _run_battery(L)
    assert not all(res.values()), f"no pin caught mutation {name}: {res}"

"""Pins of the operation census (oracle/op_census.py).

1. The census's state after each step equals the oracle's bit for bit
   (signed zeros aside) on random wet/dry grids with walls, outflow, each
   friction law, rain, Green-Ampt on a K_s map (V_inf too) and at both
   orders, and its dt sequence equals the oracle's: the census performs
   the oracle's arithmetic.
2. Its counts equal, kind by kind, those of a scalar restatement written
   here whose number type counts every operation it executes, the branches
   taken as Python takes them: the census's masks select the right cells.
3. Closed forms: at a dry cell at rest every count is a fixed number that
   can be read off the scheme (Sec. 3.1, 3.3, 3.4).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import op_census as oc
import swof_inputs as si


# ---------------------------------------------------------------------------
# scalar restatement with a self-counting number type

class CF(float):
    """A float that counts the operations done on it into CF.T."""
    T = None

    def _n(kind):
        CF.T[kind] += 1

    def __add__(s, o):
        CF._n("add")
        return CF(float(s) + float(o))

    def __radd__(s, o):
        CF._n("add")
        return CF(float(o) + float(s))

    def __sub__(s, o):
        CF._n("add")
        return CF(float(s) - float(o))

    def __rsub__(s, o):
        CF._n("add")
        return CF(float(o) - float(s))

    def __mul__(s, o):
        CF._n("mul")
        return CF(float(s) * float(o))

    def __rmul__(s, o):
        CF._n("mul")
        return CF(float(o) * float(s))

    def __truediv__(s, o):
        CF._n("div")
        return CF(float(s) / float(o))

    def __rtruediv__(s, o):
        CF._n("div")
        return CF(float(o) / float(s))

    def __neg__(s):
        return CF(-float(s))

    def __abs__(s):
        CF._n("abs")
        return CF(abs(float(s)))

    def __lt__(s, o):
        CF._n("cmp")
        return float(s) < float(o)

    def __le__(s, o):
        CF._n("cmp")
        return float(s) <= float(o)

    def __gt__(s, o):
        CF._n("cmp")
        return float(s) > float(o)

    def __ge__(s, o):
        CF._n("cmp")
        return float(s) >= float(o)


Z = CF(0.0)


def fmin(a, b):
    CF._n("minmax")
    return CF(a if float(a) <= float(b) else b)


def fmax(a, b):
    CF._n("minmax")
    return CF(a if float(a) >= float(b) else b)


def csqrt(a):
    CF._n("sqrt")
    return CF(math.sqrt(float(a)))


def cicbrt(a):
    CF._n("cbrt")
    return CF(oracle.icbrt(float(a)))


def minmod(a, b):
    if a >= 0.0 and b >= 0.0:
        return fmin(a, b)
    if a <= 0.0 and b <= 0.0:
        return fmax(a, b)
    return Z


class Scalar:
    """One run, cell by cell, the oracle's loops with each value computed
    once (the velocities and reconstruction of U^n shared by the wave
    speeds and stage 1)."""

    def __init__(self, w, friction, coef, rain, order=2, vinf=None):
        self.order, self.inf = order, bool(w.infiltration)
        self.ks = w.ks
        self.psi, self.dtheta = w.psi, w.dtheta
        self.vinf = [[CF(float(vinf[j][i])) if vinf is not None else Z for i in range(w.nx)]
                     for j in range(w.ny)]
        self.infsum = 0.0
        self.nx, self.ny, self.dx, self.dy = w.nx, w.ny, w.dx, w.dy
        self.g, self.hd, self.bc = 9.81, w.h_dry, w.bc
        self.fr = friction
        self.cf = (coef * coef if friction == 1 else coef / (8.0 * 9.81) if friction == 3
                   else 1.0 / (coef * coef) if friction in (2, 4) else 0.0)
        self.cfl, self.dtmax, self.rain = w.cfl, w.dt_max, rain
        self.z = self._pad(w.z)
        self._ghosts(self.z, 1, 1)
        self.h, self.qx, self.qy = self._pad(w.h), self._pad(w.qx), self._pad(w.qy)
        self.T = dict.fromkeys(oc.KINDS, 0)

    def _pad(self, a):
        p = [[Z] * (self.nx + 4) for _ in range(self.ny + 4)]
        for j in range(self.ny):
            for i in range(self.nx):
                p[j + 2][i + 2] = CF(float(a[j][i]))
        return p

    def _ghosts(self, a, sx, sy):
        nx, ny, bc = self.nx, self.ny, self.bc
        fx = (lambda v: -v) if sx < 0 else (lambda v: v)
        fy = (lambda v: -v) if sy < 0 else (lambda v: v)
        for j in range(2, ny + 2):
            for k in (0, 1):
                a[j][1 - k] = fx(a[j][2 + k]) if bc[0] == 0 else a[j][2]
                a[j][nx + 2 + k] = fx(a[j][nx + 1 - k]) if bc[1] == 0 else a[j][nx + 1]
        for i in range(2, nx + 2):
            for k in (0, 1):
                a[1 - k][i] = fy(a[2 + k][i]) if bc[2] == 0 else a[2][i]
                a[ny + 2 + k][i] = fy(a[ny + 1 - k][i]) if bc[3] == 0 else a[ny + 1][i]

    def _vel(self, h, qx, qy):
        nx, ny = self.nx, self.ny
        u = [[Z] * (nx + 4) for _ in range(ny + 4)]
        v = [[Z] * (nx + 4) for _ in range(ny + 4)]
        for pj in range(ny + 4):
            for pi in range(nx + 4):
                if not (2 <= pj < ny + 2 or 2 <= pi < nx + 2):
                    continue                      # corners: never read
                if h[pj][pi] > self.hd:
                    rh = 1.0 / h[pj][pi]
                    u[pj][pi] = qx[pj][pi] * rh
                    v[pj][pi] = qy[pj][pi] * rh
        return u, v

    def _muscl(self, h, z, un, ut, c, m, p):
        (cj, ci), (mj, mi), (pj, pi) = c, m, p
        hc, hm, hp = h[cj][ci], h[mj][mi], h[pj][pi]
        dh = minmod(hc - hm, hp - hc)
        half = 0.5 * dh
        hmv, hpv = hc - half, hc + half
        em, ec, ep = hm + z[mj][mi], hc + z[cj][ci], hp + z[pj][pi]
        de = minmod(ec - em, ep - ec)
        halfe = 0.5 * de
        etam, etap = ec - halfe, ec + halfe
        zmv, zpv = etam - hmv, etap - hpv
        unc, utc = un[cj][ci], ut[cj][ci]
        if hc > self.hd:
            rh = 1.0 / hc
            dun = minmod(unc - un[mj][mi], un[pj][pi] - unc)
            dut = minmod(utc - ut[mj][mi], ut[pj][pi] - utc)
            a, b = hpv * rh, hmv * rh
            hu, ht = 0.5 * dun, 0.5 * dut
            return hmv, hpv, zmv, zpv, unc - a * hu, unc + b * hu, utc - a * ht, utc + b * ht
        return hmv, hpv, zmv, zpv, unc, unc, utc, utc

    def _recon1(self, h, u, v):
        """first order: face values = cell values (no arithmetic)"""
        nx, ny, z = self.nx, self.ny, self.z
        X, Y = {}, {}
        for j in range(ny):
            for i in range(-1, nx + 1):
                c = (j + 2, i + 2)
                X[i, j] = (h[c[0]][c[1]],) * 2 + (z[c[0]][c[1]],) * 2 + (u[c[0]][c[1]],) * 2 + (v[c[0]][c[1]],) * 2
        for j in range(-1, ny + 1):
            for i in range(nx):
                c = (j + 2, i + 2)
                Y[i, j] = (h[c[0]][c[1]],) * 2 + (z[c[0]][c[1]],) * 2 + (v[c[0]][c[1]],) * 2 + (u[c[0]][c[1]],) * 2
        return X, Y

    def _recon(self, h, u, v):
        if self.order == 1:
            return self._recon1(h, u, v)
        nx, ny = self.nx, self.ny
        X, Y = {}, {}
        for j in range(ny):
            for i in range(-1, nx + 1):
                X[i, j] = self._muscl(h, self.z, u, v, (j + 2, i + 2), (j + 2, i + 1), (j + 2, i + 3))
        for j in range(-1, ny + 1):
            for i in range(nx):
                Y[i, j] = self._muscl(h, self.z, v, u, (j + 2, i + 2), (j + 1, i + 2), (j + 3, i + 2))
        return X, Y

    def _face(self, a, b):
        g, hg = self.g, 0.5 * self.g
        hpa, zpa, unpa, utpa = a[1], a[3], a[5], a[7]
        hmb, zmb, unmb, utmb = b[0], b[2], b[4], b[6]
        zmax = fmax(zpa, zmb)
        hL = fmax(Z, (hpa + zpa) - zmax)
        hR = fmax(Z, (hmb + zmb) - zmax)
        cL, cR = csqrt(g * hL), csqrt(g * hR)
        c1 = fmin(unpa - cL, unmb - cR)
        c2 = fmax(unpa + cL, unmb + cR)
        qL, qR = hL * unpa, hR * unmb
        FL = (qL, qL * unpa + hg * hL * hL, qL * utpa)
        FR = (qR, qR * unmb + hg * hR * hR, qR * utmb)
        if c1 >= 0.0:
            F = FL
        elif c2 <= 0.0:
            F = FR
        else:
            UL = (hL, qL, hL * utpa)
            UR = (hR, qR, hR * utmb)
            r = 1.0 / (c2 - c1)
            w = c1 * c2 * r
            F = tuple((c2 * FL[k] - c1 * FR[k]) * r + w * (UR[k] - UL[k]) for k in range(3))
        return F[0], F[1] + hg * (hpa * hpa - hL * hL), F[1] + hg * (hmb * hmb - hR * hR), F[2]

    def _stage(self, h, qx, qy, dt, u, v, X, Y):
        nx, ny, hg = self.nx, self.ny, 0.5 * self.g
        fx = {(i, j): self._face(X[i, j], X[i + 1, j]) for j in range(ny) for i in range(-1, nx)}
        fy = {(i, j): self._face(Y[i, j], Y[i, j + 1]) for j in range(-1, ny) for i in range(nx)}
        dtdx, dtdy = dt / self.dx, dt / self.dy
        out = [[None] * nx for _ in range(ny)], [[None] * nx for _ in range(ny)], [[None] * nx for _ in range(ny)]
        for j in range(ny):
            for i in range(nx):
                x, y = X[i, j], Y[i, j]
                fcx = hg * (x[0] + x[1]) * (x[3] - x[2])
                fcy = hg * (y[0] + y[1]) * (y[3] - y[2])
                E, W, N, S = fx[i, j], fx[i - 1, j], fy[i, j], fy[i, j - 1]
                c = (j + 2, i + 2)
                hs = h[c[0]][c[1]] - dtdx * (E[0] - W[0]) - dtdy * (N[0] - S[0])
                qxs = qx[c[0]][c[1]] - dtdx * ((E[1] - W[2]) + fcx) - dtdy * (N[3] - S[3])
                qys = qy[c[0]][c[1]] - dtdx * (E[3] - W[3]) - dtdy * ((N[1] - S[2]) + fcy)
                if hs > self.hd:
                    if self.fr:
                        uc, vc = u[c[0]][c[1]], v[c[0]][c[1]]
                        speed = csqrt(uc * uc + vc * vc)
                        if self.fr <= 2:
                            yv = cicbrt(hs)
                            yy = yv * yv
                            hinv = yy * yy
                        else:
                            hinv = 1.0 / hs
                        k = dt * self.g * self.cf
                        rden = 1.0 / (1.0 + k * speed * hinv)
                        qxs, qys = qxs * rden, qys * rden
                else:
                    qxs = qys = Z
                out[0][j][i], out[1][j][i], out[2][j][i] = hs, qxs, qys
        return out

    def step(self):
        CF.T = self.T
        nx, ny, g = self.nx, self.ny, self.g
        h, qx, qy = self.h, self.qx, self.qy
        self._ghosts(h, 1, 1)
        self._ghosts(qx, -1, 1)
        self._ghosts(qy, 1, -1)
        u, v = self._vel(h, qx, qy)
        X, Y = self._recon(h, u, v)
        lx = ly = 0.0
        for j in range(ny):
            for i in range(nx):
                x, y = X[i, j], Y[i, j]
                a = fmax(abs(x[4]) + csqrt(g * x[0]), abs(x[5]) + csqrt(g * x[1]))
                b = fmax(abs(y[4]) + csqrt(g * y[0]), abs(y[5]) + csqrt(g * y[1]))
                lx = float(fmax(a, lx))
                ly = float(fmax(b, ly))
        den = lx / self.dx + ly / self.dy
        dt = min(self.cfl / den if den > 0.0 else self.dtmax, self.dtmax)
        s1 = self._stage(h, qx, qy, dt, u, v, X, Y)
        if self.order == 2:
            p1 = [self._pad(np.array(a, dtype=object)) for a in s1]
            self._ghosts(p1[0], 1, 1)
            self._ghosts(p1[1], -1, 1)
            self._ghosts(p1[2], 1, -1)
            u1, v1 = self._vel(*p1)
            X1, Y1 = self._recon(p1[0], u1, v1)
            s2 = self._stage(*p1, dt, u1, v1, X1, Y1)
        for j in range(ny):
            for i in range(nx):
                c = (j + 2, i + 2)
                if self.order == 1:
                    hn, qxn, qyn = s1[0][j][i], s1[1][j][i], s1[2][j][i]
                else:
                    hn = 0.5 * (h[c[0]][c[1]] + s2[0][j][i])
                    qxn = 0.5 * (qx[c[0]][c[1]] + s2[1][j][i])
                    qyn = 0.5 * (qy[c[0]][c[1]] + s2[2][j][i])
                if self.rain > 0.0:
                    hn = hn + dt * self.rain
                if self.inf:
                    vi = self.vinf[j][i]
                    ks = float(self.ks[j][i]) if self.ks is not None else 0.0
                    if vi > 0.0:
                        ic = ks * (1.0 + ((self.psi + hn) * self.dtheta) / vi)
                        d = fmin(hn, dt * ic)
                    else:
                        d = hn
                    hn = hn - d
                    self.vinf[j][i] = vi + d
                    self.infsum = self.infsum + d
                if hn <= self.hd:
                    qxn = qyn = Z
                h[c[0]][c[1]], qx[c[0]][c[1]], qy[c[0]][c[1]] = hn, qxn, qyn
        return dt

    def state(self):
        return tuple(np.array([[float(a[j + 2][i + 2]) for i in range(self.nx)] for j in range(self.ny)])
                     for a in (self.h, self.qx, self.qy))


# ---------------------------------------------------------------------------

def _case(seed, nx, ny, dry_frac, bc, friction, rain, order=2, ga=False):
    """A random wet/dry workload; with ga, Green-Ampt on a K_s map and a
    starting infiltrated depth that is zero in some cells."""
    w = si.random_state(nx, ny, seed, dry_frac=dry_frac)
    w.bc = bc
    w.friction = friction
    w.manning_n = {1: 0.03, 2: 30.0, 3: 0.05, 4: 40.0}.get(friction, 0.0)
    w.rain_rate = rain
    vinf = None
    if ga:
        rng = np.random.default_rng(seed + 100)
        w.infiltration, w.psi, w.dtheta = 1, 0.1, 0.3
        w.ks = 1e-4 * np.exp(0.5 * rng.standard_normal((ny, nx)))
        vinf = 0.01 * rng.random((ny, nx)) * (rng.random((ny, nx)) < 0.7)
    return w, order, vinf


CASES = [
    (1, 9, 7, 0.3, (0, 1, 0, 1), 1, 0.0),
    (2, 8, 10, 0.5, (1, 0, 1, 0), 3, 0.0),
    (3, 11, 6, 0.0, (0, 0, 0, 0), 2, 1e-3),
    (4, 7, 7, 0.8, (1, 1, 1, 1), 4, 0.0),
    (5, 10, 9, 0.2, (0, 1, 1, 0), 0, 2e-4),
    (6, 9, 8, 0.3, (0, 1, 0, 1), 1, 0.0, 1),
    (7, 10, 7, 0.2, (1, 0, 0, 1), 3, 5e-4, 1, True),
    (8, 8, 9, 0.3, (0, 0, 1, 1), 1, 5e-4, 2, True),
]


def _census(w, order, vinf):
    return oc.Census(w.z, w.h, w.qx, w.qy, w.dx, w.dy, h_dry=w.h_dry, bc=w.bc, friction=w.friction,
                     friction_coef=w.manning_n, cfl=w.cfl, dt_max=w.dt_max, rain_rate=w.rain_rate,
                     order=order, infiltration=bool(w.infiltration), ks_map=w.ks, psi=w.psi,
                     dtheta=w.dtheta, vinf=vinf)


@pytest.mark.parametrize("case", CASES)
def test_census_matches_oracle_bitwise(case):
    w, order, vinf = _case(*case)
    o = oracle.Oracle.from_workload(w, friction_coef=w.manning_n, rain_t_on=0.0, rain_t_off=1e9, order=order)
    if vinf is not None:
        o.set_vinf(vinf)
    c = _census(w, order, vinf)
    for _ in range(3):
        dto = o.step(1)[0]
        dtc = c.step()
        assert dtc == dto
        for a, b in zip(c.state(), o.state()):
            assert np.array_equal(a, b)
        if vinf is not None:
            assert np.array_equal(c.vinf, o.vinf())


@pytest.mark.parametrize("case", CASES)
def test_census_counts_equal_scalar_count(case):
    w, order, vinf = _case(*case)
    c = _census(w, order, vinf)
    s = Scalar(w, w.friction, w.manning_n, w.rain_rate, order, vinf)
    for _ in range(2):
        assert c.step() == s.step()
        for a, b in zip(c.state(), s.state()):
            assert np.array_equal(a, b)
        assert c.T.n == s.T


def test_icbrt_equals_oracle():
    rng = np.random.default_rng(7)
    x = np.concatenate([10.0 ** rng.uniform(-12, 6, 2000), [1e-6, 0.125, 1.0, 2.0, 3.0, 8.0, 1e300, 5e-324 * 2 ** 60]])
    y = oc.icbrt(x)
    for a, b in zip(x, y):
        assert b == oracle.icbrt(float(a))


def test_dry_cell_at_rest_counts():
    """A dry flat bed at rest: every quantity is zero, so each cell takes
    the dry branch everywhere and the per-cell counts are fixed numbers
    (walls on every side; ghosts and edge faces add their own share)."""
    n = 12
    z = np.zeros((n, n))
    c = oc.Census(z, z, z, z, 1.0, 1.0, bc=(0, 0, 0, 0), friction=1, friction_coef=0.03)
    c.step()
    # per interior cell and stage (all values zero: every minmod takes a >= 0 and b >= 0,
    # c1 = 0 takes the first HLL branch, no cell is wet):
    #   velocities: 1 cmp
    #   MUSCL, per direction: 13 add (2 + 2 h, 3 + 2 + 2 eta, 2 z), 2 mul, 5 cmp, 2 minmax
    #   face, per direction: 14 add, 18 mul (2 + 10 flux, 6 S_L S_R), 2 sqrt, 5 minmax, 1 cmp
    #   centred terms and update: 18 add, 10 mul, 1 cmp
    # and once per step: wave speeds 4 abs 4 mul 4 sqrt 4 add 4 minmax; Heun 3 add 3 mul 1 cmp
    per_stage_cell = {"add": 2 * 13 + 2 * 14 + 18, "mul": 2 * 2 + 2 * 18 + 10, "sqrt": 2 * 2,
                      "minmax": 2 * 2 + 2 * 5, "cmp": 1 + 2 * 5 + 2 * 1 + 1}
    # ghost cells reconstructed: 2 per row (x) and 2 per column (y); extra faces: 1 per row and column;
    # velocities on the 2-layer ghost strips
    rec_extra, face_extra, vel_extra = 4 * n, 2 * n, 8 * n
    cells = n * n
    exp = {
        "add": 2 * (per_stage_cell["add"] * cells + 13 * rec_extra + 14 * face_extra) + 4 * cells + 3 * cells,
        "mul": 2 * (per_stage_cell["mul"] * cells + 2 * rec_extra + 18 * face_extra) + 4 * cells + 3 * cells,
        "sqrt": 2 * (per_stage_cell["sqrt"] * cells + 2 * face_extra) + 4 * cells,
        "minmax": 2 * (per_stage_cell["minmax"] * cells + 2 * rec_extra + 5 * face_extra) + 4 * cells,
        "cmp": 2 * (per_stage_cell["cmp"] * cells + 5 * rec_extra + face_extra + vel_extra) + cells,
        "abs": 4 * cells, "div": 0, "cbrt": 0,
    }
    assert c.T.n == exp


def test_wet_cells_cost_more_than_dry():
    """Per cell-update counts grow with the wet fraction, and a fully wet
    subcritical grid takes the friction, velocity and middle-HLL work at
    every cell."""
    per = []
    for frac in (1.0, 0.5, 0.0):
        w = si.random_state(16, 16, 3, dry_frac=frac, vel=0.1)
        c = oc.Census(w.z, w.h, w.qx, w.qy, w.dx, w.dy, bc=w.bc, friction=1, friction_coef=0.03)
        c.step()
        per.append(c.T.per(256))
    assert per[0]["flops"] < per[1]["flops"] < per[2]["flops"]
    assert per[2]["cbrt"] == pytest.approx(2.0)          # one inverse cube root per cell and stage


def test_committed_census_summary_matches_a_fresh_census():
    """The committed per-cell-update figures (written by the census script
    on the 4096^2 valley) agree with a fresh census of the same fully wet
    workload at 256^2 (edge cells and flow state differ slightly with the
    size: 1 %), and bench.py reads them back."""
    import copy
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    stored = bench.census_per_update("fully_wet")
    assert stored is not None and set(oc.KINDS) <= set(stored)
    w = si.valley(256)
    wet = copy.copy(w)
    wet.h = w.h + 0.5
    c, _ = oc.census(wet, 1)
    fresh = c.T.per(256 * 256)
    for k in ("add", "mul", "flops", "all"):
        assert stored[k] == pytest.approx(fresh[k], rel=0.01)
    assert stored["cbrt"] == pytest.approx(2.0, abs=1e-3)
    assert stored["flops"] == pytest.approx(sum(stored[k] for k in ("add", "mul", "div", "sqrt", "cbrt")),
                                            abs=0.01)
    r = bench.alu_roofline("fp64", 0.5, 2070.0)
    assert r["frac"] == pytest.approx(stored["flops"] * 0.5e9 / 0.625e12)

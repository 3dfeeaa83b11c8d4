"""Exact operation census of one time step of the scheme -- TEST INFRASTRUCTURE.

Counts, by kind, the floating-point operations that one second-order Heun
step (Algorithm 1: the CFL time step of Eq. (cfl), two stages of the
hydrostatic-reconstruction scheme of Sec. 3.1 with the HLL flux of
Sec. 3.3, the MUSCL-minmod reconstruction of Sec. 3.4 and the
semi-implicit friction of Sec. 3.2, then the Heun average) performs on a
given state.  Kinds: add (and subtract), mul, div, sqrt, cbrt (one inverse
cube root h^{-1/3}), minmax (min, max, and the running maximum of the
wave speeds), abs, cmp (a comparison that decides a branch or a clean-up).

What is counted is the oracle's own arithmetic in the oracle's operation
order, with each value the scheme defines computed once:
  - per cell and stage: the velocities (Sec. 3.4, zero at dry cells);
  - per cell, direction and stage: the MUSCL reconstruction (as the
    oracle's muscl_cell does it, from the cell and its two neighbours);
  - per face and stage: the hydrostatic reconstruction, the HLL flux and
    the two well-balancing corrections S_L, S_R;
  - per cell and stage: the centred term Fc, the update and the friction;
  - per cell and step: the wave speeds of Eq. (cfl), read from stage 1's
    reconstruction of U^n (the oracle reconstructs U^n a second time for
    them; that repeat is the same arithmetic and is not counted), and the
    Heun average, rain and the dry clean-up.
Products of per-run or per-step constants (g/2, dt/dx, dt/dy, dt g C_f,
dt R) are not counted; neither are the ghost copies (sign flips) nor the
O(nx + ny) edge-flux budget.  Cells outside the interior that the
reconstruction needs (two ghost layers per side, no corners) are counted
where the work is done for them.

The arithmetic is numpy over the whole grid: a value is computed
everywhere and kept where its branch is taken, and every operation adds
the number of cells (or faces) that take the branch it sits in.  The
resulting state matches the oracle's bit for bit (ties of signed zeros
aside), and the counts equal those of a scalar restatement whose number
type counts its own operations (tests/test_op_census.py).

At first order (Sec. 3.3) the face values are the cell values (no
reconstruction arithmetic), the wave speeds are taken on them, and one
Euler stage replaces the two Heun stages.  Green-Ampt infiltration
(Sec. 3.5) is counted per cell after the rain, with the step's
infiltration sum.

Supported: order 1 or 2, wall and free-outflow edges, no friction or one of
the four laws with a scalar coefficient, uniform rain on or off,
Green-Ampt with a scalar or per-cell K_s; no imposed edges.
"""
from __future__ import annotations

import numpy as np

KINDS = ("add", "mul", "div", "sqrt", "cbrt", "minmax", "abs", "cmp")

# x^{-1/3} start-value factors 2^{-r/3}, r = 0, 1, 2 (the oracle's Newton cube root)
_SR = np.array([1.0, 0.79370052598409973738, 0.62996052494743658238])


def icbrt(x: np.ndarray) -> np.ndarray:
    """x^{-1/3} for x > 0 by the oracle's method: a start value from the
    exponent bits (x = m 2^e, e = 3k + r) and four Newton steps on
    y^{-3} - x.  Elementwise, the same operations in the same order."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    bits = x.view(np.uint64)
    e = ((bits >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023
    mb = (bits & np.uint64(0x000FFFFFFFFFFFFF)) | np.uint64(0x3FF0000000000000)
    m = mb.view(np.float64)
    k = np.where(e >= 0, e // 3, -((-e + 2) // 3))
    r = e - 3 * k
    p2 = ((1023 - k).astype(np.uint64) << np.uint64(52)).view(np.float64)
    y = (1.0 - 0.2063 * (m - 1.0)) * _SR[r] * p2
    third = 1.0 / 3.0
    for _ in range(4):
        t = x * y * y * y
        y = y + y * (1.0 - t) * third
    return y


class Tally:
    """Operation counts by kind."""

    def __init__(self):
        self.n = dict.fromkeys(KINDS, 0)

    def c(self, kind: str, where, times: int = 1):
        """Add `times` operations of `kind` for every cell in `where` (a
        boolean mask, or a count)."""
        k = int(np.count_nonzero(where)) if isinstance(where, np.ndarray) else int(where)
        self.n[kind] += times * k

    def flops(self) -> int:
        """Arithmetic operations: add, mul, div, sqrt, cbrt."""
        return sum(self.n[k] for k in ("add", "mul", "div", "sqrt", "cbrt"))

    def total(self) -> int:
        return sum(self.n.values())

    def per(self, cells: int) -> dict:
        d = {k: self.n[k] / cells for k in KINDS}
        d["flops"] = self.flops() / cells
        d["all"] = self.total() / cells
        return d


def _minmod(T, a, b, m):
    """Sec. 3.4 limiter; comparisons counted as the oracle's short-circuit
    tests execute them."""
    A = a >= 0.0
    B = b >= 0.0
    T.c("cmp", m)
    T.c("cmp", m & A)
    P = A & B
    C = a <= 0.0
    D = b <= 0.0
    T.c("cmp", m & ~P)
    T.c("cmp", m & ~P & C)
    N = ~P & C & D
    T.c("minmax", m & P)
    T.c("minmax", m & N)
    return np.where(P, np.fmin(a, b), np.where(N, np.fmax(a, b), 0.0))


def _ghosts(a, bc, sx, sy):
    """Two ghost layers (wall: mirror, times sx / sy for the normal
    discharge; outflow: the edge cell extended); corners untouched."""
    ny, nx = a.shape[0] - 4, a.shape[1] - 4
    J, I = slice(2, ny + 2), slice(2, nx + 2)
    for k in (0, 1):
        a[J, 1 - k] = sx * a[J, 2 + k] if bc[0] == 0 else a[J, 2]
        a[J, nx + 2 + k] = sx * a[J, nx + 1 - k] if bc[1] == 0 else a[J, nx + 1]
    for k in (0, 1):
        a[1 - k, I] = sy * a[2 + k, I] if bc[2] == 0 else a[2, I]
        a[ny + 2 + k, I] = sy * a[ny + 1 - k, I] if bc[3] == 0 else a[ny + 1, I]


def _pad(a):
    ny, nx = a.shape
    p = np.zeros((ny + 4, nx + 4))
    p[2:ny + 2, 2:nx + 2] = a
    return p


class _Rec:
    pass


def _muscl(T, hdry, hc, hm_, hp_, zc, zm_, zp_, unc, unm_, unp_, utc, utm_, utp_):
    """One MUSCL reconstruction per cell of the arrays (c: the cell, m / p:
    its minus / plus neighbours along the direction); un, ut = normal and
    transverse velocity."""
    al = np.ones(hc.shape, dtype=bool)
    r = _Rec()
    T.c("add", al, 2)
    dh = _minmod(T, hc - hm_, hp_ - hc, al)
    T.c("mul", al)
    T.c("add", al, 2)
    r.hm = hc - 0.5 * dh
    r.hp = hc + 0.5 * dh
    T.c("add", al, 3)
    em, ec, ep = hm_ + zm_, hc + zc, hp_ + zp_
    T.c("add", al, 2)
    de = _minmod(T, ec - em, ep - ec, al)
    T.c("mul", al)
    T.c("add", al, 2)
    etam, etap = ec - 0.5 * de, ec + 0.5 * de
    T.c("add", al, 2)
    r.zm, r.zp = etam - r.hm, etap - r.hp
    W = hc > hdry
    T.c("cmp", al)
    T.c("div", W)
    with np.errstate(divide="ignore", invalid="ignore"):
        rh = 1.0 / np.where(W, hc, 1.0)
    T.c("add", W, 4)
    dun = _minmod(T, unc - unm_, unp_ - unc, W)
    dut = _minmod(T, utc - utm_, utp_ - utc, W)
    T.c("mul", W, 8)
    T.c("add", W, 4)
    a, b = r.hp * rh, r.hm * rh
    hu, ht = 0.5 * dun, 0.5 * dut
    r.unm = np.where(W, unc - a * hu, unc)
    r.unp = np.where(W, unc + b * hu, unc)
    r.utm = np.where(W, utc - a * ht, utc)
    r.utp = np.where(W, utc + b * ht, utc)
    return r


def _face(T, g, hg, hpa, zpa, unpa, utpa, hmb, zmb, unmb, utmb):
    """Hydrostatic reconstruction, HLL flux and S_L, S_R at the faces
    between the a cells (their plus side) and the b cells (minus side)."""
    al = np.ones(hpa.shape, dtype=bool)
    T.c("minmax", al, 3)
    T.c("add", al, 4)
    zmax = np.fmax(zpa, zmb)
    hL = np.fmax(0.0, (hpa + zpa) - zmax)
    hR = np.fmax(0.0, (hmb + zmb) - zmax)
    T.c("mul", al, 2)
    T.c("sqrt", al, 2)
    cL, cR = np.sqrt(g * hL), np.sqrt(g * hR)
    T.c("add", al, 4)
    T.c("minmax", al, 2)
    c1 = np.fmin(unpa - cL, unmb - cR)
    c2 = np.fmax(unpa + cL, unmb + cR)
    T.c("mul", al, 10)
    T.c("add", al, 2)
    qL, qR = hL * unpa, hR * unmb
    FL = (qL, qL * unpa + hg * hL * hL, qL * utpa)
    FR = (qR, qR * unmb + hg * hR * hR, qR * utmb)
    S1 = c1 >= 0.0
    S2 = c2 <= 0.0
    T.c("cmp", al)
    T.c("cmp", ~S1)
    M = ~S1 & ~S2
    # middle branch: 2 mul (transverse discharges), c2 - c1, 1/(c2 - c1),
    # c1 c2 r, then per component 4 mul and 3 add
    T.c("mul", M, 2 + 2 + 12)
    T.c("add", M, 1 + 9)
    T.c("div", M)
    with np.errstate(divide="ignore", invalid="ignore"):
        UL = (hL, qL, hL * utpa)
        UR = (hR, qR, hR * utmb)
        rr = 1.0 / np.where(M, c2 - c1, 1.0)
        w = c1 * c2 * rr
        F = [np.where(S1, FL[k], np.where(S2, FR[k], (c2 * FL[k] - c1 * FR[k]) * rr + w * (UR[k] - UL[k])))
             for k in range(3)]
    T.c("mul", al, 6)
    T.c("add", al, 4)
    f2l = F[1] + hg * (hpa * hpa - hL * hL)
    f2r = F[1] + hg * (hmb * hmb - hR * hR)
    return F[0], f2l, f2r, F[2]


def _friction_cf(law, g, coef):
    """C_f of Sec. 2.1: Manning n^2, Strickler 1/K^2, Darcy-Weisbach
    f/(8g), Chezy 1/C^2."""
    if law == 1:
        return coef * coef
    if law in (2, 4):
        return 1.0 / (coef * coef)
    if law == 3:
        return coef / (8.0 * g)
    return 0.0


class Census:
    """The state of one run and the counts of the steps taken so far."""

    def __init__(self, z, h, qx, qy, dx, dy, *, g=9.81, h_dry=1e-6, bc=(0, 0, 0, 0), friction=0,
                 friction_coef=0.0, cfl=0.5, dt_max=0.1, rain_rate=0.0, order=2, infiltration=False,
                 ks=0.0, ks_map=None, psi=0.0, dtheta=0.0, vinf=None):
        if any(b not in (0, 1) for b in bc):
            raise ValueError("the census covers wall and outflow edges only")
        if order not in (1, 2):
            raise ValueError("order is 1 or 2")
        self.order, self.infiltration = int(order), bool(infiltration)
        self.ks = np.asarray(ks_map, dtype=np.float64) if ks_map is not None else float(ks)
        self.psi, self.dtheta = float(psi), float(dtheta)
        self.vinf = (np.array(vinf, dtype=np.float64) if vinf is not None
                     else np.zeros(np.shape(z), dtype=np.float64))
        self.ny, self.nx = np.shape(z)
        self.dx, self.dy, self.g, self.hdry = float(dx), float(dy), float(g), float(h_dry)
        self.bc, self.friction = tuple(int(b) for b in bc), int(friction)
        self.cf = _friction_cf(self.friction, self.g, float(friction_coef))
        self.cfl, self.dt_max, self.rain = float(cfl), float(dt_max), float(rain_rate)
        self.z = _pad(np.asarray(z, dtype=np.float64))
        _ghosts(self.z, self.bc, 1.0, 1.0)
        self.h, self.qx, self.qy = (_pad(np.asarray(a, dtype=np.float64)) for a in (h, qx, qy))
        self.T = Tally()
        self.steps = 0
        ny, nx = self.ny, self.nx
        # cells whose velocities the reconstruction reads: interior + 2 ghost layers, no corners
        self.vmask = np.zeros((ny + 4, nx + 4), dtype=bool)
        self.vmask[2:ny + 2, :] = True
        self.vmask[:, 2:nx + 2] = True

    def state(self):
        ny, nx = self.ny, self.nx
        return tuple(a[2:ny + 2, 2:nx + 2].copy() for a in (self.h, self.qx, self.qy))

    def _recon1(self, h, u, v):
        """First order: the face values are the cell values (copies, no
        arithmetic), over the same cells as the MUSCL reconstruction."""
        ny, nx, z = self.ny, self.nx, self.z
        out = []
        for rows, cols, un, ut in ((slice(2, ny + 2), slice(1, nx + 3), u, v),
                                   (slice(1, ny + 3), slice(2, nx + 2), v, u)):
            r = _Rec()
            r.hm = r.hp = h[rows, cols]
            r.zm = r.zp = z[rows, cols]
            r.unm = r.unp = un[rows, cols]
            r.utm = r.utp = ut[rows, cols]
            out.append(r)
        return tuple(out)

    def _velocities(self, h, qx, qy):
        T = self.T
        W = h > self.hdry
        T.c("cmp", self.vmask)
        T.c("div", self.vmask & W)
        T.c("mul", self.vmask & W, 2)
        with np.errstate(divide="ignore", invalid="ignore"):
            rh = 1.0 / np.where(W, h, 1.0)
        return np.where(W, qx * rh, 0.0), np.where(W, qy * rh, 0.0)

    def _recon(self, h, u, v):
        ny, nx, z, hd, T = self.ny, self.nx, self.z, self.hdry, self.T
        J, C, Mi, Pi = slice(2, ny + 2), slice(1, nx + 3), slice(0, nx + 2), slice(2, nx + 4)
        X = _muscl(T, hd, h[J, C], h[J, Mi], h[J, Pi], z[J, C], z[J, Mi], z[J, Pi],
                   u[J, C], u[J, Mi], u[J, Pi], v[J, C], v[J, Mi], v[J, Pi])
        I, Cj, Mj, Pj = slice(2, nx + 2), slice(1, ny + 3), slice(0, ny + 2), slice(2, ny + 4)
        Y = _muscl(T, hd, h[Cj, I], h[Mj, I], h[Pj, I], z[Cj, I], z[Mj, I], z[Pj, I],
                   v[Cj, I], v[Mj, I], v[Pj, I], u[Cj, I], u[Mj, I], u[Pj, I])
        return X, Y

    def _stage(self, h, qx, qy, dt, pre=None):
        """One stage U -> U + dt Phi(U) (friction included) on padded
        arrays whose ghosts are filled; `pre` = the velocities and the
        reconstruction of U when already done.  Returns the interior
        result."""
        ny, nx, g, T = self.ny, self.nx, self.g, self.T
        hg = 0.5 * g
        if pre is None:
            u, v = self._velocities(h, qx, qy)
            X, Y = self._recon(h, u, v)
        else:
            u, v, X, Y = pre
        # x faces i + 1/2 for i in [-1, nx): recon columns a = i + 1, b = i + 2
        fx = _face(T, g, hg, X.hp[:, 0:nx + 1], X.zp[:, 0:nx + 1], X.unp[:, 0:nx + 1], X.utp[:, 0:nx + 1],
                   X.hm[:, 1:nx + 2], X.zm[:, 1:nx + 2], X.unm[:, 1:nx + 2], X.utm[:, 1:nx + 2])
        fy = _face(T, g, hg, Y.hp[0:ny + 1], Y.zp[0:ny + 1], Y.unp[0:ny + 1], Y.utp[0:ny + 1],
                   Y.hm[1:ny + 2], Y.zm[1:ny + 2], Y.unm[1:ny + 2], Y.utm[1:ny + 2])
        # interior cells: recon column i + 1 (x) / row j + 1 (y); east face i + 1, west i
        xe, xw, yn, ys = slice(1, nx + 1), slice(0, nx), slice(1, ny + 1), slice(0, ny)
        al = np.ones((ny, nx), dtype=bool)
        T.c("add", al, 4)
        T.c("mul", al, 4)
        fcx = hg * (X.hm[:, xe] + X.hp[:, xe]) * (X.zp[:, xe] - X.zm[:, xe])
        fcy = hg * (Y.hm[yn, :] + Y.hp[yn, :]) * (Y.zp[yn, :] - Y.zm[yn, :])
        dtdx, dtdy = dt / self.dx, dt / self.dy
        J, I = slice(2, ny + 2), slice(2, nx + 2)
        T.c("add", al, 14)
        T.c("mul", al, 6)
        hs = h[J, I] - dtdx * (fx[0][:, xe] - fx[0][:, xw]) - dtdy * (fy[0][yn, :] - fy[0][ys, :])
        qxs = (qx[J, I] - dtdx * ((fx[1][:, xe] - fx[2][:, xw]) + fcx)
               - dtdy * (fy[3][yn, :] - fy[3][ys, :]))
        qys = (qy[J, I] - dtdx * (fx[3][:, xe] - fx[3][:, xw])
               - dtdy * ((fy[1][yn, :] - fy[2][ys, :]) + fcy))
        W = hs > self.hdry
        T.c("cmp", al)
        if self.friction:
            uc, vc = u[J, I], v[J, I]
            T.c("mul", W, 2)
            T.c("add", W)
            T.c("sqrt", W)
            speed = np.sqrt(uc * uc + vc * vc)
            hpos = np.where(W, hs, 1.0)
            if self.friction <= 2:
                T.c("cbrt", W)
                T.c("mul", W, 2)
                y = icbrt(hpos)
                hinv = (y * y) * (y * y)
            else:
                T.c("div", W)
                hinv = 1.0 / hpos
            k = dt * g * self.cf
            T.c("mul", W, 2 + 2)
            T.c("add", W)
            T.c("div", W)
            den = 1.0 + k * speed * hinv
            rden = 1.0 / den
            qxs, qys = qxs * rden, qys * rden
        qxs = np.where(W, qxs, 0.0)
        qys = np.where(W, qys, 0.0)
        return hs, qxs, qys

    def _lambda(self, X, Y):
        ny, nx, g, T = self.ny, self.nx, self.g, self.T
        al = np.ones((ny, nx), dtype=bool)
        xs, ys = slice(1, nx + 1), slice(1, ny + 1)
        T.c("abs", al, 4)
        T.c("mul", al, 4)
        T.c("sqrt", al, 4)
        T.c("add", al, 4)
        T.c("minmax", al, 2 + 2)
        a = np.fmax(np.abs(X.unm[:, xs]) + np.sqrt(g * X.hm[:, xs]), np.abs(X.unp[:, xs]) + np.sqrt(g * X.hp[:, xs]))
        b = np.fmax(np.abs(Y.unm[ys, :]) + np.sqrt(g * Y.hm[ys, :]), np.abs(Y.unp[ys, :]) + np.sqrt(g * Y.hp[ys, :]))
        return max(0.0, float(a.max())), max(0.0, float(b.max()))

    def step(self) -> float:
        """One step with the CFL dt (Eq. (cfl), the sum form); returns dt."""
        ny, nx, T = self.ny, self.nx, self.T
        J, I = slice(2, ny + 2), slice(2, nx + 2)
        h0, qx0, qy0 = self.h, self.qx, self.qy
        _ghosts(h0, self.bc, 1.0, 1.0)
        _ghosts(qx0, self.bc, -1.0, 1.0)
        _ghosts(qy0, self.bc, 1.0, -1.0)
        u, v = self._velocities(h0, qx0, qy0)
        rec = self._recon(h0, u, v) if self.order == 2 else self._recon1(h0, u, v)
        lx, ly = self._lambda(*rec)
        den = lx / self.dx + ly / self.dy
        dt = self.cfl / den if den > 0.0 else self.dt_max
        dt = min(dt, self.dt_max)
        # stage 1 works from the same velocities and reconstruction of U^n
        h1, qx1, qy1 = self._stage(h0, qx0, qy0, dt, (u, v) + rec)
        al = np.ones((ny, nx), dtype=bool)
        if self.order == 1:
            hn, qxn, qyn = h1, qx1, qy1                # one Euler stage
        else:
            p1 = [_pad(a) for a in (h1, qx1, qy1)]
            _ghosts(p1[0], self.bc, 1.0, 1.0)
            _ghosts(p1[1], self.bc, -1.0, 1.0)
            _ghosts(p1[2], self.bc, 1.0, -1.0)
            h2, qx2, qy2 = self._stage(*p1, dt)
            T.c("add", al, 3)
            T.c("mul", al, 3)
            hn = 0.5 * (h0[J, I] + h2)
            qxn = 0.5 * (qx0[J, I] + qx2)
            qyn = 0.5 * (qy0[J, I] + qy2)
        if self.rain > 0.0:
            T.c("add", al)
            hn = hn + dt * self.rain
        if self.infiltration:
            # Sec. 3.5: capacity K_s (1 + (psi + h) dtheta / V_inf), all the
            # water while V_inf = 0; then h, V_inf and the step's sum
            vi = self.vinf
            P = vi > 0.0
            T.c("cmp", al)
            T.c("add", P, 2)
            T.c("mul", P, 3)
            T.c("div", P)
            T.c("minmax", P)
            with np.errstate(divide="ignore", invalid="ignore"):
                ic = self.ks * (1.0 + ((self.psi + hn) * self.dtheta) / np.where(P, vi, 1.0))
            d = np.where(P, np.fmin(hn, dt * ic), hn)
            T.c("add", al, 3)
            hn = hn - d
            self.vinf = vi + d
        T.c("cmp", al)
        dry = hn <= self.hdry
        qxn = np.where(dry, 0.0, qxn)
        qyn = np.where(dry, 0.0, qyn)
        self.h, self.qx, self.qy = (_pad(a) for a in (hn, qxn, qyn))
        self.steps += 1
        return dt


def census(w, steps: int = 1, rain: bool | None = None, order: int = 2, cfl: float | None = None,
           vinf=None) -> tuple[Census, list[float]]:
    """Run `steps` counted steps of a workload (an object with nx, ny, dx,
    dy, z, h, qx, qy, bc, friction, manning_n, cfl, dt_max, h_dry,
    rain_rate, infiltration, ks, psi, dtheta); rain is taken as on for
    every step when rain_rate > 0; vinf = the infiltrated depth at the
    start (zero if None)."""
    c = Census(w.z, w.h, w.qx, w.qy, w.dx, w.dy, h_dry=w.h_dry, bc=w.bc, friction=w.friction,
               friction_coef=w.manning_n, cfl=cfl if cfl is not None else w.cfl, dt_max=w.dt_max,
               rain_rate=w.rain_rate if (rain is None or rain) else 0.0, order=order,
               infiltration=bool(w.infiltration), ks_map=w.ks, psi=w.psi, dtheta=w.dtheta, vinf=vinf)
    dts = [c.step() for _ in range(steps)]
    return c, dts


if __name__ == "__main__":
    import argparse
    import copy
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import swof_inputs as si

    ap = argparse.ArgumentParser(description="operation census of the scheme's step")
    ap.add_argument("--case", default="valley", choices=["valley", "hillslope"])
    ap.add_argument("--side", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--t0", type=float, default=300.0, help="hillslope: start the census at this time")
    a = ap.parse_args()
    print(f"# operation census of the scheme's step: {a.case} {a.side}^2, {a.steps} steps")
    print("# operations per cell-update (oracle form, each value computed once; see oracle/op_census.py)")
    print(f"# command: python -m oracle.op_census --case {a.case} --side {a.side} --steps {a.steps}"
          + (f" --t0 {a.t0:g}" if a.case == "hillslope" else ""))
    print("# flops = add + mul + div + sqrt + cbrt; all = every kind; wet = fraction of wet cells at the end")
    runs = []
    if a.case == "valley":
        w = si.valley(a.side)
        wet = copy.copy(w)
        wet.h = w.h + 0.5
        runs = [("valley", "valley from t = 0", w, 2, None, None),
                ("fully_wet", "valley + 0.5 m everywhere (fully wet)", wet, 2, None, None),
                ("valley_order1", "valley from t = 0, first order (n_CFL = 1)", w, 1, 1.0, None)]
    else:
        import oracle as orc
        w = si.hillslope(a.side)
        o = orc.Oracle.from_workload(w)
        o.run_to(a.t0)
        w = copy.copy(w)
        w.h, w.qx, w.qy = o.state()
        runs = [("hillslope", f"hillslope with rain and Green-Ampt from the oracle's state at t = {a.t0:g} s",
                 w, 2, None, o.vinf())]
    cells = w.nx * w.ny
    for key, name, wl, order, cfl, vinf in runs:
        c, dts = census(wl, a.steps, order=order, cfl=cfl, vinf=vinf)
        per = c.T.per(cells * a.steps)
        wetf = float(np.count_nonzero(c.state()[0] > wl.h_dry)) / cells
        print(f"# {name}: dt = " + ", ".join(f"{d:.6g}" for d in dts))
        print(f"{key}: " + " ".join(f"{k}={per[k]:.3f}" for k in KINDS + ("flops", "all")) + f" wet={wetf:.4f}")

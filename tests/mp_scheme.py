"""A second, independent statement of the scheme in 50-digit arithmetic.

Used only to pin the FP64 oracle's discrete algebra on tiny grids: every
operation here is done in mpmath at 50 significant digits (division, square
root and the 4/3 power are exact to that precision), so the oracle must agree
to within FP64 rounding.  The code is written cell-by-cell from the paper's
formulas (Sec. 3.1 scheme + hydrostatic reconstruction + S_L/S_R/Fc, Sec. 3.3
HLL, Sec. 3.4 MUSCL-minmod with modified velocities, Sec. 3.2 friction and
Heun, Sec. 3.5 Green-Ampt) and the same readings of the paper's silent points
as the oracle, without sharing any of its code.  It also takes the other
friction laws of Sec. 2.1 (C_f = 1/K^2, f/(8g), 1/C^2 with h^p, p = 4/3 or
1), the first-order step of Sec. 3.3 (face values = cell values, one Euler
stage) and the Riemann-invariant edges of Sec. 2.2, whose imposed-discharge
celerity comes from the exact roots of its cubic here.
"""
from __future__ import annotations

import mpmath as mp

mp.mp.dps = 50


def _minmod(a, b):
    if a >= 0 and b >= 0:
        return min(a, b)
    if a <= 0 and b <= 0:
        return max(a, b)
    return mp.mpf(0)


class MPScheme:
    def __init__(self, nx, ny, dx, dy, z, h, qx, qy, *, g=9.81, h_dry=1e-6,
                 bc=(0, 0, 0, 0), manning_n=0.0, rain_rate=0.0, ks=0.0,
                 psi=0.0, dtheta=0.0, infiltration=False, friction=None, friction_coef=None,
                 order=2, bc_h=(0.0,) * 4, bc_q=(0.0,) * 4):
        """friction: 1 Manning (n), 2 Strickler (K), 3 Darcy-Weisbach (f),
        4 Chezy (C), coefficient in friction_coef; by default Manning with
        manning_n.  bc: 0 wall, 1 outflow, 2 imposed depth (bc_h), 3
        imposed inflow discharge (bc_q), 4 both; sides W, E, S, N."""
        M = mp.mpf
        self.nx, self.ny = nx, ny
        self.dx, self.dy = M(dx), M(dy)
        self.g, self.h_dry = M(g), M(h_dry)
        self.bc = bc
        self.order = order
        self.bc_h = [M(v) for v in bc_h]
        self.bc_q = [M(v) for v in bc_q]
        law = 1 if friction is None else friction
        coef = M(manning_n if friction_coef is None else friction_coef)
        # C_f of the law and the power p of h in S_f = C_f |u| u / h^p
        if law == 1:
            self.n2, self.p = coef ** 2, M(4) / 3
        elif law == 2:
            self.n2, self.p = 1 / coef ** 2, M(4) / 3
        elif law == 3:
            self.n2, self.p = coef / (8 * self.g), M(1)
        elif law == 4:
            self.n2, self.p = 1 / coef ** 2, M(1)
        else:
            self.n2, self.p = M(0), M(4) / 3
        self.R = M(rain_rate)
        self.ks, self.psi, self.dtheta = M(ks), M(psi), M(dtheta)
        self.infiltration = infiltration
        self.z = [[M(float(z[j][i])) for i in range(nx)] for j in range(ny)]
        self.h = [[M(float(h[j][i])) for i in range(nx)] for j in range(ny)]
        self.qx = [[M(float(qx[j][i])) for i in range(nx)] for j in range(ny)]
        self.qy = [[M(float(qy[j][i])) for i in range(nx)] for j in range(ny)]
        self.vinf = [[M(0) for _ in range(nx)] for _ in range(ny)]

    # --- ghost values: map an out-of-range index onto the interior -------
    def _imposed(self, side, h1, qn1, qt1):
        """Boundary state (h, inward normal discharge, tangential discharge)
        of an imposed edge from its edge cell (Sec. 2.2): the outgoing
        invariant R = w1 - 2 sqrt(g h1) is kept, the imposed variable
        replaces the incoming one."""
        g, typ = self.g, self.bc[side]
        w1 = qn1 / h1 if h1 > self.h_dry else mp.mpf(0)
        t1 = qt1 / h1 if h1 > self.h_dry else mp.mpf(0)
        R = w1 - 2 * mp.sqrt(g * h1)
        hb, qb = self.bc_h[side], self.bc_q[side]
        if typ == 4:
            return hb, qb, mp.mpf(0)
        if typ == 2:
            w = R + 2 * mp.sqrt(g * hb)
            return hb, hb * w, hb * t1
        # q imposed: c = sqrt(g h) with q g / c^2 - 2c = R, the positive
        # root of 2 c^3 + R c^2 - q g (q = 0: c = max(-R/2, 0))
        Q = qb * g
        if Q > 0:
            roots = mp.polyroots([2, R, 0, -Q], maxsteps=200, extraprec=200)
            c = max(mp.re(r) for r in roots if abs(mp.im(r)) < mp.mpf(10) ** -30 and mp.re(r) > 0)
        else:
            c = max(-R / 2, mp.mpf(0))
        hh = c * c / g
        return hh, qb, hh * t1

    def _cell(self, arrs, i, j):
        """(h, qx, qy, z) at (i, j), ghosts from the boundary conditions."""
        h, qx, qy = arrs
        # imposed edges: both ghost layers hold the edge cell's boundary
        # state; the bed extends the edge cell
        for side, out, ei, ej, sgn, normal_x in ((0, i < 0, 0, j, 1, True),
                                                  (1, i >= self.nx, self.nx - 1, j, -1, True),
                                                  (2, j < 0, i, 0, 1, False),
                                                  (3, j >= self.ny, i, self.ny - 1, -1, False)):
            if out and self.bc[side] >= 2:
                h1, qx1, qy1 = h[ej][ei], qx[ej][ei], qy[ej][ei]
                qn1, qt1 = (sgn * qx1, qy1) if normal_x else (sgn * qy1, qx1)
                b = self._imposed(side, h1, qn1, qt1)
                if normal_x:
                    return b[0], sgn * b[1], b[2], self.z[ej][ei]
                return b[0], b[2], sgn * b[1], self.z[ej][ei]
        sx = sy = 1
        if i < 0:
            if self.bc[0] == 0:
                i, sx = -1 - i, -1
            else:
                i = 0
        elif i >= self.nx:
            if self.bc[1] == 0:
                i, sx = 2 * self.nx - 1 - i, -1
            else:
                i = self.nx - 1
        if j < 0:
            if self.bc[2] == 0:
                j, sy = -1 - j, -1
            else:
                j = 0
        elif j >= self.ny:
            if self.bc[3] == 0:
                j, sy = 2 * self.ny - 1 - j, -1
            else:
                j = self.ny - 1
        return h[j][i], sx * qx[j][i], sy * qy[j][i], self.z[j][i]

    def _vel(self, h, q):
        return q / h if h > self.h_dry else mp.mpf(0)

    def _recon(self, arrs, i, j, axis):
        """MUSCL values of cell (i, j) along axis: (h-,h+,z-,z+,un-,un+,ut-,ut+);
        at first order the cell values themselves."""
        di, dj = (1, 0) if axis == 0 else (0, 1)
        if self.order == 1:
            c = self._cell(arrs, i, j)
            un = self._vel(c[0], c[1 + axis])
            ut = self._vel(c[0], c[2 - axis])
            return c[0], c[0], c[3], c[3], un, un, ut, ut
        cells = [self._cell(arrs, i + k * di, j + k * dj) for k in (-1, 0, 1)]
        hs = [c[0] for c in cells]
        es = [c[0] + c[3] for c in cells]
        un = [self._vel(c[0], c[1 + axis]) for c in cells]
        ut = [self._vel(c[0], c[2 - axis]) for c in cells]
        Dh = _minmod(hs[1] - hs[0], hs[2] - hs[1])
        De = _minmod(es[1] - es[0], es[2] - es[1])
        hm, hp = hs[1] - Dh / 2, hs[1] + Dh / 2
        em, ep = es[1] - De / 2, es[1] + De / 2
        if hs[1] > self.h_dry:
            Dn = _minmod(un[1] - un[0], un[2] - un[1])
            Dt = _minmod(ut[1] - ut[0], ut[2] - ut[1])
            unm = un[1] - hp / hs[1] * Dn / 2
            unp = un[1] + hm / hs[1] * Dn / 2
            utm = ut[1] - hp / hs[1] * Dt / 2
            utp = ut[1] + hm / hs[1] * Dt / 2
        else:
            unm = unp = un[1]
            utm = utp = ut[1]
        return hm, hp, em - hm, ep - hp, unm, unp, utm, utp

    def _hll(self, hL, unL, utL, hR, unR, utR):
        g = self.g
        c1 = min(unL - mp.sqrt(g * hL), unR - mp.sqrt(g * hR))
        c2 = max(unL + mp.sqrt(g * hL), unR + mp.sqrt(g * hR))
        FL = (hL * unL, hL * unL * unL + g * hL * hL / 2, hL * unL * utL)
        FR = (hR * unR, hR * unR * unR + g * hR * hR / 2, hR * unR * utR)
        UL = (hL, hL * unL, hL * utL)
        UR = (hR, hR * unR, hR * utR)
        if c1 >= 0:
            return FL
        if c2 <= 0:
            return FR
        return tuple((c2 * FL[k] - c1 * FR[k]) / (c2 - c1)
                     + c1 * c2 / (c2 - c1) * (UR[k] - UL[k]) for k in range(3))

    def _face(self, arrs, i, j, axis):
        """Fluxes at the plus face of (i, j): (F1, F2 with S_L, F2 with S_R, F3)."""
        di, dj = (1, 0) if axis == 0 else (0, 1)
        a = self._recon(arrs, i, j, axis)
        b = self._recon(arrs, i + di, j + dj, axis)
        zmax = max(a[3], b[2])
        hL = max(mp.mpf(0), a[1] + a[3] - zmax)
        hR = max(mp.mpf(0), b[0] + b[2] - zmax)
        F = self._hll(hL, a[5], a[7], hR, b[4], b[6])
        g = self.g
        return (F[0], F[1] + g * (a[1] ** 2 - hL ** 2) / 2,
                F[1] + g * (b[0] ** 2 - hR ** 2) / 2, F[2])

    def lam(self):
        lx = ly = mp.mpf(0)
        arrs = (self.h, self.qx, self.qy)
        for j in range(self.ny):
            for i in range(self.nx):
                a = self._recon(arrs, i, j, 0)
                b = self._recon(arrs, i, j, 1)
                lx = max(lx, abs(a[4]) + mp.sqrt(self.g * a[0]), abs(a[5]) + mp.sqrt(self.g * a[1]))
                ly = max(ly, abs(b[4]) + mp.sqrt(self.g * b[0]), abs(b[5]) + mp.sqrt(self.g * b[1]))
        # an imposed edge's boundary state feeds the edge fluxes, so the
        # face value of the ghost cell facing the domain counts too
        for j in range(self.ny):
            if self.bc[0] >= 2:
                a = self._recon(arrs, -1, j, 0)
                lx = max(lx, abs(a[5]) + mp.sqrt(self.g * a[1]))
            if self.bc[1] >= 2:
                a = self._recon(arrs, self.nx, j, 0)
                lx = max(lx, abs(a[4]) + mp.sqrt(self.g * a[0]))
        for i in range(self.nx):
            if self.bc[2] >= 2:
                b = self._recon(arrs, i, -1, 1)
                ly = max(ly, abs(b[5]) + mp.sqrt(self.g * b[1]))
            if self.bc[3] >= 2:
                b = self._recon(arrs, i, self.ny, 1)
                ly = max(ly, abs(b[4]) + mp.sqrt(self.g * b[0]))
        return lx, ly

    def _stage(self, arrs, dt):
        g = self.g
        h, qx, qy = arrs
        out_h = [[None] * self.nx for _ in range(self.ny)]
        out_x = [[None] * self.nx for _ in range(self.ny)]
        out_y = [[None] * self.nx for _ in range(self.ny)]
        for j in range(self.ny):
            for i in range(self.nx):
                E = self._face(arrs, i, j, 0)
                W = self._face(arrs, i - 1, j, 0)
                N = self._face(arrs, i, j, 1)
                S = self._face(arrs, i, j - 1, 1)
                rx = self._recon(arrs, i, j, 0)
                ry = self._recon(arrs, i, j, 1)
                Fcx = -g * (rx[0] + rx[1]) / 2 * (rx[3] - rx[2])
                Fcy = -g * (ry[0] + ry[1]) / 2 * (ry[3] - ry[2])
                hs = h[j][i] - dt / self.dx * (E[0] - W[0]) - dt / self.dy * (N[0] - S[0])
                qxs = (qx[j][i] - dt / self.dx * (E[1] - W[2] - Fcx)
                       - dt / self.dy * (N[3] - S[3]))
                qys = (qy[j][i] - dt / self.dx * (E[3] - W[3])
                       - dt / self.dy * (N[1] - S[2] - Fcy))
                if hs > self.h_dry:
                    u = self._vel(h[j][i], qx[j][i])
                    v = self._vel(h[j][i], qy[j][i])
                    den = 1 + dt * g * self.n2 * mp.sqrt(u * u + v * v) / hs ** self.p
                    qxs, qys = qxs / den, qys / den
                else:
                    qxs = qys = mp.mpf(0)
                out_h[j][i], out_x[j][i], out_y[j][i] = hs, qxs, qys
        return out_h, out_x, out_y

    def step(self, dt):
        dt = mp.mpf(dt)
        U0 = (self.h, self.qx, self.qy)
        U1 = self._stage(U0, dt)
        U2 = self._stage(U1, dt) if self.order == 2 else None
        for j in range(self.ny):
            for i in range(self.nx):
                if self.order == 1:                     # one Euler stage
                    h, qx, qy = U1[0][j][i], U1[1][j][i], U1[2][j][i]
                else:
                    h = (U0[0][j][i] + U2[0][j][i]) / 2
                    qx = (U0[1][j][i] + U2[1][j][i]) / 2
                    qy = (U0[2][j][i] + U2[2][j][i]) / 2
                h = h + dt * self.R
                if self.infiltration:
                    V = self.vinf[j][i]
                    if V > 0:
                        ic = self.ks * (1 + (self.psi + h) / (V / self.dtheta))
                        d = min(h, dt * ic)
                    else:
                        d = h
                    h -= d
                    self.vinf[j][i] = V + d
                if h <= self.h_dry:
                    qx = qy = mp.mpf(0)
                self.h[j][i], self.qx[j][i], self.qy[j][i] = h, qx, qy

    def state(self):
        import numpy as np
        return tuple(np.array([[float(a[j][i]) for i in range(self.nx)]
                               for j in range(self.ny)]) for a in (self.h, self.qx, self.qy))

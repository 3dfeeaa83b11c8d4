"""Closed-form dam-break solutions of the 1-D shallow water equations.

The paper validates FullSWOF against SWASHES analytic solutions (Sec. 4.1);
these are the two textbook dam-break Riemann problems, restated from first
principles (characteristics of Eq. (SW1DH) with eigenvalues u -+ sqrt(g h),
Sec. 2.2, and the Rankine-Hugoniot conditions):

  * Ritter (dry bed, h_r = 0): a centred rarefaction from x0 - c_l t to
    x0 + 2 c_l t, inside which u + 2c = 2 c_l and c - u = ... so that
    h = (2 c_l - xi)^2 / (9 g), u = 2 (xi + c_l) / 3, xi = (x - x0)/t.
  * Stoker (wet bed, 0 < h_r < h_l): the same left rarefaction down to an
    intermediate state (h_m, u_m) with u_m + 2 sqrt(g h_m) = 2 c_l, joined to
    the still right state by a shock: u_m = (h_m - h_r) sqrt(g (h_m + h_r) /
    (2 h_m h_r)), moving at s = h_m u_m / (h_m - h_r).
"""
from __future__ import annotations

import math

import numpy as np


def stoker_state(h_l: float, h_r: float, g: float = 9.81):
    """Intermediate depth/velocity and shock speed (bisection on h_m)."""
    c_l = math.sqrt(g * h_l)

    def f(hm):
        u_raref = 2.0 * (c_l - math.sqrt(g * hm))
        u_shock = (hm - h_r) * math.sqrt(g * (hm + h_r) / (2.0 * hm * h_r))
        return u_raref - u_shock

    lo, hi = h_r, h_l
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    hm = 0.5 * (lo + hi)
    um = 2.0 * (c_l - math.sqrt(g * hm))
    s = hm * um / (hm - h_r)
    return hm, um, s


def dam_break_profile(x: np.ndarray, t: float, x0: float, h_l: float,
                      h_r: float, g: float = 9.81):
    """(h, u) at positions x and time t > 0 for the dam break at x0."""
    c_l = math.sqrt(g * h_l)
    xi = (np.asarray(x, dtype=np.float64) - x0) / t
    h = np.empty_like(xi)
    u = np.zeros_like(xi)
    raref_h = (2.0 * c_l - xi) ** 2 / (9.0 * g)
    raref_u = 2.0 * (xi + c_l) / 3.0
    if h_r == 0.0:
        left = xi <= -c_l
        fan = (xi > -c_l) & (xi < 2.0 * c_l)
        h[left] = h_l
        h[fan] = raref_h[fan]
        u[fan] = raref_u[fan]
        h[xi >= 2.0 * c_l] = 0.0
        return h, u
    hm, um, s = stoker_state(h_l, h_r, g)
    cm = math.sqrt(g * hm)
    left = xi <= -c_l
    fan = (xi > -c_l) & (xi <= um - cm)
    mid = (xi > um - cm) & (xi < s)
    right = xi >= s
    h[left] = h_l
    h[fan] = raref_h[fan]
    u[fan] = raref_u[fan]
    h[mid] = hm
    u[mid] = um
    h[right] = h_r
    return h, u

"""Pins of the oracle's scalar building blocks against hand values and the
mathematics (no GPU).  Paper: Sec. 3.4 (minmod), Sec. 3.1 (hydrostatic
reconstruction), Sec. 3.3 (HLL), Sec. 2.1 (Manning h^{4/3})."""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle

G = 9.81


def test_minmod_branches():
    mm = oracle.minmod
    assert mm(1.0, 2.0) == 1.0          # both positive: min
    assert mm(3.0, 0.5) == 0.5
    assert mm(-1.0, -2.0) == -1.0       # both negative: max
    assert mm(-3.0, -0.25) == -0.25
    assert mm(1.0, -1.0) == 0.0         # opposite signs: 0
    assert mm(-2.0, 5.0) == 0.0
    assert mm(0.0, 5.0) == 0.0          # a zero slope wins
    assert mm(-5.0, 0.0) == 0.0


def _F(h, un, ut):
    q = h * un
    return np.array([q, q * un + 0.5 * G * h * h, q * ut])


@pytest.mark.parametrize("h,un,ut", [(1.0, 0.3, -0.2), (0.5, -1.1, 0.7), (2.0, 0.0, 0.0),
                                     (1e-3, 0.01, 0.02)])
def test_hll_consistency(h, un, ut):
    """F(U, U) = F(U) for the HLL flux (consistency), subsonic states."""
    F = oracle.hll(G, h, un, ut, h, un, ut)
    np.testing.assert_allclose(F, _F(h, un, ut), rtol=2e-15, atol=1e-300)


def test_hll_supersonic_branches():
    # 0 <= c1: everything moves right -> F(U_L) exactly
    hL, uL, hR, uR = 0.2, 5.0, 0.1, 6.0
    F = oracle.hll(G, hL, uL, 0.3, hR, uR, -0.4)
    assert np.array_equal(F, _F(hL, uL, 0.3))
    # c2 <= 0: everything moves left -> F(U_R) exactly
    F = oracle.hll(G, 0.2, -6.0, 0.1, 0.1, -5.0, 0.2)
    assert np.array_equal(F, _F(0.1, -5.0, 0.2))


def test_hll_middle_branch_hand_value():
    """Middle branch against the formula evaluated in 40-digit arithmetic."""
    mp.mp.dps = 40
    hL, uL, tL, hR, uR, tR = 1.0, 0.5, 0.25, 0.4, -0.3, 0.1
    g = mp.mpf(G)
    cL, cR = mp.sqrt(g * hL), mp.sqrt(g * mp.mpf(hR))
    c1 = min(uL - cL, mp.mpf(uR) - cR)
    c2 = max(uL + cL, mp.mpf(uR) + cR)
    hLm, uLm, tLm, hRm, uRm, tRm = map(mp.mpf, (hL, uL, tL, hR, uR, tR))
    FL = [hLm * uLm, hLm * uLm ** 2 + g * hLm ** 2 / 2, hLm * uLm * tLm]
    FR = [hRm * uRm, hRm * uRm ** 2 + g * hRm ** 2 / 2, hRm * uRm * tRm]
    UL = [hLm, hLm * uLm, hLm * tLm]
    UR = [hRm, hRm * uRm, hRm * tRm]
    exp = [(c2 * FL[k] - c1 * FR[k]) / (c2 - c1) + c1 * c2 / (c2 - c1) * (UR[k] - UL[k])
           for k in range(3)]
    F = oracle.hll(G, hL, uL, tL, hR, uR, tR)
    np.testing.assert_allclose(F, [float(e) for e in exp], rtol=1e-14)


def test_hll_dry_faces_give_zero_flux():
    assert np.array_equal(oracle.hll(G, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0), np.zeros(3))
    # a dry face state with a nonzero reconstructed velocity still carries nothing
    F = oracle.hll(G, 0.0, 0.7, 0.1, 0.0, -0.2, 0.3)
    assert np.array_equal(np.abs(F), np.zeros(3))


def test_hll_mirror_wall_has_zero_mass_flux():
    """Mirrored states (h, u) | (h, -u) as produced by a wall ghost: the mass
    flux is exactly zero and the momentum flux is the wall pressure."""
    for h, u in [(1.0, 0.3), (0.37, -2.1), (2.5, 0.0), (1e-4, 1.7)]:
        F = oracle.hll(G, h, u, 0.2, h, -u, 0.2)
        assert F[0] == 0.0


def test_icbrt_against_library_cbrt():
    rng = np.random.default_rng(0)
    xs = np.concatenate([10.0 ** rng.uniform(-8, 4, 20000),
                         [1e-6, 1.0, 8.0, 27.0, 0.125, 2.0, 4.0, 1e-300 * 1e290, 7.999999999999999]])
    worst = 0.0
    for x in xs:
        y = oracle.icbrt(float(x))
        ref = 1.0 / np.cbrt(x)
        worst = max(worst, abs(y - ref) / ref)
    assert worst < 4 * 2.0 ** -52, worst


def test_icbrt_exact_cubes():
    for k in range(-20, 21):
        x = 2.0 ** (3 * k)
        assert abs(oracle.icbrt(x) - 2.0 ** (-k)) <= 2 * 2.0 ** -52 * 2.0 ** (-k)


def test_manning_power_matches_h_4_3():
    for h in [1e-5, 0.01, 0.3, 1.0, 7.5, 40.0, 600.0]:
        y = oracle.icbrt(h)
        ref = float(mp.mpf(h) ** (mp.mpf(-4) / 3))
        assert math.isclose((y * y) * (y * y), ref, rel_tol=2e-15)

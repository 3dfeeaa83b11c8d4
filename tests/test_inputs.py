"""The seeded input generators against the recipes they state (CPU only).

Every workload the tests and the benchmark use comes from swof_inputs; these
checks pin each one to its written recipe -- the formula of the bed, the
initial water, the forcing and parameters, the boundary codes -- so that a
slip in a generator cannot pass for a property of the scheme.
"""
import numpy as np
import pytest

import swof_inputs as si


def centres(n, dx):
    return (np.arange(n) + 0.5) * dx


def test_generators_are_deterministic_in_their_seeds():
    a, b, c = si.valley(128), si.valley(128), si.valley(128, seed=2)
    assert np.array_equal(a.z, b.z) and np.array_equal(a.h, b.h)
    assert not np.array_equal(a.z, c.z)
    h1, h2 = si.hillslope(64), si.hillslope(64)
    assert np.array_equal(h1.z, h2.z) and np.array_equal(h1.ks, h2.ks)
    assert np.array_equal(si.dem(96, 80, 3, 0.01, 0.1), si.dem(96, 80, 3, 0.01, 0.1))


def test_fractal_noise_peak_mean_and_spectral_slope():
    """max |noise| = peak, no mean (DC removed), and a radially averaged
    power spectrum falling as k^-(2H+2)."""
    H, n = 0.8, 256
    f = si.fractal_noise(n, n, H, 5, 1.5)
    assert np.max(np.abs(f)) == pytest.approx(1.5, rel=1e-12)
    assert abs(f.mean()) < 1e-12 * n * n
    p = np.abs(np.fft.fft2(f)) ** 2
    k = np.sqrt(np.fft.fftfreq(n)[None, :] ** 2 + np.fft.fftfreq(n)[:, None] ** 2)
    bins = np.logspace(np.log10(2.0 / n), np.log10(0.4), 16)
    idx = np.digitize(k.ravel(), bins)
    kk, pp = [], []
    for b in range(1, len(bins)):
        sel = idx == b
        if sel.sum() > 8:
            kk.append(k.ravel()[sel].mean())
            pp.append(p.ravel()[sel].mean())
    slope = np.polyfit(np.log(kk), np.log(pp), 1)[0]
    assert slope == pytest.approx(-(2 * H + 2), abs=0.3)


def test_valley_bed_pool_and_parameters():
    """z = 0.15 |x - x_c| + 0.003 (L_y - y) + fractal noise (H = 0.8, seed,
    peak 1.5); a level pool up to the noise-free thalweg elevation of the
    last reservoir row + 40 m behind row n/8, dry downstream; at rest;
    Manning 0.033; outflow at j = ny - 1, walls elsewhere."""
    n, dx = 256, 2.0
    w = si.valley(n)
    x, y = centres(n, dx), centres(n, dx)
    L = n * dx
    base = 0.15 * np.abs(x[None, :] - 0.5 * L) + 0.003 * (L - y[:, None])
    assert np.allclose(w.z - base, si.fractal_noise(n, n, 0.8, 1, 1.5), rtol=0, atol=1e-12)
    dam = n // 8
    eta = 0.003 * (L - y[dam - 1]) + 40.0
    assert np.array_equal(w.h[:dam], np.maximum(0.0, eta - w.z[:dam]))
    assert not np.any(w.h[dam:])
    wet = w.h[:dam] > 0
    assert np.allclose(w.h[:dam][wet] + w.z[:dam][wet], eta, rtol=0, atol=1e-9)
    assert not np.any(w.qx) and not np.any(w.qy)
    assert w.bc == (si.BC_WALL, si.BC_WALL, si.BC_WALL, si.BC_OUTFLOW)
    assert w.friction == 1 and w.manning_n == 0.033 and w.dx == w.dy == 2.0
    assert w.h_dry == 1e-6 and w.rain_rate == 0.0
    lit = si.valley(n, literal_pool=True)
    assert np.all(lit.h[:dam] == 40.0) and not np.any(lit.h[dam:])


def test_valley_4096_dam_row_and_confined_pool():
    """At 4096^2 the dam is at row 512 and the pool (40 m over the thalweg)
    stops on the valley walls, which rise 0.15 m per metre to ~614 m."""
    w = si.valley(4096)
    assert w.extra["dam_row"] == 512
    assert np.any(w.h[511]) and not np.any(w.h[512:])
    assert 0 < np.count_nonzero(w.h[:512]) < 512 * 4096 // 4


def test_hillslope_bed_soil_and_forcing():
    """z = 0.05 (L_y - y) + 0.1 sin(2 pi x / 0.75) + 0.02 N(0, 1), the
    sinusoid sampled at cell centres (x = i + 1/2 m: it equals
    -0.1 sin(2 pi x / 3), the 3 m alias); K_s lognormal, median 1e-6 m/s,
    sigma 0.5; rain 50 mm/h for 600 s; Green-Ampt psi 0.1 m, dtheta 0.3;
    Manning 0.05; dry start; outflow downslope; dt_max 1 s, t_end 1200 s."""
    n = 256
    w = si.hillslope(n)
    x, y = centres(n, 1.0), centres(n, 1.0)
    furrow = 0.1 * np.sin(2 * np.pi * x / 0.75)
    assert np.allclose(furrow, -0.1 * np.sin(2 * np.pi * x / 3.0), atol=1e-12)
    r = (w.z - 0.05 * (n - y[:, None]) - furrow[None, :]) / 0.02
    assert abs(r.mean()) < 0.02 and r.std() == pytest.approx(1.0, rel=0.02)
    xi = np.log(w.ks / 1e-6) / 0.5
    assert abs(xi.mean()) < 0.02 and xi.std() == pytest.approx(1.0, rel=0.02)
    assert np.median(w.ks) == pytest.approx(1e-6, rel=0.03)
    assert w.rain_rate == pytest.approx(50e-3 / 3600) and w.rain_t_on == 0.0 and w.rain_t_off == 600.0
    assert w.infiltration == 1 and w.psi == 0.1 and w.dtheta == 0.3
    assert w.friction == 1 and w.manning_n == 0.05
    assert not np.any(w.h) and not np.any(w.qx) and not np.any(w.qy)
    assert w.bc == (si.BC_WALL, si.BC_WALL, si.BC_WALL, si.BC_OUTFLOW)
    assert w.dt_max == 1.0 and w.t_end == 1200.0


@pytest.mark.parametrize("axis", ["x", "y"])
def test_dam_break_layout(axis):
    """200^2, dx = 0.05 m, flat bed, h = 1 m left of x = 5 m and 0.5 m
    right of it, at rest, walls, t_end = 1 s; axis y is the transpose."""
    w = si.dam_break(200, axis=axis)
    prof = np.where(np.arange(200) < 100, 1.0, 0.5)
    expect = np.tile(prof, (200, 1))
    assert np.array_equal(w.h, expect if axis == "x" else expect.T)
    assert not np.any(w.z) and not np.any(w.qx) and not np.any(w.qy)
    assert w.bc == (0, 0, 0, 0) and w.dx == 0.05 and w.t_end == 1.0 and w.friction == 0


def test_lake_at_rest_level_and_emerged_bumps():
    w = si.lake_at_rest(64, level=1.0)
    wet = w.h > 0
    assert np.allclose((w.h + w.z)[wet], 1.0, rtol=0, atol=1e-15)
    assert np.all(w.z[~wet] >= 1.0)
    assert np.count_nonzero(~wet) > 0 and np.count_nonzero(wet) > 0
    assert not np.any(w.qx) and not np.any(w.qy)


def test_ensemble_specs_ranges_and_members():
    """256 scenarios from seed 4: sides uniform over {128, ..., 1024},
    reservoir U(5, 40) m, Manning U(0.02, 0.06), rain U(0, 80) mm/h; a
    member is a valley of its side with the dam at row side/8 and its
    parameters."""
    specs = si.ensemble_specs()
    assert len(specs) == 256
    sides = np.array([s.side for s in specs])
    assert set(sides) <= set(si.ENSEMBLE_SIDES) and len(set(sides)) == len(si.ENSEMBLE_SIDES)
    for s in specs:
        assert 5.0 <= s.reservoir <= 40.0 and 0.02 <= s.manning_n <= 0.06 and 0.0 <= s.rain_mm_h <= 80.0
    # mean member size near the mean of the six sides squared
    assert np.mean(sides.astype(float) ** 2) == pytest.approx(np.mean(np.array(si.ENSEMBLE_SIDES) ** 2.0),
                                                               rel=0.15)
    m = si.ensemble_member(specs[3])
    assert m.nx == m.ny == specs[3].side and m.extra["dam_row"] == max(1, specs[3].side // 8)
    assert m.manning_n == specs[3].manning_n and m.rain_rate == pytest.approx(specs[3].rain_mm_h * si.RAIN_MM_PER_H)
    assert m.extra["reservoir"] == specs[3].reservoir and m.infiltration == 0


def test_dem_tilt_noise_quantum_and_holes():
    """float32: 0.002 (x + 2y) tilt in cell units + the fractal noise of
    the seed (peak 1.5); quantised to multiples of the quantum; holes at
    the no-data value in about the requested fraction of cells; beyond 4096
    cells the 4096-periodic noise repeats."""
    nx, ny = 300, 200
    z = si.dem(nx, ny, 9)
    assert z.dtype == np.float32 and z.shape == (ny, nx)
    tilt = (np.float32(0.002) * np.arange(nx, dtype=np.float32))[None, :] + \
        (np.float32(0.004) * np.arange(ny, dtype=np.float32))[:, None]
    noise = si.fractal_noise(nx, ny, 0.8, 9, 1.5).astype(np.float32)
    assert np.allclose(z, noise + tilt, rtol=0, atol=1e-6)
    q = si.dem(nx, ny, 9, quantum=0.05)
    assert np.allclose(q / np.float32(0.05), np.round(q / np.float32(0.05)), atol=1e-3)
    holes = si.dem(nx, ny, 9, nodata_frac=0.1, nodata=-9999.0) == np.float32(-9999.0)
    assert holes.mean() == pytest.approx(0.1, abs=0.01)
    big = si.dem(4096 + 64, 8, 9)
    assert np.allclose(big[:, 4096:] - big[:, :64], 0.002 * 4096, rtol=0, atol=2e-3)

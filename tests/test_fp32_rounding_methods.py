"""The two numerical methods of the FP32 stage kernels, restated in numpy
and checked against exact arithmetic (the device code itself is covered by
the FP32 accuracy tests on the GPU):

- the depth update a + b rounded stochastically: TwoSum gives the rounding
  error exactly, and choosing the neighbouring float on the error's side
  with probability |error| / spacing (random bits from the "lowbias32"
  integer hash of a cell index and a time key) is unbiased: the mean of the
  rounded results over many draws equals a + b, while rounding to nearest
  keeps a constant bias;
- the reciprocal from an approximation with relative error up to 2^-22
  refined by one Newton-Raphson step r + r (1 - a r): within one float32 ulp
  of 1 / a.
"""
import numpy as np

F = np.float32


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    e = F(F(a - F(s - bb)) + F(b - bb))
    return s, e


def lowbias32(x):
    x = np.uint32(x)
    x ^= x >> np.uint32(16)
    x = np.uint32((int(x) * 0x7FEB352D) & 0xFFFFFFFF)
    x ^= x >> np.uint32(15)
    x = np.uint32((int(x) * 0x846CA68B) & 0xFFFFFFFF)
    x ^= x >> np.uint32(16)
    return x


def sr_add(a, b, cell, ts):
    s, e = two_sum(F(a), F(b))
    if not s > 0 or e == 0:
        return s
    sb = s.view(np.uint32)
    nb = (sb + np.uint32(1) if e > 0 else sb - np.uint32(1)).view(F)
    gap = abs(float(nb) - float(s))
    u = int(lowbias32(np.uint32(cell) ^ ts))
    return nb if (u >> 8) * 2.0 ** -24 * gap < abs(float(e)) else s


def test_two_sum_error_is_exact():
    rng = np.random.default_rng(1)
    a = (rng.uniform(0, 64, 20000)).astype(F)
    b = (rng.standard_normal(20000) * 1e-5).astype(F)
    for x, y in zip(a, b):
        s, e = two_sum(x, y)
        # float32 values are exact in float64, and so is their exact sum here
        assert float(s) + float(e) == float(x) + float(y)


def test_stochastic_rounding_is_unbiased_where_nearest_is_not():
    # a deep cell (h = 40 m, ulp 3.8e-6) receiving 0.3 ulp per step: rounded to
    # nearest the increment is lost every step; rounded stochastically the
    # depth follows the exact sum on average
    a0, inc, steps, cells = F(40.0), F(0.3 * 2.0 ** -18), 400, 64
    exact = float(a0) + steps * float(inc)
    nearest = a0
    for _ in range(steps):
        nearest = F(nearest + inc)
    assert float(nearest) == float(a0)                      # the bias: nothing added
    finals = []
    for c in range(cells):
        h = a0
        for k in range(steps):
            t = np.float64(k * 0.05).view(np.uint64)
            ts = lowbias32(np.uint32(int(t) & 0xFFFFFFFF) ^ lowbias32(np.uint32((int(t) >> 32) + 0x9E3779B9)))
            h = sr_add(h, inc, 1000 + c, ts)
        finals.append(float(h))
    mean = np.mean(finals)
    ulp = 2.0 ** -18
    # the mean over the cells sits within a few standard errors of the exact sum
    se = np.std(finals) / np.sqrt(cells) + 1e-30
    assert abs(mean - exact) <= 4 * se + 0.05 * ulp
    # each cell's error is a random walk of at most a few tens of ulps
    assert max(abs(f - exact) for f in finals) <= 30 * ulp


def test_one_newton_step_reciprocal_within_an_ulp():
    rng = np.random.default_rng(2)
    a = (10.0 ** rng.uniform(-6, 6, 100000)).astype(F)
    r0 = (1.0 / a.astype(np.float64) * (1.0 + rng.uniform(-1, 1, a.size) * 2.0 ** -22)).astype(F)
    # r + r (1 - a r) with fused multiply-adds: float64 products of float32
    # values are exact, so each fma is one float32 rounding
    e = (1.0 - a.astype(np.float64) * r0.astype(np.float64)).astype(F)
    r1 = (r0.astype(np.float64) * e.astype(np.float64) + r0.astype(np.float64)).astype(F)
    exact = 1.0 / a.astype(np.float64)
    ulp = np.spacing(exact.astype(F)).astype(np.float64)
    assert np.max(np.abs(r1.astype(np.float64) - exact) / ulp) <= 1.0

"""The surrogate's GELU uses erf by Abramowitz & Stegun formula 7.1.28,
1 - (1 + a1 x + ... + a6 x^6)^-16 (x >= 0, odd extension), with the
handbook's bound |error| <= 3e-7.  This checks the constants against
math.erf over the whole range the network sees, in FP64 and in FP32
arithmetic like the device's (whose result is then rounded to bf16)."""
import math

import numpy as np

A = [0.0705230784, 0.0422820123, 0.0092705272, 0.0001520143, 0.0002765672, 0.0000430638]


def erf_as(x, dtype):
    x = np.asarray(x, dtype=dtype)
    a = np.abs(x)
    p = dtype(A[5])
    for c in A[4::-1]:
        p = p * a + dtype(c)
    p = p * a + dtype(1)
    p = p ** 16
    with np.errstate(over="ignore"):
        r = dtype(1) / p
    return np.copysign(dtype(1) - r, x)


def test_formula_7_1_28_within_its_bound():
    x = np.linspace(-8.0, 8.0, 200001)
    ref = np.array([math.erf(v) for v in x])
    assert np.max(np.abs(erf_as(x, np.float64) - ref)) <= 3.0e-7
    # FP32 evaluation: the rounding of the polynomial is raised to the 16th
    # power, ~16 float32 ulps of 1 near x = 0
    assert np.max(np.abs(erf_as(x, np.float32).astype(np.float64) - ref)) <= 2.0e-6


def test_gelu_from_it_is_far_inside_bf16_resolution():
    z = np.linspace(-10.0, 10.0, 40001)
    exact = 0.5 * z * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in z]))
    approx = 0.5 * z * (1.0 + erf_as(z / math.sqrt(2.0), np.float64))
    assert np.max(np.abs(approx - exact) / np.maximum(np.abs(exact), 1.0)) <= 2.0e-6


def gelu_select(z, dtype):
    """The device's GELU form: r = (1 + a1 x + ... + a6 x^6)^-16 at x = |z| / sqrt 2,
    then z - z r / 2 for z >= 0 and z r / 2 for z < 0 (1 + erf = 2 - r or r)."""
    z = np.asarray(z, dtype=dtype)
    a = np.abs(z) * dtype(1.0 / math.sqrt(2.0))
    p = dtype(A[5])
    for c in A[4::-1]:
        p = p * a + dtype(c)
    p = p * a + dtype(1)
    with np.errstate(over="ignore"):
        r = dtype(1) / p ** 16
    h = (dtype(0.5) * z) * r
    return np.where(z >= 0, z - h, h)


def test_gelu_select_form_equals_the_erf_form_and_keeps_the_tail():
    z = np.linspace(-10.0, 10.0, 40001)
    exact = 0.5 * z * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in z]))
    via_erf = 0.5 * z * (1.0 + erf_as(z / math.sqrt(2.0), np.float64))
    sel = gelu_select(z, np.float64)
    assert np.max(np.abs(sel - via_erf)) <= 1e-14
    assert np.max(np.abs(sel - exact) / np.maximum(np.abs(exact), 1.0)) <= 2.0e-6
    # FP32 like the device: the formula's own error (A&S's absolute bound,
    # times |z| / 2) plus float32 rounding, far below a bf16 unit of values >= 1
    s32 = gelu_select(z, np.float32).astype(np.float64)
    assert np.max(np.abs(s32 - exact) / np.maximum(np.abs(exact), 1.0)) <= 1.0e-6

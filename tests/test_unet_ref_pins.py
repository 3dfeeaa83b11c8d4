"""Pins of the numpy U-Net reference (CPU, no GPU): its backward agrees with
central finite differences of its own forward in exact (non-bf16)
arithmetic, and the layer list matches the parameter count the paper-side
design states (~2M parameters at base width 32)."""
import numpy as np

from oracle.unet_ref import UNetRef, layers_spec


def test_parameter_count_base32_is_about_two_million():
    spec, n = layers_spec(32, 4, 3)
    logical = sum(d["ncols"] * (9 if d["kind"] == 0 else 1) * d["cin"] for d in spec) + sum(d["cout"] for d in spec)
    assert 1.9e6 < logical < 2.1e6
    assert len(spec) == 18


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    C, H = 16, 16
    spec, n = layers_spec(C, 4, 3)
    p = np.zeros(n)
    for d in spec:
        taps = 9 if d["kind"] == 0 else 1
        sd = np.sqrt(2.0 / (taps * d["cin"]))
        W = p[d["woff"]: d["woff"] + d["ncols"] * d["Kp"]].reshape(d["ncols"], d["Kp"])
        for t in range(taps):
            W[:, t * d["cin_p"]: t * d["cin_p"] + d["cin"]] = sd * rng.standard_normal((d["ncols"], d["cin"]))
        p[d["boff"]: d["boff"] + d["cout"]] = 0.1 * rng.standard_normal(d["cout"])
    x = np.zeros((1, H, H, 16))
    x[..., :4] = rng.standard_normal((1, H, H, 4))
    tgt = rng.standard_normal((1, H, H, 3))
    net = UNetRef(C, 4, 3, p, use_bf16=False)
    loss, g = net.loss_and_grads(x, tgt)
    # sample weights of every layer (logical entries) and biases
    idx = []
    for d in spec:
        idx.append(d["woff"] + int(rng.integers(0, d["ncols"])) * d["Kp"] + int(rng.integers(0, d["cin"])))
        idx.append(d["boff"] + int(rng.integers(0, d["cout"])))
    eps = 1e-5
    P = H * H
    for i in idx:
        pp = p.copy()
        pp[i] += eps
        lp = UNetRef(C, 4, 3, pp, use_bf16=False).loss_and_grads(x, tgt)[0]
        pp[i] -= 2 * eps
        lm = UNetRef(C, 4, 3, pp, use_bf16=False).loss_and_grads(x, tgt)[0]
        fd = (lp - lm) / (2 * eps) / (P * 3)      # the gradient is of the mean
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])

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


def _torch_unet_loss(p, spec, x, tgt, in_ch, out_ch):
    """The same network restated with PyTorch's own CPU operators (conv2d,
    conv_transpose2d, avg_pool2d, exact-erf gelu) in float64, its weights
    read from the flat parameter vector p ([columns][Kp] rows, column K =
    tap * cin_padded + c, taps row-major over the 3 x 3 window; transposed
    2 x 2 convolutions with column sub * cout + o, sub = 2 dy + dx)."""
    import torch
    import torch.nn.functional as F

    def wb(l):
        d = spec[l]
        return p[d["woff"]: d["woff"] + d["ncols"] * d["Kp"]].view(d["ncols"], d["Kp"]), \
            p[d["boff"]: d["boff"] + d["cout"]]

    def conv(l, x):
        d = spec[l]
        Wm, b = wb(l)
        cin = x.shape[1]
        if d["kind"] == 2:                                   # 2x2 stride-2 transposed
            w = Wm[:, :cin].reshape(4, d["cout"], cin).permute(2, 1, 0).reshape(cin, d["cout"], 2, 2)
            return F.conv_transpose2d(x, w, b, stride=2)
        if d["kind"] == 1:                                   # 1x1
            return F.conv2d(x, Wm[:, :cin].reshape(d["cout"], cin, 1, 1), b)
        w = torch.stack([Wm[:, t * d["cin_p"]: t * d["cin_p"] + cin] for t in range(9)], dim=-1)
        return F.conv2d(x, w.reshape(d["cout"], cin, 3, 3), b, padding=1)

    h = torch.from_numpy(x[..., :in_ch]).permute(0, 3, 1, 2)
    skips, inp = [], h
    for l in range(4):
        if l > 0:
            inp = F.avg_pool2d(skips[l - 1], 2)
        bo = F.gelu(conv(2 * l + 1, F.gelu(conv(2 * l, inp))))
        if l < 3:
            skips.append(bo)
        else:
            below = bo
    for l in (2, 1, 0):
        base = 8 + 3 * (2 - l)
        cat = torch.cat([skips[l], conv(base, below)], dim=1)
        below = F.gelu(conv(base + 2, F.gelu(conv(base + 1, cat))))
    out = conv(17, below).permute(0, 2, 3, 1)
    d = out[..., :out_ch] - torch.from_numpy(tgt)
    return out, (d * d).sum()


def test_forward_loss_and_gradient_match_torch_restatement():
    """The numpy reference (exact arithmetic) against an independent
    restatement with PyTorch's convolution, transposed convolution, pooling
    and GELU operators and its autograd: output, loss and the whole flat
    gradient (of the mean squared error) agree to FP64 rounding.  This pins
    the forward itself -- padding, tap order, pooling, the up-convolution's
    sub-pixel layout, the skip concatenation order -- which the
    finite-difference pin (backward against the reference's own forward)
    cannot."""
    import torch
    rng = np.random.default_rng(5)
    C, H, B, in_ch, out_ch = 8, 16, 2, 4, 3
    spec, n = layers_spec(C, in_ch, out_ch)
    p = np.zeros(n)
    for d in spec:
        taps = 9 if d["kind"] == 0 else 1
        W = p[d["woff"]: d["woff"] + d["ncols"] * d["Kp"]].reshape(d["ncols"], d["Kp"])
        for t in range(taps):
            W[:, t * d["cin_p"]: t * d["cin_p"] + d["cin"]] = \
                np.sqrt(2.0 / (taps * d["cin"])) * rng.standard_normal((d["ncols"], d["cin"]))
        p[d["boff"]: d["boff"] + d["cout"]] = 0.1 * rng.standard_normal(d["cout"])
    x = np.zeros((B, H, H, 16))
    x[..., :in_ch] = rng.standard_normal((B, H, H, in_ch))
    tgt = rng.standard_normal((B, H, H, out_ch))
    net = UNetRef(C, in_ch, out_ch, p, use_bf16=False)
    out, _ = net.forward(x)
    loss, g = net.loss_and_grads(x, tgt)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    tout, tloss = _torch_unet_loss(pt, spec, x, tgt, in_ch, out_ch)
    (tloss / (B * H * H * out_ch)).backward()
    tout = tout.detach().numpy()
    assert np.max(np.abs(out - tout)) <= 1e-12 * np.max(np.abs(tout))
    assert abs(loss - tloss.item()) <= 1e-12 * loss
    tg = pt.grad.numpy()
    assert np.max(np.abs(g - tg)) <= 1e-10 * np.max(np.abs(tg))


def test_bf16_rounding_is_round_to_nearest_even():
    """The reference's bfloat16 rounding (the points where the GPU stores
    bf16) equals PyTorch's float32 -> bfloat16 conversion bit for bit,
    including exact ties (which go to the even mantissa), signed zeros,
    overflow to infinity and subnormals; values given as float64 are first
    rounded to float32, as the GPU's float accumulators are."""
    import torch
    from oracle.unet_ref import bf16
    rng = np.random.default_rng(11)
    f = np.concatenate([
        rng.standard_normal(20000).astype(np.float32) * np.float32(10.0) ** rng.integers(-30, 30, 20000),
        # exact ties: bf16 mantissa with the dropped half exactly 0x8000, both parities
        (np.arange(1, 4001, dtype=np.uint32) << 16 | 0x8000).view(np.float32),
        np.array([0.0, -0.0, 3.4e38, -3.4e38, 1e-40, -1e-40, 1.0, -1.0], dtype=np.float32),
    ])
    ours = bf16(f)
    ref = torch.from_numpy(f).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref, equal_nan=True)
    assert np.array_equal(np.signbit(ours), np.signbit(ref))
    x64 = rng.standard_normal(1000) * 1e3
    assert np.array_equal(bf16(x64), torch.from_numpy(x64.astype(np.float32)).to(torch.bfloat16).double().numpy())

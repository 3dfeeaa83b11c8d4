"""Plain numpy reference of the surrogate U-Net -- TEST INFRASTRUCTURE.

Forward and backward in FP64 of the network libswof builds (4 levels:
conv3x3-GELU x2 per level, 2x2 average pooling, 2x2 stride-2 transposed
convolutions, skip concatenations, 1x1 output convolution; MSE loss), in the
same flat parameter layout (each layer's weights as [columns][Kp] rows,
K = tap * cin_padded + c, then all biases).  With `bf16=True` it rounds to
bfloat16 (round-to-nearest-even) at the points where the GPU stores bf16
(inputs, weights, pre-activations, activations, pooled maps, output
gradients before each GEMM), so GPU and reference differ only by the order
of FP32 vs FP64 accumulation; with `bf16=False` it is the exact network,
whose backward the finite-difference pins check.
"""
from __future__ import annotations

import numpy as np
from math import erf, sqrt, pi

K_CONV3, K_CONV1, K_CONVT = 0, 1, 2


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


_erf = np.vectorize(erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / sqrt(2.0))) + z * np.exp(-0.5 * z * z) / sqrt(2.0 * pi)


def layers_spec(C: int, in_ch: int, out_ch: int):
    """The layer list in libswof's order: (kind, cin, cout, act)."""
    L = [(K_CONV3, in_ch, C, 1), (K_CONV3, C, C, 1)]
    for l in range(1, 4):
        L += [(K_CONV3, C << (l - 1), C << l, 1), (K_CONV3, C << l, C << l, 1)]
    for l in (2, 1, 0):
        L += [(K_CONVT, C << (l + 1), C << l, 0), (K_CONV3, 2 * (C << l), C << l, 1), (K_CONV3, C << l, C << l, 1)]
    L += [(K_CONV1, C, 16, 0)]
    out = []
    off = 0
    for kind, cin, cout, act in L:
        cin_p = max(cin, 16)
        ncols = 4 * cout if kind == K_CONVT else cout
        taps = 9 if kind == K_CONV3 else 1
        Kp = (taps * cin_p + 63) // 64 * 64
        out.append(dict(kind=kind, cin=cin, cin_p=cin_p, cout=cout, ncols=ncols, Kp=Kp, act=act, woff=off))
        off += ncols * Kp
    for d in out:
        d["boff"] = off
        off += d["cout"]
    return out, off


class UNetRef:
    def __init__(self, C, in_ch, out_ch, params: np.ndarray, use_bf16: bool = True):
        self.C, self.in_ch, self.out_ch = C, in_ch, out_ch
        self.spec, n = layers_spec(C, in_ch, out_ch)
        assert params.size == n
        self.p = params.astype(np.float64).copy()
        self.use_bf16 = use_bf16

    def r(self, x):
        return bf16(x) if self.use_bf16 else np.asarray(x, dtype=np.float64)

    def weights(self, l):
        d = self.spec[l]
        Wm = self.p[d["woff"]: d["woff"] + d["ncols"] * d["Kp"]].reshape(d["ncols"], d["Kp"])
        b = self.p[d["boff"]: d["boff"] + d["cout"]]
        return self.r(Wm), b

    # ---- layer primitives (NHWC) ----
    @staticmethod
    def _taps(x, ks):
        B, H, W, c = x.shape
        h = ks // 2
        xp = np.pad(x, ((0, 0), (h, h), (h, h), (0, 0)))
        return [xp[:, dy:dy + H, dx:dx + W, :] for dy in range(ks) for dx in range(ks)]

    def conv(self, l, x):
        d = self.spec[l]
        Wm, b = self.weights(l)
        B, H, W, c = x.shape
        xin = np.zeros((B, H, W, d["cin_p"]))
        xin[..., :c] = x
        if d["kind"] == K_CONVT:
            Y = xin.reshape(-1, d["cin_p"]) @ Wm[:, : d["cin_p"]].T     # [P, 4*cout]
            co = d["cout"]
            out = np.zeros((B, 2 * H, 2 * W, co))
            Y = Y.reshape(B, H, W, 4, co)
            for sub in range(4):
                out[:, (sub >> 1)::2, (sub & 1)::2, :] = Y[..., sub, :] + b
            return out
        ks = 3 if d["kind"] == K_CONV3 else 1
        cols = np.concatenate(self._taps(xin, ks), axis=-1)             # [B,H,W,taps*cin_p]
        K = cols.shape[-1]
        return cols @ Wm[:, :K].T + b

    def conv_bwd(self, l, x, dz):
        """dz: gradient of the layer output (pre-activation). Returns dW (padded
        [ncols][Kp] layout), db, dx (w.r.t. x with its real channels)."""
        d = self.spec[l]
        Wm, _ = self.weights(l)
        B, H, W, c = x.shape
        xin = np.zeros((B, H, W, d["cin_p"]))
        xin[..., :c] = x
        dW = np.zeros((d["ncols"], d["Kp"]))
        if d["kind"] == K_CONVT:
            co = d["cout"]
            G = np.stack([dz[:, (sub >> 1)::2, (sub & 1)::2, :] for sub in range(4)], axis=3)  # [B,H,W,4,co]
            G = G.reshape(-1, 4 * co)
            dW[:, : d["cin_p"]] = G.T @ xin.reshape(-1, d["cin_p"])
            db = G.reshape(-1, 4, co).sum(axis=(0, 1))
            dx = (G @ Wm[:, : d["cin_p"]]).reshape(B, H, W, d["cin_p"])
            return dW, db, dx[..., :c]
        ks = 3 if d["kind"] == K_CONV3 else 1
        taps = self._taps(xin, ks)
        cols = np.concatenate(taps, axis=-1)
        K = cols.shape[-1]
        Gf = dz.reshape(-1, d["ncols"])
        dW[:, :K] = Gf.T @ cols.reshape(-1, K)
        db = Gf.sum(axis=0)
        dcols = (Gf @ Wm[:, :K]).reshape(B, H, W, K)
        h = ks // 2
        dxp = np.zeros((B, H + 2 * h, W + 2 * h, d["cin_p"]))
        t = 0
        for dy in range(ks):
            for dxx in range(ks):
                dxp[:, dy:dy + H, dxx:dxx + W, :] += dcols[..., t * d["cin_p"]:(t + 1) * d["cin_p"]]
                t += 1
        dx = dxp[:, h:h + H, h:h + W, :]
        return dW, db, dx[..., :c]

    @staticmethod
    def pool(x):
        return 0.25 * (x[:, 0::2, 0::2] + x[:, 1::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 1::2])

    @staticmethod
    def pool_bwd(g):
        return np.repeat(np.repeat(0.25 * g, 2, axis=1), 2, axis=2)

    # ---- network ----
    def forward(self, x):
        """x: [B,H,W,16] network input (already normalised). Returns the
        16-channel FP64 output and the cache for backward."""
        r = self.r
        C = self.C
        cache = {}
        h = r(x)
        cache["x0"] = h
        cat = {}
        inp = h
        for l in range(4):
            if l > 0:
                inp = r(self.pool(cat[l - 1][..., : C << (l - 1)]))
                cache[f"pool{l}"] = inp
            za = r(self.conv(2 * l, inp))
            a = r(gelu(za))
            zb = r(self.conv(2 * l + 1, a))
            bo = r(gelu(zb))
            cache[f"in{l}"], cache[f"za{l}"], cache[f"a{l}"], cache[f"zb{l}"] = inp, za, a, zb
            if l < 3:
                cat[l] = np.concatenate([bo, np.zeros_like(bo)], axis=-1)
            else:
                cache["bott"] = bo
        below = cache["bott"]
        for l in (2, 1, 0):
            base = 8 + 3 * (2 - l)
            up = r(self.conv(base, below))
            c = C << l
            cat[l][..., c:] = up
            cache[f"below{l}"] = below
            cache[f"cat{l}"] = cat[l].copy()
            zda = r(self.conv(base + 1, cat[l]))
            da = r(gelu(zda))
            zdb = r(self.conv(base + 2, da))
            db = r(gelu(zdb))
            cache[f"zda{l}"], cache[f"da{l}"], cache[f"zdb{l}"], cache[f"db{l}"] = zda, da, zdb, db
            below = db
        out = self.conv(17, below)
        return out, cache

    def loss_and_grads(self, x, tgt):
        """MSE over the first out_ch channels; returns (sum of squared
        errors, flat gradient)."""
        r = self.r
        C = self.C
        out, ca = self.forward(x)
        P = out.shape[0] * out.shape[1] * out.shape[2]
        d = out[..., : self.out_ch] - tgt
        loss = float(np.sum(d * d))
        g = np.zeros_like(self.p)

        def put(l, dW, db):
            s = self.spec[l]
            g[s["woff"]: s["woff"] + s["ncols"] * s["Kp"]] += dW.ravel()
            g[s["boff"]: s["boff"] + s["cout"]] += db

        dy = np.zeros_like(out)
        dy[..., : self.out_ch] = 2.0 * d / (P * self.out_ch)
        dW, db, dx = self.conv_bwd(17, ca["db0"], r(dy))
        put(17, dW, db)
        g_db = {0: dx}
        g_cat = {}
        for l in (0, 1, 2):
            base = 8 + 3 * (2 - l)
            c = C << l
            dz = r(g_db[l] * gelu_grad(ca[f"zdb{l}"]))
            dW, db, dx = self.conv_bwd(base + 2, ca[f"da{l}"], dz)
            put(base + 2, dW, db)
            dz = r(dx * gelu_grad(ca[f"zda{l}"]))
            dW, db, dx = self.conv_bwd(base + 1, ca[f"cat{l}"], dz)
            put(base + 1, dW, db)
            g_cat[l] = dx
            dz = r(g_cat[l][..., c:])
            dW, db, dx = self.conv_bwd(base, ca[f"below{l}"], dz)
            put(base, dW, db)
            if l < 2:
                g_db[l + 1] = dx
            else:
                g_bott = dx
        for l in (3, 2, 1, 0):
            c = C << l
            dyb = g_bott if l == 3 else g_cat[l][..., :c]
            dz = r(dyb * gelu_grad(ca[f"zb{l}"]))
            dW, db, dx = self.conv_bwd(2 * l + 1, ca[f"a{l}"], dz)
            put(2 * l + 1, dW, db)
            dz = r(dx * gelu_grad(ca[f"za{l}"]))
            dW, db, dx = self.conv_bwd(2 * l, ca[f"in{l}"], dz)
            put(2 * l, dW, db)
            if l > 0:
                g_cat[l - 1][..., : C << (l - 1)] += self.pool_bwd(dx)
        return loss, g

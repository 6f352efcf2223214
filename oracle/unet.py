"""The learned warm start's network, FP64 (test infrastructure only).

A 4-level convolutional U-Net with 32 base channels maps a frame pair
(p0, p1) to the four fields of a converged Algorithm 1 state (Mx, My, r, a),
which then warm-start the solver (Sec. III-B: the iterates are cached and
warm-started; this network predicts the cache for a new pair).  The plain
iterations always run to the stopping rule afterwards, so the network only
changes how many iterations that takes.

Architecture (every 3x3 convolution zero-padded, followed by ReLU except the
1x1 head):
  enc0: 2 -> C, C -> C          at H x W            (skip s0)
  enc1: C -> 2C, 2C -> 2C       at H/2 (2x2 average pooling before)  (s1)
  enc2: 2C -> 4C, 4C -> 4C      at H/4              (s2)
  bott: 4C -> 8C, 8C -> 8C      at H/8
  dec2: [up(8C), s2] -> 4C, 4C -> 4C      (nearest-neighbour 2x upsampling)
  dec1: [up(4C), s1] -> 2C, 2C -> 2C
  dec0: [up(2C), s0] -> C, C -> C
  head: C -> 4 (1x1)
Layout [N][C][H][W]; H and W divisible by 8.

Plain definitions, no fusion: conv2d is the direct sum over input channels
and kernel offsets; its gradients are the same sums with the roles of the
tensors exchanged.  Pinned in tests/test_oracle_unet.py by central finite
differences of the loss.

Storage precision.  ``forward`` and ``backward`` take an optional rounding
``rnd`` applied wherever a mixed-precision implementation stores a tensor in
a narrower type: every hidden activation (after ReLU), every pooled tensor,
every data gradient and every summed gradient (upsampling's adjoint, the
skip plus pooled paths).  The network output, the loss gradient and the
weight gradients are not rounded.  ``round_bf16`` is the bfloat16 rounding
(8 significant bits, ties to even); with ``rnd=None`` everything is FP64.
"""
from __future__ import annotations

import numpy as np


def round_bf16(x) -> np.ndarray:
    """Nearest bfloat16 value (8 significant bits, ties to even), in FP64."""
    m, e = np.frexp(np.asarray(x, np.float64))      # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)


def _ident(v):
    return v


def layer_specs(base: int = 32, cin: int = 2, cout: int = 4) -> list[tuple[str, int, int, int]]:
    """(name, in channels, out channels, kernel size) of every convolution, in
    forward order."""
    c = base
    return [("enc0a", cin, c, 3), ("enc0b", c, c, 3),
            ("enc1a", c, 2 * c, 3), ("enc1b", 2 * c, 2 * c, 3),
            ("enc2a", 2 * c, 4 * c, 3), ("enc2b", 4 * c, 4 * c, 3),
            ("botta", 4 * c, 8 * c, 3), ("bottb", 8 * c, 8 * c, 3),
            ("dec2a", 8 * c + 4 * c, 4 * c, 3), ("dec2b", 4 * c, 4 * c, 3),
            ("dec1a", 4 * c + 2 * c, 2 * c, 3), ("dec1b", 2 * c, 2 * c, 3),
            ("dec0a", 2 * c + c, c, 3), ("dec0b", c, c, 3),
            ("head", c, cout, 1)]


def init_params(rng: np.random.Generator, base: int = 32) -> dict:
    """He-normal weights, zero biases."""
    out = {}
    for name, ci, co, k in layer_specs(base):
        std = np.sqrt(2.0 / (ci * k * k))
        out[name] = (rng.normal(0.0, std, (co, ci, k, k)), np.zeros(co))
    return out


def conv2d(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n, o, i, j] = b[o] + sum_{c, u, v} w[o, c, u, v] x[n, c, i + u - p, j + v - p],
    p = (k - 1) / 2, zero outside the image."""
    k = w.shape[-1]
    p = (k - 1) // 2
    n, c, h, wd = x.shape
    xp = np.zeros((n, c, h + 2 * p, wd + 2 * p))
    xp[:, :, p:p + h, p:p + wd] = x
    y = np.zeros((n, w.shape[0], h, wd)) + b[None, :, None, None]
    for u in range(k):
        for v in range(k):
            y += np.einsum("oc,nchw->nohw", w[:, :, u, v], xp[:, :, u:u + h, v:v + wd])
    return y


def conv2d_grads(x: np.ndarray, w: np.ndarray, gy: np.ndarray):
    """Gradients of conv2d with respect to x, w and b, given dL/dy."""
    k = w.shape[-1]
    p = (k - 1) // 2
    n, c, h, wd = x.shape
    xp = np.zeros((n, c, h + 2 * p, wd + 2 * p))
    xp[:, :, p:p + h, p:p + wd] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for u in range(k):
        for v in range(k):
            gw[:, :, u, v] = np.einsum("nohw,nchw->oc", gy, xp[:, :, u:u + h, v:v + wd])
            gxp[:, :, u:u + h, v:v + wd] += np.einsum("oc,nohw->nchw", w[:, :, u, v], gy)
    return gxp[:, :, p:p + h, p:p + wd], gw, gy.sum(axis=(0, 2, 3))


def avgpool2(x: np.ndarray) -> np.ndarray:
    n, c, h, w = x.shape
    return x.reshape(n, c, h // 2, 2, w // 2, 2).mean(axis=(3, 5))


def avgpool2_grad(g: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3) / 4.0


def up2(x: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up2_grad(g: np.ndarray) -> np.ndarray:
    n, c, h, w = g.shape
    return g.reshape(n, c, h // 2, 2, w // 2, 2).sum(axis=(3, 5))


def forward(params: dict, x: np.ndarray, rnd=None):
    """Network output [N, 4, H, W] and the activations the backward pass needs."""
    rnd = rnd or _ident
    cache = {"x": x}

    def cr(name, inp):
        w, b = params[name]
        y = rnd(np.maximum(conv2d(inp, w, b), 0.0))
        cache[name] = (inp, y)
        return y

    s0 = cr("enc0b", cr("enc0a", x))
    s1 = cr("enc1b", cr("enc1a", rnd(avgpool2(s0))))
    s2 = cr("enc2b", cr("enc2a", rnd(avgpool2(s1))))
    bt = cr("bottb", cr("botta", rnd(avgpool2(s2))))
    d2 = cr("dec2b", cr("dec2a", np.concatenate([up2(bt), s2], axis=1)))
    d1 = cr("dec1b", cr("dec1a", np.concatenate([up2(d2), s1], axis=1)))
    d0 = cr("dec0b", cr("dec0a", np.concatenate([up2(d1), s0], axis=1)))
    w, b = params["head"]
    out = conv2d(d0, w, b)
    cache["head"] = (d0, out)
    return out, cache


def backward(params: dict, cache: dict, g_out: np.ndarray, rnd=None) -> dict:
    """dL/d(params) given dL/d(output)."""
    rnd = rnd or _ident
    grads = {}

    def back(name, gy, relu=True):
        inp, y = cache[name]
        if relu:
            gy = gy * (y > 0)
        gx, gw, gb = conv2d_grads(inp, params[name][0], gy)
        grads[name] = (gw, gb)
        return rnd(gx)

    c8 = params["bottb"][0].shape[0]
    c4 = params["dec2b"][0].shape[0]
    c2 = params["dec1b"][0].shape[0]
    g = back("head", g_out, relu=False)
    g = back("dec0a", back("dec0b", g))
    g_up1, g_s0 = g[:, :c2], g[:, c2:]
    g = back("dec1a", back("dec1b", rnd(up2_grad(g_up1))))
    g_up2, g_s1 = g[:, :c4], g[:, c4:]
    g = back("dec2a", back("dec2b", rnd(up2_grad(g_up2))))
    g_bt, g_s2 = g[:, :c8], g[:, c8:]
    g = back("botta", back("bottb", rnd(up2_grad(g_bt))))
    g = back("enc2a", back("enc2b", rnd(avgpool2_grad(g) + g_s2)))
    g = back("enc1a", back("enc1b", rnd(avgpool2_grad(g) + g_s1)))
    back("enc0a", back("enc0b", rnd(avgpool2_grad(g) + g_s0)))
    return grads


def mse(out: np.ndarray, target: np.ndarray) -> tuple[float, np.ndarray]:
    """Mean squared error over all entries and its gradient."""
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size

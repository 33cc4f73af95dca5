"""Plain numpy oracle of the warm-start U-Net: forward and backward in FP64.

TEST INFRASTRUCTURE ONLY (used by the tests to check the GPU network's
outputs and gradients; pinned itself by central finite differences).

Same architecture and parameter layout as the library's network:
  level 0:  conv(16 -> w0) relu, conv(w0 -> w0) relu                  -> e0
  level l:  avgpool2(e_{l-1}), conv(-> w_l) relu, conv relu           -> e_l
  decoder:  concat[up2(d_{l+1} or e3), e_l] -> conv relu, conv relu  -> d_l
  head:     conv(w0 -> 16), output channel 0
every convolution 3x3 with zero padding, weights [Cout][9][Cin] with
tap = 3*(dy+1) + (dx+1), followed by the bias [Cout]; the 4 input features
are zero-padded to 16 channels.  With bf16=True the activations are rounded
to bfloat16 (round to nearest even) where the GPU stores them.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def layers(w):
    """(cin, cout, relu) of the 15 convolutions, in parameter order."""
    L = [(16, w[0], True), (w[0], w[0], True)]
    for l in range(1, 4):
        L += [(w[l - 1], w[l], True), (w[l], w[l], True)]
    L += [(w[3] + w[2], w[2], True), (w[2], w[2], True), (w[2] + w[1], w[1], True), (w[1], w[1], True),
          (w[1] + w[0], w[0], True), (w[0], w[0], True), (w[0], 16, False)]
    return L


def unpack(params, w):
    out, off = [], 0
    for cin, cout, relu in layers(w):
        W = params[off:off + cout * 9 * cin].reshape(cout, 9, cin)
        off += cout * 9 * cin
        b = params[off:off + cout]
        off += cout
        out.append((W, b, relu))
    assert off == params.size
    return out


def conv(x, W, b):
    H, Wd, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    y = np.zeros((H, Wd, W.shape[0]))
    for tap in range(9):
        dy, dx = tap // 3, tap % 3
        y += xp[dy:dy + H, dx:dx + Wd, :] @ W[:, tap, :].T
    return y + b


def conv_backward(x, W, gy):
    """Gradients of y = conv(x, W) + b with respect to x, W and b."""
    H, Wd, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for tap in range(9):
        dy, dx = tap // 3, tap % 3
        xs = xp[dy:dy + H, dx:dx + Wd, :]
        gW[:, tap, :] = np.einsum("hwo,hwi->oi", gy, xs)
        gxp[dy:dy + H, dx:dx + Wd, :] += gy @ W[:, tap, :]
    return gxp[1:-1, 1:-1, :], gW, gy.sum(axis=(0, 1))


def pool(x):
    return 0.25 * (x[0::2, 0::2] + x[0::2, 1::2] + x[1::2, 0::2] + x[1::2, 1::2])


def pool_backward(g):
    return 0.25 * np.repeat(np.repeat(g, 2, axis=0), 2, axis=1)


def up(x):
    return np.repeat(np.repeat(x, 2, axis=0), 2, axis=1)


def up_backward(g):
    return g[0::2, 0::2] + g[0::2, 1::2] + g[1::2, 0::2] + g[1::2, 1::2]


def forward(params, w, feat, bf16=False):
    """feat [H][W][4] -> out [H][W] and the cache for backward."""
    R = bf16_round if bf16 else (lambda a: a)
    P = unpack(params, w)
    H, Wd, _ = feat.shape
    x = np.zeros((H, Wd, 16))
    x[..., :4] = feat
    x = R(x)
    cache = {"x": [], "y": []}

    def run(k, inp):
        Wk, bk, relu = P[k]
        y = conv(inp, R(Wk), bk)
        if relu:
            y = np.maximum(y, 0.0)
        y = R(y) if k != 14 else y
        cache["x"].append((k, inp))
        cache["y"].append((k, y))
        return y

    e = []
    h = x
    for l in range(4):
        if l > 0:
            h = R(pool(e[-1]))
        a = run(2 * l, h)
        e.append(run(2 * l + 1, a))
    d = e[3]
    for l, k in zip((2, 1, 0), (8, 10, 12)):
        cat = np.concatenate([up(d), e[l]], axis=2)
        b_ = run(k, cat)
        d = run(k + 1, b_)
    out = run(14, d)
    return out[..., 0], cache


def loss_and_grad(params, w, feat, target, bf16=False, trace=None):
    """Mean squared error of output channel 0 and its gradient (flat).  With
    a dict `trace`, trace[k] receives (input, output gradient after the ReLU
    mask, weights as used) of convolution k: the operands of its weight and
    bias gradients."""
    R = bf16_round if bf16 else (lambda a: a)
    P = unpack(params, w)
    out, cache = forward(params, w, feat, bf16)
    xs = dict(cache["x"])
    ys = dict(cache["y"])
    n = out.size
    loss = float(np.mean((out - target) ** 2))
    grads = [None] * 15

    def back(k, gy):
        Wk, bk, relu = P[k]
        if relu:
            gy = gy * (ys[k] > 0)
        if trace is not None:
            trace[k] = (xs[k], gy, R(Wk))
        gx, gW, gb = conv_backward(xs[k], R(Wk), gy)
        grads[k] = (gW, gb)
        return R(gx)

    H, Wd = out.shape
    gout = np.zeros((H, Wd, 16))
    gout[..., 0] = R(2.0 * (out - target) / n)
    gd = back(14, gout)
    ge = {}
    for l, k in zip((0, 1, 2), (12, 10, 8)):
        gb_ = back(k + 1, gd)
        gcat = back(k, gb_)
        cup = gcat.shape[2] - w[l]
        ge[l] = gcat[..., cup:]
        gd = R(up_backward(gcat[..., :cup]))
    g_e = gd  # gradient of e3
    for l in (3, 2, 1, 0):
        if l < 3:
            g_e = R(ge[l] + g_pool)
        ga = back(2 * l + 1, g_e)
        gin = back(2 * l, ga)
        if l > 0:
            g_pool = R(pool_backward(gin))
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def num_params(w):
    return sum(cout * 9 * cin + cout for cin, cout, _ in layers(w))

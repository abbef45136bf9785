"""FP64 reference of the multigrid warm-start network (TEST INFRASTRUCTURE ONLY).

A 3D U-Net maps the normalised pressure right-hand side and density,
(f / rms(f), rho / max(rho)), to the normalised pressure p / (rms(f) max(rho) h^2)
(h: the grid spacing).  The paper has no network; this is a learned
first guess for the pressure solve (a form of the solver, not of the
method).  Only tests/ and the bench's CPU legs use this module.

Architecture (one 3x3x3 convolution per level, zero padding, ReLU after every
convolution but the last, 2x2x2 average pooling down, nearest upsampling up,
skip connections by channel concatenation):

    e0 = relu(conv(x, 2->16));          e1 = relu(conv(pool(e0), 16->32))
    e2 = relu(conv(pool(e1), 32->64));  b  = relu(conv(pool(e2), 64->128))
    d2 = relu(conv([up(b), e2], 192->64))
    d1 = relu(conv([up(d2), e1], 96->32))
    d0 = relu(conv([up(d1), e0], 48->16))
    y  = conv1x1(d0, 16->1)

Arrays are channels-last: an activation is (nz, ny, nx, C); a 3x3x3 weight is
(27, Cout, Cin) with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1); biases are (Cout,).
Everything here is plain FP64 numpy written from the definitions: a
convolution is a sum over the 27 shifted inputs, its gradients are the
transposed sums.

Storage precision.  forward() and backward() take an optional `store`
function applied to every array the GPU network keeps in memory (the input,
each convolution's activated output, each pooled array, the loss gradient,
each data gradient and each accumulated skip gradient).  With store=None the
network is plain FP64.  With store=bf16_round the stored values, and with them
the ReLU decisions (y > 0) that select which gradients flow, are those of a
network that keeps its activations in bfloat16, so that comparisons with such
a network compare arithmetic rather than the discontinuous ReLU masks.  The
arithmetic between storage points stays FP64.
"""
from __future__ import annotations

import numpy as np

LAYERS = [  # name, Cin, Cout, taps
    ("e0", 2, 16, 27), ("e1", 16, 32, 27), ("e2", 32, 64, 27), ("b", 64, 128, 27),
    ("d2", 192, 64, 27), ("d1", 96, 32, 27), ("d0", 48, 16, 27), ("head", 16, 1, 1),
]


def bf16_round(a):
    """Round to bfloat16 (8 exponent bits, 7 stored mantissa bits) by
    round-to-nearest, ties-to-even, of the FP32 value; returned as FP64.
    The FP32 bit pattern keeps its top 16 bits after adding 0x7FFF plus the
    lowest kept bit (the tie breaker).  Finite inputs only."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _identity(a):
    return a


def param_count() -> int:
    return sum(t * ci * co + co for _, ci, co, t in LAYERS)


def init_params(seed: int = 0) -> dict:
    """He-normal weights, zero biases (a seeded input to both sides)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co, t in LAYERS:
        P[name + ".w"] = rng.standard_normal((t, co, ci)) * np.sqrt(2.0 / (t * ci))
        P[name + ".b"] = np.zeros(co)
    return P


def _taps(ntap):
    if ntap == 1:
        return [(0, 0, 0)]
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(x, dz, dy, dx):
    """out[z, y, x] = x[z+dz, y+dy, x+dx], zero outside the box."""
    nz, ny, nx = x.shape[:3]
    out = np.zeros_like(x)
    zs, ys, xs = slice(max(0, -dz), nz - max(0, dz)), slice(max(0, -dy), ny - max(0, dy)), slice(max(0, -dx), nx - max(0, dx))
    zd, yd, xd = slice(max(0, dz), nz - max(0, -dz)), slice(max(0, dy), ny - max(0, -dy)), slice(max(0, dx), nx - max(0, -dx))
    out[zs, ys, xs] = x[zd, yd, xd]
    return out


def conv(x, w, b):
    """y[v, co] = b[co] + sum_t sum_ci x[v + off(t), ci] w[t, co, ci]."""
    y = np.zeros(x.shape[:3] + (w.shape[1],)) + b
    for t, (dz, dy, dx) in enumerate(_taps(w.shape[0])):
        y += _shift(x, dz, dy, dx) @ w[t].T
    return y


def conv_backward(x, w, dy):
    """Gradients of conv with respect to x, w and b."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (dz, dy_, dx_) in enumerate(_taps(w.shape[0])):
        xs = _shift(x, dz, dy_, dx_)
        dw[t] = np.einsum("zyxo,zyxi->oi", dy, xs)
        dx += _shift(dy @ w[t], -dz, -dy_, -dx_)
    db = dy.sum(axis=(0, 1, 2))
    return dx, dw, db


def pool(x):
    nz, ny, nx, c = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(1, 3, 5))


def pool_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_backward(dy):
    nz, ny, nx, c = dy.shape
    return dy.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).sum(axis=(1, 3, 5))


def forward(P, x, store=None):
    """x: (nz, ny, nx, 2); extents divisible by 8.  Returns y (nz, ny, nx, 1)
    and the cache the backward pass needs.  store: see the module docstring."""
    S = store or _identity
    c = {"x": S(x)}
    relu = lambda a: np.maximum(a, 0.0)
    c["e0"] = S(relu(conv(c["x"], P["e0.w"], P["e0.b"])))
    c["p0"] = S(pool(c["e0"]))
    c["e1"] = S(relu(conv(c["p0"], P["e1.w"], P["e1.b"])))
    c["p1"] = S(pool(c["e1"]))
    c["e2"] = S(relu(conv(c["p1"], P["e2.w"], P["e2.b"])))
    c["p2"] = S(pool(c["e2"]))
    c["b"] = S(relu(conv(c["p2"], P["b.w"], P["b.b"])))
    c["c2"] = np.concatenate([up(c["b"]), c["e2"]], axis=3)
    c["d2"] = S(relu(conv(c["c2"], P["d2.w"], P["d2.b"])))
    c["c1"] = np.concatenate([up(c["d2"]), c["e1"]], axis=3)
    c["d1"] = S(relu(conv(c["c1"], P["d1.w"], P["d1.b"])))
    c["c0"] = np.concatenate([up(c["d1"]), c["e0"]], axis=3)
    c["d0"] = S(relu(conv(c["c0"], P["d0.w"], P["d0.b"])))
    y = conv(c["d0"], P["head.w"], P["head.b"])
    return y, c


def loss(y, t):
    """Mean squared error over all voxels."""
    return float(np.mean((y - t) ** 2))


def backward(P, c, y, t, store=None):
    """Gradients of the mean squared error with respect to every parameter.
    store: see the module docstring."""
    S = store or _identity
    G = {}
    dy = S(2.0 * (y - t) / y.size)

    def cb(x, w, g):
        dx, dw, db = conv_backward(x, w, g)
        return S(dx), dw, db

    dd0, G["head.w"], G["head.b"] = cb(c["d0"], P["head.w"], dy)
    dd0 = dd0 * (c["d0"] > 0)
    dc0, G["d0.w"], G["d0.b"] = cb(c["c0"], P["d0.w"], dd0)
    k = c["d1"].shape[3]
    dd1 = S(up_backward(dc0[..., :k])) * (c["d1"] > 0)
    de0 = dc0[..., k:]
    dc1, G["d1.w"], G["d1.b"] = cb(c["c1"], P["d1.w"], dd1)
    k = c["d2"].shape[3]
    dd2 = S(up_backward(dc1[..., :k])) * (c["d2"] > 0)
    de1 = dc1[..., k:]
    dc2, G["d2.w"], G["d2.b"] = cb(c["c2"], P["d2.w"], dd2)
    k = c["b"].shape[3]
    db_ = S(up_backward(dc2[..., :k])) * (c["b"] > 0)
    de2 = dc2[..., k:]
    dp2, G["b.w"], G["b.b"] = cb(c["p2"], P["b.w"], db_)
    de2 = S(de2 + pool_backward(dp2)) * (c["e2"] > 0)
    dp1, G["e2.w"], G["e2.b"] = cb(c["p1"], P["e2.w"], de2)
    de1 = S(de1 + pool_backward(dp1)) * (c["e1"] > 0)
    dp0, G["e1.w"], G["e1.b"] = cb(c["p0"], P["e1.w"], de1)
    de0 = S(de0 + pool_backward(dp0)) * (c["e0"] > 0)
    _, G["e0.w"], G["e0.b"] = conv_backward(c["x"], P["e0.w"], de0)
    return G


def adam_step(P, G, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) of every parameter in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m." + k, np.zeros_like(P[k]))
        v = state.setdefault("v." + k, np.zeros_like(P[k]))
        m[...] = b1 * m + (1 - b1) * G[k]
        v[...] = b2 * v + (1 - b2) * G[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[k] -= lr * mh / (np.sqrt(vh) + eps)

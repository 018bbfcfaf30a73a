"""ORACLE (test infrastructure).  The learned warm start: a 3D convolutional U-Net, its
gradients, the mean-squared loss and the Adam update, in plain float64 numpy.

Sec. 5 names the solver as a source of datasets for data-driven models without fixing a model;
the network here is the one this project builds as such a model (a 4-level 3D U-Net, 3x3x3
convolutions with zero padding, ReLU, 2x2x2 average pooling, nearest-neighbour upsampling with
skip concatenation, a 1x1x1 output head).  Every operation is written from its definition:

    conv3d:  y[b,o,z,y,x] = bias[o] + sum_{i,dz,dy,dx} w[o,i,dz,dy,dx] x[b,i,z+dz-1,y+dy-1,x+dx-1]
             (x = 0 outside the grid; a 1x1x1 head has a single tap at offset 0)
    pool:    y[b,c,Z,Y,X] = mean of the 2x2x2 block of x at (2Z, 2Y, 2X)
    up:      y[b,c,z,y,x] = x[b,c,z//2,y//2,x//2]
    relu:    max(x, 0)
    loss:    L = mean over every element of (y - t)^2
    Adam:    m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
             p <- p - lr (m / (1-b1^k)) / (sqrt(v / (1-b2^k)) + eps)      (step k = 1, 2, ...)

Arrays are (batch, channels, z, y, x).  The backward functions return the exact adjoints of the
forward ones.  No blocking or reordering beyond these definitions.

Storage precision.  forward / backward take an optional rounding function q applied where a
reduced-precision implementation stores values: the network input, every weight, each
convolution's activated output, each pooled map, and the gradient entering each convolution's
backward (after the ReLU mask).  bf16() rounds to bfloat16 (round to nearest, ties to even).
With q = None everything stays float64.
"""
from __future__ import annotations

import numpy as np

# -- single operations ------------------------------------------------------------------------


def bf16(a):
    """round to the nearest bfloat16 (8 significant bits; ties to even), returned as float64"""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def taps(k):
    """offsets (dz, dy, dx) of a k x k x k kernel (k = 3 or 1), in the weight array's order"""
    r = range(-(k // 2), k // 2 + 1)
    return [(dz, dy, dx) for dz in r for dy in r for dx in r]


def shift(x, dz, dy, dx):
    """s[..., z, y, x] = x[..., z+dz, y+dy, x+dx], zero outside the grid"""
    out = np.zeros_like(x)
    Z, Y, X = x.shape[-3:]
    zs, ys, xs = slice(max(0, -dz), min(Z, Z - dz)), slice(max(0, -dy), min(Y, Y - dy)), slice(max(0, -dx), min(X, X - dx))
    zt, yt, xt = slice(max(0, dz), min(Z, Z + dz)), slice(max(0, dy), min(Y, Y + dy)), slice(max(0, dx), min(X, X + dx))
    out[..., zs, ys, xs] = x[..., zt, yt, xt]
    return out


def conv3d(x, w, b):
    """x (B, Ci, Z, Y, X), w (Co, Ci, k, k, k), b (Co,) -> (B, Co, Z, Y, X)"""
    k = w.shape[-1]
    y = np.zeros((x.shape[0], w.shape[0]) + x.shape[2:])
    for t, (dz, dy, dx) in enumerate(taps(k)):
        wt = w.reshape(w.shape[0], w.shape[1], -1)[:, :, t]
        y += np.einsum("oi,bizyx->bozyx", wt, shift(x, dz, dy, dx))
    return y + b[None, :, None, None, None]


def conv3d_backward(x, w, dy):
    """adjoints of conv3d: (dx, dw, db) for upstream gradient dy"""
    k = w.shape[-1]
    dx = np.zeros_like(x)
    dw = np.zeros_like(w).reshape(w.shape[0], w.shape[1], -1)
    for t, (dz, dy_, dx_) in enumerate(taps(k)):
        wt = w.reshape(w.shape[0], w.shape[1], -1)[:, :, t]
        xs = shift(x, dz, dy_, dx_)
        dw[:, :, t] = np.einsum("bozyx,bizyx->oi", dy, xs)
        # the adjoint of shift(+d) is shift(-d)
        dx += shift(np.einsum("oi,bozyx->bizyx", wt, dy), -dz, -dy_, -dx_)
    return dx, dw.reshape(w.shape), dy.sum(axis=(0, 2, 3, 4))


def pool(x):
    B, C, Z, Y, X = x.shape
    return x.reshape(B, C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(3, 5, 7))


def pool_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, axis=2), 2, axis=3), 2, axis=4) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=2), 2, axis=3), 2, axis=4)


def up_backward(dy):
    B, C, Z, Y, X = dy.shape
    return dy.reshape(B, C, Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(3, 5, 7))


def relu(x):
    return np.maximum(x, 0.0)


def mse(y, t):
    """loss and its gradient with respect to y"""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


# -- the network ------------------------------------------------------------------------------


def layer_names(levels):
    """parameter names in a fixed order: encoder convs, decoder convs, head"""
    names = []
    for l in range(levels):
        names += [f"enc{l}a", f"enc{l}b"]
    for l in range(levels - 2, -1, -1):
        names += [f"dec{l}a", f"dec{l}b"]
    return names + ["head"]


def shapes(cin, cout, chans):
    """{name: (Co, Ci, k)} for the U-Net with per-level channels `chans`"""
    L = len(chans)
    s = {}
    c_prev = cin
    for l in range(L):
        s[f"enc{l}a"] = (chans[l], c_prev, 3)
        s[f"enc{l}b"] = (chans[l], chans[l], 3)
        c_prev = chans[l]
    for l in range(L - 2, -1, -1):
        s[f"dec{l}a"] = (chans[l], c_prev + chans[l], 3)    # upsampled deeper features ++ skip
        s[f"dec{l}b"] = (chans[l], chans[l], 3)
        c_prev = chans[l]
    s["head"] = (cout, chans[0], 1)
    return s


def init(cin, cout, chans, seed):
    """He-normal weights, zero biases (float64)"""
    g = np.random.default_rng(seed)
    p = {}
    for n, (co, ci, k) in shapes(cin, cout, chans).items():
        p[n + ".w"] = g.normal(0.0, np.sqrt(2.0 / (ci * k ** 3)), size=(co, ci, k, k, k))
        p[n + ".b"] = np.zeros(co)
    return p


def forward(p, x, levels, q=None):
    """U-Net forward; returns the output and the cache the backward pass needs"""
    q = q or (lambda a: a)
    cache = {"q": q}
    h = q(x)
    skips = []
    for l in range(levels):
        if l > 0:
            h = q(pool(h))
        for s in "ab":
            n = f"enc{l}{s}"
            cache[n] = h
            h = q(relu(conv3d(h, q(p[n + ".w"]), p[n + ".b"])))
            cache[n + ".out"] = h
        skips.append(h)
    for l in range(levels - 2, -1, -1):
        h = np.concatenate([up(h), skips[l]], axis=1)
        for s in "ab":
            n = f"dec{l}{s}"
            cache[n] = h
            h = q(relu(conv3d(h, q(p[n + ".w"]), p[n + ".b"])))
            cache[n + ".out"] = h
    cache["head"] = h
    return conv3d(h, q(p["head.w"]), p["head.b"]), cache


def backward(p, cache, dout, levels):
    """gradients {name: array} of the loss with respect to every parameter"""
    q = cache["q"]
    g = {}
    dx, g["head.w"], g["head.b"] = conv3d_backward(cache["head"], q(p["head.w"]), q(dout))
    dskip = {}
    for l in range(0, levels - 1):
        for s in "ba":
            n = f"dec{l}{s}"
            dpre = q(dx * (cache[n + ".out"] > 0))
            dx, g[n + ".w"], g[n + ".b"] = conv3d_backward(cache[n], q(p[n + ".w"]), dpre)
        c_up = dx.shape[1] - cache[f"enc{l}b.out"].shape[1]
        dskip[l] = dx[:, c_up:]
        dx = up_backward(dx[:, :c_up])
    for l in range(levels - 1, -1, -1):
        if l in dskip:
            dx = dx + dskip[l]
        for s in "ba":
            n = f"enc{l}{s}"
            dpre = q(dx * (cache[n + ".out"] > 0))
            dx, g[n + ".w"], g[n + ".b"] = conv3d_backward(cache[n], q(p[n + ".w"]), dpre)
        if l > 0:
            dx = pool_backward(dx)
    return g


def flat(p, levels):
    """parameters as one vector: per layer (in layer_names order) the weights, then the biases"""
    return np.concatenate([np.concatenate([p[n + ".w"].ravel(), p[n + ".b"].ravel()]) for n in layer_names(levels)])


def unflat(v, cin, cout, chans):
    p, o = {}, 0
    s = shapes(cin, cout, chans)
    for n in layer_names(len(chans)):
        co, ci, k = s[n]
        p[n + ".w"] = np.asarray(v[o:o + co * ci * k ** 3], dtype=np.float64).reshape(co, ci, k, k, k)
        o += co * ci * k ** 3
        p[n + ".b"] = np.asarray(v[o:o + co], dtype=np.float64)
        o += co
    return p


def adam(p, g, m, v, k, lr, b1=0.9, b2=0.999, eps=1e-8):
    """one Adam step k (1-based) on every parameter, in place"""
    for n in p:
        m[n] = b1 * m[n] + (1 - b1) * g[n]
        v[n] = b2 * v[n] + (1 - b2) * g[n] ** 2
        mh = m[n] / (1 - b1 ** k)
        vh = v[n] / (1 - b2 ** k)
        p[n] = p[n] - lr * mh / (np.sqrt(vh) + eps)


def train_step(p, m, v, k, x, t, levels, lr):
    y, cache = forward(p, x, levels)
    loss, dy = mse(y, t)
    g = backward(p, cache, dy, levels)
    adam(p, g, m, v, k, lr)
    return loss

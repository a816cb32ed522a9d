"""FP64 CPU oracle of the warm-start U-Net (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import this
module; the CUDA library never uses it.  It restates the network from its definition:

  encoder   conv3x3 + ReLU pairs with 12, 24, 48, 96 channels, 2x2 average pooling between
  decoder   nearest 2x upsampling, channel concatenation [upsampled, skip], conv3x3 + ReLU pairs
            with 48, 24, 12 channels, then a 1x1 convolution to one channel (no ReLU)

Tensors are NHWC.  The parameter vector holds, layer by layer, W[Cout][3][3][Cin] (W[Cout][Cin]
for the 1x1) and then b[Cout].  Convolutions are zero-padded, stride 1, and compute
out[b,y,x,o] = b[o] + sum_{dy,dx,i} in[b, y+dy-1, x+dx-1, i] W[o,dy,dx,i].

``bf16=True`` rounds the input, the weights and every stored activation to bfloat16 (round to
nearest even), as the GPU network stores them, while all arithmetic stays FP64.
"""
from __future__ import annotations

import numpy as np

SPEC = [  # (Cin, Cout, kernel)
    (2, 12, 3), (12, 12, 3),        # level 0 encoder
    (12, 24, 3), (24, 24, 3),       # level 1
    (24, 48, 3), (48, 48, 3),       # level 2
    (48, 96, 3), (96, 96, 3),       # level 3 (bottom)
    (96 + 48, 48, 3), (48, 48, 3),  # level 2 decoder
    (48 + 24, 24, 3), (24, 24, 3),  # level 1 decoder
    (24 + 12, 12, 3), (12, 12, 3),  # level 0 decoder
    (12, 1, 1),                     # output
]


def num_params() -> int:
    return sum(co * k * k * ci + co for ci, co, k in SPEC)


def unpack(theta):
    out, o = [], 0
    for ci, co, k in SPEC:
        nw = co * k * k * ci
        W = theta[o:o + nw].reshape((co, k, k, ci) if k == 3 else (co, ci))
        o += nw
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    return out


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    x = np.asarray(a, dtype=np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, W, b):
    B, H, Wd, C = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1, :] = x
    out = np.broadcast_to(b, (B, H, Wd, W.shape[0])).copy()
    for dy in range(3):
        for dx in range(3):
            out += xp[:, dy:dy + H, dx:dx + Wd, :] @ W[:, dy, dx, :].T
    return out


def conv3x3_backward(x, W, dout):
    """Gradients of sum(dout * conv3x3(x, W, b)) with respect to x, W and b."""
    B, H, Wd, C = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1, :] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + H, dx:dx + Wd, :]
            dW[:, dy, dx, :] = np.einsum("bhwo,bhwi->oi", dout, patch)
            dxp[:, dy:dy + H, dx:dx + Wd, :] += dout @ W[:, dy, dx, :]
    return dxp[:, 1:-1, 1:-1, :], dW, dout.sum(axis=(0, 1, 2))


def avgpool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(dout):
    return np.repeat(np.repeat(dout, 2, axis=1), 2, axis=2) * 0.25


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(dout):
    B, H, W, C = dout.shape
    return dout.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(theta, x, bf16=False):
    """Network output (B, H, W) for input x (B, H, W, 2); also returns the activation cache."""
    rnd = bf16_round if bf16 else (lambda a: a)
    P = [(rnd(W), b) for W, b in unpack(np.asarray(theta, dtype=np.float64))]
    cache = {"P": P}
    h = rnd(x)
    cache["in"] = h

    def cr(name, layer, inp):
        W, b = P[layer]
        a = rnd(np.maximum(conv3x3(inp, W, b), 0.0))
        cache[name] = a
        return a

    a0 = cr("a0", 0, h); s0 = cr("s0", 1, a0)
    p0 = rnd(avgpool2(s0)); cache["p0"] = p0
    a1 = cr("a1", 2, p0); s1 = cr("s1", 3, a1)
    p1 = rnd(avgpool2(s1)); cache["p1"] = p1
    a2 = cr("a2", 4, p1); s2 = cr("s2", 5, a2)
    p2 = rnd(avgpool2(s2)); cache["p2"] = p2
    a3 = cr("a3", 6, p2); b3 = cr("b3", 7, a3)
    k2 = np.concatenate([upsample2(b3), s2], axis=3); cache["k2"] = k2
    e2 = cr("e2", 8, k2); d2 = cr("d2", 9, e2)
    k1 = np.concatenate([upsample2(d2), s1], axis=3); cache["k1"] = k1
    e1 = cr("e1", 10, k1); d1 = cr("d1", 11, e1)
    k0 = np.concatenate([upsample2(d1), s0], axis=3); cache["k0"] = k0
    e0 = cr("e0", 12, k0); d0 = cr("d0", 13, e0)
    W, b = P[14]
    out = d0 @ W[0] + b[0]
    return out, cache


def backward(theta, x, dout, bf16=False):
    """Gradient of sum(dout * forward(theta, x)) with respect to theta (flat, FP64)."""
    _, c = forward(theta, x, bf16)
    P = c["P"]
    grads = [None] * len(SPEC)

    def layer_back(layer, inp, post, dpost):
        dpre = dpost * (post > 0)
        dx, dW, db = conv3x3_backward(inp, P[layer][0], dpre)
        grads[layer] = (dW, db)
        return dx

    W, b = P[14]
    grads[14] = (np.einsum("bhw,bhwc->c", dout, c["d0"])[None, :], np.array([dout.sum()]))
    dd0 = dout[..., None] * W[0]
    de0 = layer_back(13, c["e0"], c["d0"], dd0)
    dk0 = layer_back(12, c["k0"], c["e0"], de0)
    dd1 = upsample2_backward(dk0[..., :24]); ds0 = dk0[..., 24:]
    de1 = layer_back(11, c["e1"], c["d1"], dd1)
    dk1 = layer_back(10, c["k1"], c["e1"], de1)
    dd2 = upsample2_backward(dk1[..., :48]); ds1 = dk1[..., 48:]
    de2 = layer_back(9, c["e2"], c["d2"], dd2)
    dk2 = layer_back(8, c["k2"], c["e2"], de2)
    db3 = upsample2_backward(dk2[..., :96]); ds2 = dk2[..., 96:]
    da3 = layer_back(7, c["a3"], c["b3"], db3)
    dp2 = layer_back(6, c["p2"], c["a3"], da3)
    ds2 = ds2 + avgpool2_backward(dp2)
    da2 = layer_back(5, c["a2"], c["s2"], ds2)
    dp1 = layer_back(4, c["p1"], c["a2"], da2)
    ds1 = ds1 + avgpool2_backward(dp1)
    da1 = layer_back(3, c["a1"], c["s1"], ds1)
    dp0 = layer_back(2, c["p0"], c["a1"], da1)
    ds0 = ds0 + avgpool2_backward(dp0)
    da0 = layer_back(1, c["a0"], c["s0"], ds0)
    layer_back(0, c["in"], c["a0"], da0)
    flat = []
    for (dW, db) in grads:
        flat.append(dW.reshape(-1))
        flat.append(db.reshape(-1))
    return np.concatenate(flat)


def features(f, n):
    """The network input for a right-hand side f (N,): [f / rms f, lap(f) / rms(lap f)], where
    lap is the 5-point stencil 4 f - (4 neighbours) with replicated boundary values."""
    F = f.reshape(n, n)
    Fp = np.pad(F, 1, mode="edge")
    lap = 4 * F - Fp[:-2, 1:-1] - Fp[2:, 1:-1] - Fp[1:-1, :-2] - Fp[1:-1, 2:]
    rf = np.sqrt(np.mean(F * F))
    rl = np.sqrt(np.mean(lap * lap))
    return np.stack([F / rf, lap / rl], axis=-1)[None], rl

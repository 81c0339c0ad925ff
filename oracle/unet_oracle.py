"""FP64 CPU oracle of the warm-start U-Net surrogate (forward, backward, loss, Adam).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are its only callers. It shares no code with the CUDA library.

The network (a convolutional U-Net in the sense of Ronneberger, Fischer and Brox,
MICCAI 2015) maps a packed-emulsion channel, resampled to an H x W image (H across the
channel, W along the flow), to its relaxed state. Layout is NHWC: x[b, y, x, c].

* levels L (default 4) with widths C_l = base * 2**l (base 32: 32, 64, 128, 256);
* encoder level l < L-1: conv3x3 -> ReLU -> conv3x3 -> ReLU (= skip_l), then 2x2 max pool;
* bottom level: conv3x3 -> ReLU -> conv3x3 -> ReLU;
* decoder level l (from L-2 down to 0): nearest 2x upsampling, conv3x3 to C_l -> ReLU,
  concatenation [upconv output, skip_l], conv3x3 -> ReLU -> conv3x3 -> ReLU;
* head: 1x1 convolution to the output channels, no activation.

Padding of every 3x3 convolution: zeros beyond the first and last row (the channel walls),
periodic along x (the channel is periodic in the flow direction). Max-pool ties go to
the first element of the window in the order (0,0), (0,1), (1,0), (1,1).

Loss: L = (1/P) sum_p sum_j lam_j (y_pj - t_pj)^2, P = number of pixels (B H W).
Adam (Kingma and Ba, 2015, Algorithm 1) with bias correction.

Parameters are a list of (weight, bias) pairs in layer order: enc_0a, enc_0b, ...,
enc_{L-1}a, enc_{L-1}b (the bottom), then for l = L-2 .. 0: up_l, dec_la, dec_lb, then the
head. A 3x3 weight is [C_out, 3, 3, C_in] (taps (dy, dx) from -1 to +1); the head is
[C_out, C_in].

``emulate_bf16``: round, to bfloat16 (round to nearest even from FP32), every value the
GPU path stores in bfloat16 -- inputs, weights, every activation and every activation
gradient -- so that the remaining differences are those of FP32 versus FP64 accumulation.

Parity status: every function is pinned in tests/test_unet_oracle.py (scipy correlation,
central finite differences of the loss, closed forms, shift equivariance).
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------- bfloat16


def bf16(a) -> np.ndarray:
    """Round to bfloat16 (returned as float64): convert to FP32 (nearest), then keep the
    upper 16 bits of the FP32 pattern, rounding to nearest, ties to even."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _q(a, emulate):
    return bf16(a) if emulate else a

# ---------------------------------------------------------------------------- network spec


def layer_shapes(levels=4, base=32, in_ch=5, out_ch=3):
    """[(name, weight_shape)] in parameter order; each layer also has a bias [C_out]."""
    C = [base * 2 ** l for l in range(levels)]
    out = []
    cin = in_ch
    for l in range(levels):
        out.append((f"enc{l}a", (C[l], 3, 3, cin)))
        out.append((f"enc{l}b", (C[l], 3, 3, C[l])))
        cin = C[l]
    for l in range(levels - 2, -1, -1):
        out.append((f"up{l}", (C[l], 3, 3, C[l + 1])))
        out.append((f"dec{l}a", (C[l], 3, 3, 2 * C[l])))
        out.append((f"dec{l}b", (C[l], 3, 3, C[l])))
    out.append(("head", (out_ch, C[0])))
    return out

# ---------------------------------------------------------------------------- operators


def pad_same(x):
    """[B, H, W, C] -> [B, H+2, W+2, C]: zero rows above and below, periodic columns."""
    xp = np.concatenate([x[:, :, -1:, :], x, x[:, :, :1, :]], axis=2)
    z = np.zeros_like(xp[:, :1])
    return np.concatenate([z, xp, z], axis=1)


def conv3x3(x, w, b):
    """y[b,y,x,o] = b[o] + sum_{dy,dx,c} w[o,dy+1,dx+1,c] xpad[b,y+dy,x+dx,c]."""
    B, H, W, _ = x.shape
    xp = pad_same(x)
    y = np.zeros((B, H, W, w.shape[0])) + b
    for ty in range(3):
        for tx in range(3):
            y += xp[:, ty:ty + H, tx:tx + W, :] @ w[:, ty, tx, :].T
    return y


def conv3x3_bwd(x, w, dy):
    """Gradients of conv3x3 given dL/dy: returns (dx, dw, db)."""
    B, H, W, _ = x.shape
    xp = pad_same(x)
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    dyf = dy.reshape(-1, dy.shape[-1])
    for ty in range(3):
        for tx in range(3):
            patch = xp[:, ty:ty + H, tx:tx + W, :]
            dw[:, ty, tx, :] = dyf.T @ patch.reshape(-1, patch.shape[-1])
            dxp[:, ty:ty + H, tx:tx + W, :] += dy @ w[:, ty, tx, :]
    # fold the padding back: rows beyond the walls are constants, columns wrap around
    dx = dxp[:, 1:H + 1, 1:W + 1, :].copy()
    dx[:, :, -1, :] += dxp[:, 1:H + 1, 0, :]
    dx[:, :, 0, :] += dxp[:, 1:H + 1, W + 1, :]
    db = dyf.sum(axis=0)
    return dx, dw, db


def conv1x1(x, w, b):
    return x @ w.T + b


def conv1x1_bwd(x, w, dy):
    dyf = dy.reshape(-1, dy.shape[-1])
    return dy @ w, dyf.T @ x.reshape(-1, x.shape[-1]), dyf.sum(axis=0)


def relu(x):
    return np.maximum(x, 0.0)


def relu_bwd(y, dy):
    """dL/d(pre-activation) from the ReLU output y and dL/dy."""
    return np.where(y > 0, dy, 0.0)


def maxpool2(x):
    """2x2 max pool; also returns the argmax (0..3, first maximum in window order)."""
    B, H, W, C = x.shape
    win = x.reshape(B, H // 2, 2, W // 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H // 2, W // 2, 4, C)
    arg = np.argmax(win, axis=3)  # numpy returns the first occurrence of the maximum
    return np.take_along_axis(win, arg[:, :, :, None, :], axis=3)[:, :, :, 0, :], arg


def maxpool2_bwd(arg, dy):
    B, h, w, C = dy.shape
    win = np.zeros((B, h, w, 4, C))
    np.put_along_axis(win, arg[:, :, :, None, :], dy[:, :, :, None, :], axis=3)
    return win.reshape(B, h, w, 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, 2 * h, 2 * w, C)


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_bwd(dy):
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def mse(y, t, lam=None):
    """L = (1/P) sum lam_j (y - t)^2 and dL/dy."""
    lam = np.ones(y.shape[-1]) if lam is None else np.asarray(lam, dtype=np.float64)
    P = y.size // y.shape[-1]
    d = y - t
    return float((lam * d * d).sum() / P), 2.0 * lam * d / P


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t >= 1 is the step number after this update); returns new copies."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v

# ---------------------------------------------------------------------------- the U-Net


def forward(params, x, levels=4, emulate_bf16=False):
    """Returns (y, cache). params: list of (w, b) in layer_shapes order."""
    e = emulate_bf16
    q = lambda a: _q(a, e)  # noqa: E731
    P = [(q(w), b) for w, b in params]
    cache = {"x": q(x)}
    h = cache["x"]
    k = 0
    skips, args = [], []
    for l in range(levels):
        a = q(relu(conv3x3(h, *P[k])))
        cache[f"enc{l}a_in"], cache[f"enc{l}a"] = h, a
        s = q(relu(conv3x3(a, *P[k + 1])))
        cache[f"enc{l}b"] = s
        k += 2
        if l < levels - 1:
            skips.append(s)
            h, arg = maxpool2(s)
            args.append(arg)
        else:
            h = s
    cache["args"] = args
    for l in range(levels - 2, -1, -1):
        u = upsample2(h)
        cache[f"up{l}_in"] = u
        uo = q(relu(conv3x3(u, *P[k])))
        cat = np.concatenate([uo, skips[l]], axis=-1)
        cache[f"up{l}"], cache[f"cat{l}"] = uo, cat
        a = q(relu(conv3x3(cat, *P[k + 1])))
        b = q(relu(conv3x3(a, *P[k + 2])))
        cache[f"dec{l}a"], cache[f"dec{l}b"] = a, b
        h = b
        k += 3
    y = conv1x1(h, *P[k])
    cache["head_in"] = h
    cache["P"] = P
    return y, cache


def backward(params, cache, dy, levels=4, emulate_bf16=False):
    """Gradients of the loss for every (w, b), given dL/dy of the head output."""
    q = lambda a: _q(a, emulate_bf16)  # noqa: E731
    P = cache["P"]
    grads = [None] * len(params)
    k = len(params) - 1
    dh, dw, db = conv1x1_bwd(cache["head_in"], P[k][0], dy)
    grads[k] = (dw, db)
    dh = q(dh)
    dskip = {}
    # decoder, finest level first: level l owns parameters k, k+1, k+2 = up_l, dec_la, dec_lb
    for l in range(0, levels - 1):
        k -= 3
        g = relu_bwd(cache[f"dec{l}b"], dh)
        da, dw, db = conv3x3_bwd(cache[f"dec{l}a"], P[k + 2][0], g)
        grads[k + 2] = (dw, db)
        g = relu_bwd(cache[f"dec{l}a"], q(da))
        dcat, dw, db = conv3x3_bwd(cache[f"cat{l}"], P[k + 1][0], g)
        grads[k + 1] = (dw, db)
        dcat = q(dcat)
        C = cache[f"up{l}"].shape[-1]
        dskip[l] = dcat[..., C:]
        g = relu_bwd(cache[f"up{l}"], dcat[..., :C])
        du, dw, db = conv3x3_bwd(cache[f"up{l}_in"], P[k][0], g)
        grads[k] = (dw, db)
        dh = q(upsample2_bwd(q(du)))
    # encoder, coarsest level first: level l owns parameters 2l, 2l+1
    for l in range(levels - 1, -1, -1):
        k = 2 * l
        if l < levels - 1:
            dh = q(dskip[l] + maxpool2_bwd(cache["args"][l], dh))
        g = relu_bwd(cache[f"enc{l}b"], dh)
        da, dw, db = conv3x3_bwd(cache[f"enc{l}a"], P[k + 1][0], g)
        grads[k + 1] = (dw, db)
        g = relu_bwd(cache[f"enc{l}a"], q(da))
        dx, dw, db = conv3x3_bwd(cache[f"enc{l}a_in"], P[k][0], g)
        grads[k] = (dw, db)
        dh = q(dx)
    return grads


def loss_and_grads(params, x, t, levels=4, lam=None, emulate_bf16=False):
    y, cache = forward(params, x, levels, emulate_bf16)
    L, dy = mse(y, t, lam)
    return L, backward(params, cache, dy, levels, emulate_bf16), y

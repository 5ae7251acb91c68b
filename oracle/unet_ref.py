"""FP64 reference of the EPID-image denoiser (the learned denoiser the paper names as future work, Sec. 5).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py``; the CUDA product path never imports it, and it
shares no code with the CUDA library.

The paper names a learned denoiser only as future work (Sec. 5); the network
is a stated reading: a 2D U-Net with four levels of 32, 64, 128 and 256
channels.  Encoder level l: two 3x3 convolutions (zero padding 1) with bias
and ReLU; 2x2 max pooling between levels.  Decoder level l (l = 2, 1, 0):
nearest-neighbour 2x upsampling of the level below, concatenated with the
encoder output of level l (upsampled channels first), then two 3x3
convolutions with ReLU.  Output: a 1x1 convolution to one channel, linear.
Loss: mean squared error over all pixels.  Optimiser: Adam (Kingma and Ba,
ICLR 2015, Algorithm 1) with bias correction.

Everything is written from the definitions: a convolution is the sum over
taps and input channels; its backward pass is the same sums taken with
respect to the input, the weights and the bias.  Tensors are NHWC;
weights [Co][k][k][Ci].  ``emulate_bf16`` rounds, to bfloat16 (round to
nearest even), exactly the tensors the GPU stores in bfloat16: the network
input, the weights, every layer output, the output gradient and every
propagated gradient; weight and bias gradients stay unrounded (the GPU keeps
them in float32).

Pins (tests/test_unet_oracle.py): the convolution against brute-force loops
and scipy's 2D correlation; every backward function and the whole network's
gradient against central finite differences; max pooling and upsampling
against loops; Adam against its closed form after one step; bf16 rounding
against torch's CPU conversion.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


# ----------------------------------------------------------- rounding ----

def bf16_round(a):
    """Round to bfloat16 (via float32, round to nearest even), returned as float64."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


# ------------------------------------------------------------ layers -----

def conv2d(x, w, b):
    """y[n,i,j,o] = b[o] + sum_{dy,dx,c} x[n, i+dy-p, j+dx-p, c] w[o,dy,dx,c], zero outside, p = k // 2."""
    N, H, W, Ci = x.shape
    Co, k, _, _ = w.shape
    p = k // 2
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    y = np.zeros((N, H, W, Co))
    for dy in range(k):
        for dx in range(k):
            y += np.einsum("nhwc,oc->nhwo", xp[:, dy:dy + H, dx:dx + W, :], w[:, dy, dx, :])
    return y + b


def conv2d_backward(x, w, dy):
    """Gradients of conv2d with respect to x, w and b, given dL/dy."""
    N, H, W, Ci = x.shape
    Co, k, _, _ = w.shape
    p = k // 2
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w, dtype=np.float64)
    for ky in range(k):
        for kx in range(k):
            dxp[:, ky:ky + H, kx:kx + W, :] += np.einsum("nhwo,oc->nhwc", dy, w[:, ky, kx, :])
            dw[:, ky, kx, :] = np.einsum("nhwo,nhwc->oc", dy, xp[:, ky:ky + H, kx:kx + W, :])
    dx = dxp[:, p:p + H, p:p + W, :]
    db = dy.sum(axis=(0, 1, 2))
    return dx, dw, db


def relu(z):
    return np.maximum(z, 0.0)


def relu_backward(y, dy):
    """dL/dz for y = relu(z), from the output y (y > 0 exactly where z > 0)."""
    return np.where(y > 0.0, dy, 0.0)


def maxpool2(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).max(axis=(2, 4))


def maxpool2_backward(x, dy):
    """Routes each gradient to the first maximum of its 2x2 window in the
    order (0,0), (0,1), (1,0), (1,1)."""
    N, H, W, C = x.shape
    win = x.reshape(N, H // 2, 2, W // 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(N, H // 2, W // 2, 4, C)
    first = np.argmax(win, axis=3)                       # argmax returns the first maximum
    dx = np.zeros((N, H // 2, W // 2, 4, C))
    np.put_along_axis(dx, first[:, :, :, None, :], dy[:, :, :, None, :], axis=3)
    return dx.reshape(N, H // 2, W // 2, 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(N, H, W, C)


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def upsample2_backward(dy):
    N, H, W, C = dy.shape
    return dy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def mse(yhat, t):
    """Mean squared error over every element and its gradient."""
    d = yhat - t
    return float(np.mean(d * d)), 2.0 * d / d.size


# ------------------------------------------------------------ network ----

@dataclass(frozen=True)
class UNetSpec:
    levels: int = 4
    c0: int = 32
    cin: int = 1

    def channels(self, l):
        return self.c0 << l


def layers(spec: UNetSpec):
    """The convolutions in parameter order: (name, Co, k, Ci)."""
    out = []
    ci = spec.cin
    for l in range(spec.levels):
        c = spec.channels(l)
        out += [(f"enc{l}a", c, 3, ci), (f"enc{l}b", c, 3, c)]
        ci = c
    for l in range(spec.levels - 2, -1, -1):
        c = spec.channels(l)
        out += [(f"dec{l}a", c, 3, spec.channels(l + 1) + c), (f"dec{l}b", c, 3, c)]
    out.append(("out", 1, 1, spec.c0))
    return out


def param_count(spec: UNetSpec) -> int:
    return sum(co * k * k * ci + co for _, co, k, ci in layers(spec))


def unpack(spec: UNetSpec, flat):
    """Flat parameter vector -> {name: (w [Co][k][k][Ci], b [Co])}: per layer
    the weights in that order, then the biases."""
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == param_count(spec)
    out, o = {}, 0
    for name, co, k, ci in layers(spec):
        nw = co * k * k * ci
        out[name] = (flat[o:o + nw].reshape(co, k, k, ci), flat[o + nw:o + nw + co])
        o += nw + co
    return out


def pack(spec: UNetSpec, d):
    return np.concatenate([np.concatenate([d[n][0].ravel(), d[n][1].ravel()]) for n, _, _, _ in layers(spec)])


def forward(spec: UNetSpec, flat, x, emulate_bf16=False):
    """Network output [N,H,W,1] and the cache the backward pass needs."""
    q = bf16_round if emulate_bf16 else (lambda a: a)
    P = unpack(spec, flat)
    Pq = {n: (q(w), b) for n, (w, b) in P.items()}
    cache = {"x": q(np.asarray(x, dtype=np.float64))}
    h = cache["x"]
    skips = []
    for l in range(spec.levels):
        if l > 0:
            h = maxpool2(h)
            cache[f"pool{l}"] = h
        for s in "ab":
            cache[f"in_enc{l}{s}"] = h
            h = q(relu(conv2d(h, *Pq[f"enc{l}{s}"])))
            cache[f"enc{l}{s}"] = h
        skips.append(h)
    for l in range(spec.levels - 2, -1, -1):
        u = upsample2(h)
        h = np.concatenate([u, skips[l]], axis=3)
        for s in "ab":
            cache[f"in_dec{l}{s}"] = h
            h = q(relu(conv2d(h, *Pq[f"dec{l}{s}"])))
            cache[f"dec{l}{s}"] = h
    cache["in_out"] = h
    y = q(conv2d(h, *Pq["out"]))
    cache["Pq"] = Pq
    return y, cache


def backward(spec: UNetSpec, cache, dy, emulate_bf16=False):
    """Flat gradient of the loss given dL/d(output)."""
    q = bf16_round if emulate_bf16 else (lambda a: a)
    Pq = cache["Pq"]
    grads = {}
    g = q(dy)
    dh, dw, db = conv2d_backward(cache["in_out"], Pq["out"][0], g)
    grads["out"] = (dw, db)
    dskip = [None] * spec.levels
    # decoder, from the top (level 0) down to level levels-2
    for l in range(0, spec.levels - 1):
        for s in "ba":
            dz = relu_backward(cache[f"dec{l}{s}"], q(dh))
            dh, dw, db = conv2d_backward(cache[f"in_dec{l}{s}"], Pq[f"dec{l}{s}"][0], dz)
            grads[f"dec{l}{s}"] = (dw, db)
        cu = spec.channels(l + 1)
        du, dskip[l] = q(dh[..., :cu]), q(dh[..., cu:])
        dh = q(upsample2_backward(du))
    # encoder, from the bottleneck up
    for l in range(spec.levels - 1, -1, -1):
        if l < spec.levels - 1:
            dh = dh + dskip[l]
        for s in "ba":
            dz = relu_backward(cache[f"enc{l}{s}"], q(dh))
            dh, dw, db = conv2d_backward(cache[f"in_enc{l}{s}"], Pq[f"enc{l}{s}"][0], dz)
            grads[f"enc{l}{s}"] = (dw, db)
        if l > 0:
            dh = maxpool2_backward(cache[f"enc{l - 1}b"], q(dh))
    return pack(spec, grads)


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Algorithm 1 of Kingma and Ba), step number t >= 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train_step(spec: UNetSpec, flat, x, target, state, lr, emulate_bf16=False):
    """Forward, MSE loss, backward and one Adam step; state = (m, v, t)."""
    y, cache = forward(spec, flat, x, emulate_bf16)
    loss, dy = mse(y, target)
    g = backward(spec, cache, dy, emulate_bf16)
    m, v, t = state
    p, m, v = adam_step(np.asarray(flat, dtype=np.float64), g, m, v, t + 1, lr)
    return p, (m, v, t + 1), loss, g

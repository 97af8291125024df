"""Plain FP64 numpy reference of the warm-start surrogate network.

TEST INFRASTRUCTURE ONLY: the tests use it to check the CUDA training and
inference kernels; the product path never imports it.

The network is a stack of 3D convolutions (layout [batch][channel][D][H][W],
"same" zero padding, odd kernels, per-layer dilation) with tanh between
layers and a linear last layer, trained on the mean squared error.  Every
function below is the definition written out with numpy loops over kernel
taps; nothing is fused or reordered.
"""
from __future__ import annotations

import numpy as np


def conv3d(x, w, b, dil):
    """y[n,o,d,h,v] = b[o] + sum_{i,a,c,e} w[o,i,a,c,e] * x[n,i,d+da,h+dc,v+de], zero outside,
    with da = dil[0]*(a - (KD-1)/2) etc."""
    N, Ci, D, H, V = x.shape
    Co, Ci2, KD, KH, KW = w.shape
    assert Ci == Ci2
    y = np.zeros((N, Co, D, H, V))
    y += b[None, :, None, None, None]
    for a in range(KD):
        for c in range(KH):
            for e in range(KW):
                sd = dil[0] * (a - (KD - 1) // 2)
                sh = dil[1] * (c - (KH - 1) // 2)
                sw = dil[2] * (e - (KW - 1) // 2)
                xs = shift(x, sd, sh, sw)
                y += np.einsum("oi,nidhv->nodhv", w[:, :, a, c, e], xs)
    return y


def shift(x, sd, sh, sw):
    """xs[..., d, h, v] = x[..., d+sd, h+sh, v+sw], zero where out of range."""
    out = np.zeros_like(x)
    D, H, V = x.shape[2:]

    def rng(n, s):
        lo, hi = max(0, -s), min(n, n - s)
        return lo, hi

    d0, d1 = rng(D, sd)
    h0, h1 = rng(H, sh)
    v0, v1 = rng(V, sw)
    if d0 < d1 and h0 < h1 and v0 < v1:
        out[:, :, d0:d1, h0:h1, v0:v1] = x[:, :, d0 + sd:d1 + sd, h0 + sh:h1 + sh, v0 + sw:v1 + sw]
    return out


def conv3d_backward(x, w, dil, gy):
    """Gradients of sum(gy * conv3d(x, w, b, dil)) with respect to x, w, b."""
    Co, Ci, KD, KH, KW = w.shape
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    gb = gy.sum(axis=(0, 2, 3, 4))
    for a in range(KD):
        for c in range(KH):
            for e in range(KW):
                sd = dil[0] * (a - (KD - 1) // 2)
                sh = dil[1] * (c - (KH - 1) // 2)
                sw = dil[2] * (e - (KW - 1) // 2)
                xs = shift(x, sd, sh, sw)
                gw[:, :, a, c, e] = np.einsum("nodhv,nidhv->oi", gy, xs)
                # x[d+sd] contributed w * gy[d]  ->  gx[d'] += w * gy[d' - sd]
                gx += shift(np.einsum("oi,nodhv->nidhv", w[:, :, a, c, e], gy), -sd, -sh, -sw)
    return gx, gw, gb


class Net:
    """layers: list of (Cin, Cout, (KD, KH, KW), (dD, dH, dW), act) with act in {"tanh", None}."""

    def __init__(self, layers, params):
        self.layers = layers
        self.params = params  # list of (w, b) float64

    def forward(self, x):
        acts = [x]
        h = x
        for (ci, co, k, dil, act), (w, b) in zip(self.layers, self.params):
            z = conv3d(h, w, b, dil)
            h = np.tanh(z) if act == "tanh" else z
            acts.append(h)
        return h, acts

    def loss_and_grads(self, x, target):
        """MSE = mean((y - target)^2) and its gradients, by backpropagation."""
        y, acts = self.forward(x)
        diff = y - target
        loss = float(np.mean(diff ** 2))
        g = 2.0 * diff / diff.size
        grads = [None] * len(self.layers)
        for li in range(len(self.layers) - 1, -1, -1):
            ci, co, k, dil, act = self.layers[li]
            if act == "tanh":
                g = g * (1.0 - acts[li + 1] ** 2)
            w, b = self.params[li]
            gx, gw, gb = conv3d_backward(acts[li], w, dil, g)
            grads[li] = (gw, gb)
            g = gx
        return loss, grads


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), in place; returns nothing."""
    m *= b1
    m += (1.0 - b1) * g
    v *= b2
    v += (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    p -= lr * mh / (np.sqrt(vh) + eps)

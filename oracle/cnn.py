"""FP64 CPU reference of the learned coarse-grid corrector's network.

Test infrastructure only (see ``oracle/__init__``). The paper has no learned
component; the corrector is an addition around its method. This module
states the network and its gradients plainly so that the GPU training
kernels can be checked against it:

* 3 x 3 convolution with zero padding ("same" size): for input x of shape
  (H, W, Cin), weights w of shape (3, 3, Cin, Cout) and bias b (Cout,),
  y[i, j, o] = b[o] + sum_{a, c, k} x[i + a - 1, j + c - 1, k] w[a, c, k, o];
* ReLU after layers 1 .. L-1, none after the last; residual output
  out = x + net(x) (the network predicts a correction);
* loss = mean over pixels and channels of (out - target)^2;
* restriction of a fine field to a grid r times coarser: the mean over each
  r x r block of the conserved variables (rho, j_x, j_y, e), then
  (rho, u, v, T) with T = e/rho - |u|^2/2 (the scheme's gas, R = 1);
* features of a state: (log rho, u, v, log T).
"""
import numpy as np


def conv3x3(x, w, b):
    H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (H, W, w.shape[3])).astype(np.float64).copy()
    for a in range(3):
        for c in range(3):
            y += np.tensordot(xp[a:a + H, c:c + W, :], w[a, c], axes=(2, 0))
    return y


def conv3x3_backward(x, w, dy):
    """Gradients (dx, dw, db) of sum(dy * conv3x3(x, w, b))."""
    H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for a in range(3):
        for c in range(3):
            dw[a, c] = np.tensordot(xp[a:a + H, c:c + W, :], dy, axes=((0, 1), (0, 1)))
            dxp[a:a + H, c:c + W, :] += np.tensordot(dy, w[a, c], axes=(2, 1))
    return dxp[1:-1, 1:-1, :], dw, dy.sum(axis=(0, 1))


def bf16(a):
    """Rounds to the nearest bfloat16 (8 significant bits), ties to even:
    keep the upper 16 bits of the IEEE single, adding half an ulp of the
    kept part (0x7FFF plus the lowest kept bit) first. Finite inputs only."""
    a = np.asarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def forward(x, params, x_res=None, store=None, scale=None):
    """params: list of (w, b). Returns (out, cache); out = x_res + scale *
    net(x) with x_res = x unless given (the network may see a rounded copy of
    the features while the residual adds the unrounded ones) and scale a
    per-channel factor (default 1): the network predicts the correction in
    units of ``scale``."""
    store = store or (lambda a: a)
    scale = np.ones(x.shape[-1]) if scale is None else np.asarray(scale, dtype=np.float64)
    acts = [x]
    pres = []
    h = x
    L = len(params)
    for l, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        pres.append(z)
        h = store(np.maximum(z, 0.0)) if l < L - 1 else z
        acts.append(h)
    return (x if x_res is None else x_res) + scale * h, (acts, pres)


def loss_and_grads(x, target, params, x_res=None, store=None, scale=None, loss="mse"):
    """Loss and per-layer (dw, db). ``store`` (default: identity) is applied
    wherever a mixed-precision pipeline stores a value: the hidden
    activations and the gradient flowing into each layer's output. ``loss``:
    "mse" (mean of (out - target)^2) or "l1" (mean of |out - target|, with
    the subgradient sign(out - target), 0 where they are equal)."""
    out, (acts, pres) = forward(x, params, x_res, store, scale)
    store = store or (lambda a: a)
    scale = np.ones(x.shape[-1]) if scale is None else np.asarray(scale, dtype=np.float64)
    n = out.size
    d = out - target
    if loss == "l1":
        value = float(np.abs(d).sum() / n)
        g = store(scale * np.sign(d) / n)    # d loss / d net (chain rule through scale)
    else:
        value = float((d ** 2).sum() / n)
        g = store(2.0 * scale * d / n)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        if l < len(params) - 1:
            g = store(g * (pres[l] > 0.0))
        dx, dw, db = conv3x3_backward(acts[l], w, g)
        grads[l] = (dw, db)
        g = dx
    return value, grads


def restrict(rho, u, v, T, r):
    """Block means of the conserved variables over r x r blocks."""
    e = rho * T + 0.5 * rho * (u * u + v * v)
    H, W = rho.shape

    def blk(q):
        return q.reshape(H // r, r, W // r, r).mean(axis=(1, 3))
    R, JX, JY, E = blk(rho), blk(rho * u), blk(rho * v), blk(e)
    U, V = JX / R, JY / R
    return R, U, V, E / R - 0.5 * (U * U + V * V)


def features(rho, u, v, T):
    return np.stack([np.log(rho), u, v, np.log(T)], axis=-1)

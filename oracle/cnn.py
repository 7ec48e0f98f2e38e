"""FP64 CPU oracle of the per-patch refinement-flag predictor (test
infrastructure only; see oracle/__init__.py).

The network (a learned stand-in for the flag buffer of Sec. 3.2): input
planes of a level (C_in = 5 features per cell), three 3x3 convolutions with
16 channels and ReLU, and a 1x1 convolution to one logit per cell.  Zero
padding at the plane's edge ("same" size).  Loss: binary cross-entropy with
logits, averaged over the cells where mask = 1.  Optimiser: Adam.

Written with explicit loops over the 3x3 offsets (array slices), no im2col,
so each line can be checked against the definition of a cross-correlation:
    y[o, i, j] = b[o] + sum_c sum_{di,dj} w[o, c, di, dj] x[c, i+di-1, j+dj-1].

Parameter layout (shared with the GPU library's flat weight vector):
  layer k (k = 0, 1, 2): W_k (C_out=16, C_in_k, 3, 3) then b_k (16),
  head: W_3 (1, 16) then b_3 (1); C_in_0 = 5, C_in_1 = C_in_2 = 16.
"""
from __future__ import annotations

import numpy as np

C_IN = 5
HID = 16
LAYERS = [(C_IN, HID, 3), (HID, HID, 3), (HID, HID, 3), (HID, 1, 1)]


def n_params() -> int:
    return sum(co * ci * k * k + co for ci, co, k in LAYERS)


def unpack(theta: np.ndarray):
    out, p = [], 0
    for ci, co, k in LAYERS:
        w = theta[p:p + co * ci * k * k].reshape(co, ci, k, k)
        p += co * ci * k * k
        b = theta[p:p + co]
        p += co
        out.append((w, b))
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for ci, co, k in LAYERS:
        fan = ci * k * k
        parts.append(rng.normal(0.0, np.sqrt(2.0 / fan), co * ci * k * k))
        parts.append(np.zeros(co))
    return np.concatenate(parts)


def conv(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x (N, C, H, W) -> (N, O, H, W), zero padding, stride 1."""
    n, c, h, wd = x.shape
    o, _, k, _ = w.shape
    r = k // 2
    xp = np.zeros((n, c, h + 2 * r, wd + 2 * r))
    xp[:, :, r:r + h, r:r + wd] = x
    y = np.zeros((n, o, h, wd)) + b[None, :, None, None]
    for di in range(k):
        for dj in range(k):
            patch = xp[:, :, di:di + h, dj:dj + wd]                 # (N, C, H, W)
            y += np.einsum("oc,nchw->nohw", w[:, :, di, dj], patch)
    return y


def forward(theta: np.ndarray, x: np.ndarray):
    """Returns logits (N, H, W) and the activations needed by backward."""
    acts = [x]
    a = x
    params = unpack(theta)
    for k, (w, b) in enumerate(params):
        z = conv(a, w, b)
        a = np.maximum(z, 0.0) if k < len(params) - 1 else z
        acts.append(a)
    return acts[-1][:, 0], acts


def bce_loss(logits: np.ndarray, target: np.ndarray, mask: np.ndarray) -> float:
    """mean over masked cells of log(1 + e^z) - t z (stable form)."""
    z = logits
    l = np.maximum(z, 0.0) - z * target + np.log1p(np.exp(-np.abs(z)))
    m = mask.sum()
    return float((l * mask).sum() / max(m, 1.0))


def backward(theta: np.ndarray, x: np.ndarray, target: np.ndarray, mask: np.ndarray):
    """Loss and its gradient with respect to the flat parameter vector."""
    logits, acts = forward(theta, x)
    loss = bce_loss(logits, target, mask)
    m = max(mask.sum(), 1.0)
    sig = 1.0 / (1.0 + np.exp(-logits))
    g = ((sig - target) * mask / m)[:, None]                       # dL/dz of the head (N, 1, H, W)
    params = unpack(theta)
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        w, b = params[k]
        a_in = acts[k]
        o, c, kk, _ = w.shape
        r = kk // 2
        n, _, h, wd = a_in.shape
        ap = np.zeros((n, c, h + 2 * r, wd + 2 * r))
        ap[:, :, r:r + h, r:r + wd] = a_in
        gw = np.zeros_like(w)
        for di in range(kk):
            for dj in range(kk):
                gw[:, :, di, dj] = np.einsum("nohw,nchw->oc", g, ap[:, :, di:di + h, dj:dj + wd])
        gb = g.sum(axis=(0, 2, 3))
        grads[k] = (gw, gb)
        if k > 0:
            # dL/da_in = correlation of g with the flipped kernel, then ReLU'
            gp = np.zeros((n, o, h + 2 * r, wd + 2 * r))
            gp[:, :, r:r + h, r:r + wd] = g
            ga = np.zeros((n, c, h, wd))
            for di in range(kk):
                for dj in range(kk):
                    ga += np.einsum("oc,nohw->nchw", w[:, :, kk - 1 - di, kk - 1 - dj], gp[:, :, di:di + h, dj:dj + wd])
            g = ga * (acts[k] > 0.0)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), t counted from 1."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(h, hu, hv, B, covered, flag, drytol=1e-3, eta_scale=0.1, depth_scale=1000.0, mom_scale=10.0):
    """Input planes of a level: (eta/eta_scale on wet cells, clipped depth
    -B/depth_scale, |hu|/mom_scale, |hv|/mom_scale, current criterion flag),
    zero where no patch covers the cell."""
    wet = (h >= drytol) & covered
    f = np.zeros((C_IN,) + h.shape)
    f[0] = np.where(wet, (h + B) / eta_scale, 0.0)
    f[1] = np.where(covered, np.clip(-B / depth_scale, -1.0, 5.0), 0.0)
    f[2] = np.where(covered, np.abs(hu) / mom_scale, 0.0)
    f[3] = np.where(covered, np.abs(hv) / mom_scale, 0.0)
    f[4] = np.where(covered, flag.astype(float), 0.0)
    return f

"""FP64 oracle of the learned initialisation (not part of the paper: a data-driven initial
object for Algorithm 1, built from the paper's forward model, Sec. 2 Eqs. exit_wave and
expected_count).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/`` and the CPU legs of
``bench.py`` use it, and it shares no code with the CUDA path.  Plain numpy in float64.

Pipeline, per diffraction pattern y_k (M = m x m pixels, orthonormal DFT F):
  1. physics input  e_k = F^-1( sqrt(y_k) . u ) . conj(P) / (|P|^2 + eps max|P|^2) with
     u = F(P) / max(|F(P)|, 1e-3 max|F(P)|) (the far-field magnitudes combined with the
     probe's own far-field phase, propagated back and divided by the probe: a rough object
     estimate inside the illuminated disk; u fades where F(P) nearly vanishes, whose phase
     single precision cannot resolve), as two channels (Re, Im);
  2. a 6-layer convolutional encoder-decoder maps it to the object patch (Re, Im);
  3. the patch estimates are averaged into one object with weights |P|^2 over the
     overlaps; pixels no probe covers keep 1.

Network (channels, spatial side for m = 128; 3 x 3 kernels, zero padding 1):
  L1 2 -> C1 stride 2 (128 -> 64), ReLU      L4 x2 nearest upsample, C3 -> C2 (16 -> 32), ReLU
  L2 C1 -> C2 stride 2 (64 -> 32), ReLU      L5 x2 upsample, C2 -> C1 (32 -> 64), ReLU
  L3 C2 -> C3 stride 2 (32 -> 16), ReLU      L6 x2 upsample, C1 -> 2 (64 -> 128), linear
Loss: mean over the probe support (|P| > 0) and both channels of (out - target)^2.
"""
from __future__ import annotations

import numpy as np

U_FLOOR = 1e-3   # F(P) / max(|F(P)|, U_FLOOR max|F(P)|): the phasor fades where F(P) nearly vanishes

# (c_in, c_out, stride, upsample, relu) per layer, from the widths (C1, C2, C3)
def layer_specs(widths=(32, 64, 128)):
    c1, c2, c3 = widths
    return [(2, c1, 2, False, True), (c1, c2, 2, False, True), (c2, c3, 2, False, True),
            (c3, c2, 1, True, True), (c2, c1, 1, True, True), (c1, 2, 1, True, False)]


def upsample2(x):
    """Nearest-neighbour x2 upsampling of [N, C, H, W]."""
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def conv3x3(x, W, b, stride=1, up=False):
    """out[n, o, i, j] = b[o] + sum_{c, u, v} W[o, c, u, v] xp[n, c, s i + u, s j + v] with xp
    the (upsampled) input zero-padded by 1; output side = input side / stride."""
    if up:
        x = upsample2(x)
    N, C, H, Wd = x.shape
    Ho, Wo = H // stride, Wd // stride
    xp = np.zeros((N, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((N, W.shape[0], Ho, Wo))
    for u in range(3):
        for v in range(3):
            patch = xp[:, :, u:u + stride * Ho:stride, v:v + stride * Wo:stride]   # [N, C, Ho, Wo]
            out += np.einsum("oc,nchw->nohw", W[:, :, u, v], patch)
    return out + b[None, :, None, None]


def conv3x3_backward(x, W, g, stride=1, up=False):
    """Gradients (dx, dW, db) of sum(g * conv3x3(x, W, b)) w.r.t. x (the layer's input,
    before any upsampling), W and b."""
    xu = upsample2(x) if up else x
    N, C, H, Wd = xu.shape
    Ho, Wo = g.shape[2], g.shape[3]
    xp = np.zeros((N, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = xu
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for u in range(3):
        for v in range(3):
            sl = (slice(None), slice(None), slice(u, u + stride * Ho, stride), slice(v, v + stride * Wo, stride))
            dW[:, :, u, v] = np.einsum("nohw,nchw->oc", g, xp[sl])
            dxp[sl] += np.einsum("oc,nohw->nchw", W[:, :, u, v], g)
    dxu = dxp[:, :, 1:-1, 1:-1]
    dx = dxu.reshape(N, C, H // 2, 2, Wd // 2, 2).sum(axis=(3, 5)) if up else dxu
    db = g.sum(axis=(0, 2, 3))
    return dx, dW, db


def init_params(widths=(32, 64, 128), seed=0):
    """He-normal weights (std sqrt(2 / (9 c_in))), zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for ci, co, _, _, _ in layer_specs(widths):
        params.append((rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci)), np.zeros(co)))
    return params


def net_forward(params, x, widths=(32, 64, 128)):
    """Activations [x, a1, ..., a6] (a6 = network output)."""
    acts = [x]
    for (W, b), (_, _, s, up, relu) in zip(params, layer_specs(widths)):
        z = conv3x3(acts[-1], W, b, s, up)
        acts.append(np.maximum(z, 0.0) if relu else z)
    return acts


def net_loss_and_grads(params, x, target, mask, widths=(32, 64, 128), relu_masks=None):
    """L = sum(mask * (out - target)^2) / (2 sum(mask)) over both channels and the batch
    (mask [H, W] broadcast), and dL/dW, dL/db per layer.  relu_masks: optional list of the
    five hidden layers' ReLU decisions (boolean arrays shaped like their outputs) to use in
    the backward pass instead of acts > 0 -- the decisions a lower-precision evaluation of
    the same network took (a pre-activation within its rounding of zero can fall on either
    side of the kink)."""
    acts = net_forward(params, x, widths)
    out = acts[-1]
    n_terms = 2.0 * x.shape[0] * float(mask.sum())
    r = (out - target) * mask[None, None]
    loss = float(np.sum(r * r) / n_terms)
    g = 2.0 * r / n_terms
    grads = [None] * len(params)
    specs = layer_specs(widths)
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        _, _, s, up, relu = specs[l]
        if relu:
            g = g * (relu_masks[l] if relu_masks is not None else (acts[l + 1] > 0.0))
        dx, dW, db = conv3x3_backward(acts[l], W, g, s, up)
        grads[l] = (dW, db)
        g = dx
    return loss, grads


def physics_input(y, P, eps=1e-3):
    """e_k of step 1 for y [K, m, m] (natural DFT order) and probe P [m, m]: [K, 2, m, m]."""
    FP = np.fft.fft2(P, norm="ortho")
    u = FP / np.maximum(np.abs(FP), U_FLOOR * np.abs(FP).max())
    e = np.fft.ifft2(np.sqrt(np.maximum(y, 0.0)) * u[None], norm="ortho")
    d = np.abs(P) ** 2 + eps * np.max(np.abs(P) ** 2)
    e = e * (np.conj(P) / d)[None]
    return np.stack([e.real, e.imag], axis=1)


def stitch(patches, positions, P, shape):
    """Overlap average of complex patch estimates [K, m, m] with weights |P|^2; 1 where no
    probe reaches."""
    num = np.zeros(shape, complex)
    den = np.zeros(shape)
    w = np.abs(P) ** 2
    m0, m1 = P.shape
    for (r, c), Q in zip(positions, patches):
        num[r:r + m0, c:c + m1] += w * Q
        den[r:r + m0, c:c + m1] += w
    out = np.ones(shape, complex)
    nz = den > 0
    out[nz] = num[nz] / den[nz]
    return out


def to_bf16(a):
    """Round float64 values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)

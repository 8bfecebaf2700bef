"""FP64 CPU oracle of the surrogate network (TEST INFRASTRUCTURE ONLY: imported by tests/ only).

Multilayer perceptron (E, omega, lambda, p_x, p_y, s) -> 4 x [256, GELU] -> (mu, log sigma^2),
Gaussian negative log-likelihood L = mean_b[(y'_b - mu_b)^2 exp(-l_b) + l_b]/2 on the
standardised target y' = (y - y0) ys, inputs standardised as x' = (x - shift) scale.

With ``bf16=True`` the GEMM operands are rounded to bfloat16 (round to nearest even) at the
same points as the GPU kernels (inputs, weights, hidden activations, dL/dz); every product and
sum is then carried out in FP64.  With ``bf16=False`` it is the plain FP64 network, pinned by
finite differences in tests/test_mlp_oracle.py.
"""
import numpy as np
from scipy.special import erf

DIN = (6, 256, 256, 256, 256)
DOUT = (256, 256, 256, 256, 2)


def n_params():
    return sum(i * o + o for i, o in zip(DIN, DOUT))


def unpack(params):
    """Per layer W [out][in] then b [out], in order."""
    out, off = [], 0
    for i, o in zip(DIN, DOUT):
        W = params[off:off + i * o].reshape(o, i)
        off += i * o
        b = params[off:off + o]
        off += o
        out.append((W, b))
    return out


def bf16(x):
    """Round to bfloat16 (nearest even) through float32, returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(params, x, norm, bf=True):
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack(np.asarray(params, dtype=np.float64))
    shift, scale = np.asarray(norm[:6], float), np.asarray(norm[6:12], float)
    a = r((np.asarray(x, float) - shift) * scale)
    acts, zs = [a], []
    for l, (W, b) in enumerate(layers):
        z = a @ r(W).T + b
        zs.append(z)
        if l < len(layers) - 1:
            a = r(gelu(z))
            acts.append(a)
    return zs[-1], acts, zs


def loss_and_grad(params, x, y, norm, bf=True):
    """Loss and gradient with respect to all parameters (same layout as params)."""
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack(np.asarray(params, dtype=np.float64))
    out, acts, zs = forward(params, x, norm, bf)
    B = out.shape[0]
    y0, ys = float(norm[12]), float(norm[13])
    mu, lv = out[:, 0], out[:, 1]
    res = (np.asarray(y, float) - y0) * ys - mu
    w = np.exp(-lv)
    loss = 0.5 * np.mean(res * res * w + lv)
    dz = np.stack([-res * w / B, 0.5 * (1.0 - res * res * w) / B], axis=1)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        gW = r(dz).T @ acts[l]
        gb = dz.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            dz = (r(dz) @ r(W)) * gelu_grad(zs[l - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat

"""Error model of the surrogate network's BF16 arithmetic against the plain FP64 network.

The tensor-core kernels round the GEMM operands to bfloat16 (inputs, weights, hidden activations
and, in the backward pass, dL/dz) and accumulate in FP32.  Worst-case (magnitude) bounds of such
a network grow with |W_1| ... |W_4| and overestimate the error by five orders of magnitude, so
the tolerance of the GPU tests comes from the first-order probabilistic model of rounding errors
(independent, zero-mean errors, as in Higham and Mary's probabilistic error analysis):

* rounding x to bfloat16 (8 significand bits, round to nearest) adds an error of variance at most
  u^2 x^2 / 3, u = 2^-8 (half an ulp of 1, ulp(1) = 2^-7; uniform within half an ulp);
* FP32 accumulation adds variance n (2^-24)^2 / 3 times the sum of the squared products, and the
  kernels' FP32 GELU an error below 1e-6 (|z| + sigma_z);
* errors propagate linearly (first order): through W (signed weights, variances summed with
  W^2), GELU' on the way forward, and GELU'' (for the backward pass's GELU'(z) at a perturbed z).

Forward, per row (a_0 = standardised input, z_l = W_l a_l + b_l, a_{l+1} = GELU(z_l)):
    var(a_0)     = u^2 a_0^2 / 3
    var(z_l)     = W_l^2 var(a_l) + (u^2/3) W_l^2 a_l^2 + n_l (2^-24)^2/3 W_l^2 a_l^2
    var(a_{l+1}) = GELU'(z_l)^2 var(z_l) + (u^2/3) GELU(z_l)^2
Backward (dz_4 = dL/dz_4 of the Gaussian NLL; dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1})):
    var(dz_4) from var(mu) and var(log sigma^2) through the loss's derivative,
    var(dz_{l-1}) = GELU'^2 [W^2 (var(dz_l) + (u^2/3) dz_l^2) + (u^2/3) dz_l^2 W^2]
                    + (dz_l W)^2 GELU''(z_{l-1})^2 var(z_{l-1}),
    var(dL/dW_l) = sum_b a^2 (var(dz) + (u^2/3) dz^2) + dz^2 var(a),
    var(dL/db_l) = sum_b var(dz).
The rounding of the weights is one perturbation shared by every row, so each variance is
carried in two parts, from per-row roundings and from the weights' rounding; over the batch the
first adds in variance and the second in standard deviation (fully correlated rows, the worst
case); the loss's weight part is exact to first order, (u^2/3) sum_theta (theta dL/dtheta)^2.
The variances are propagated per element (the diagonal of the covariance), and the tests
accept a deviation of up to K = 6 standard deviations.  tests/test_mlp_oracle.py checks the
model against the oracle's own bfloat16 arithmetic (bf=True): its deviations from the FP64
network stay within the model's 6 sigma.
"""
import numpy as np

from oracle import mlp_oracle as M

U2 = (2.0 ** -8) ** 2 / 3.0
E2 = (2.0 ** -24) ** 2 / 3.0
K = 6.0


def _gelu_second(z):
    phi = np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)
    return phi * (2.0 - z * z)


def forward_sigma(params, x, norm):
    """(out, (vz_a, vz_w), (va_a, va_w), zs, acts): the FP64 network's outputs [B][2] and, per
    layer, the model's variances of z_l and a_l, split into the part from per-row roundings
    (inputs, activations: independent across rows) and the part from the rounding of the
    weights (shared by every row)."""
    out, acts, zs = M.forward(params, x, norm, bf=False)
    layers = M.unpack(np.asarray(params, dtype=np.float64))
    va_a, va_w = [U2 * acts[0] ** 2], [np.zeros_like(acts[0])]
    vz_a, vz_w = [], []
    for l, (W, b) in enumerate(layers):
        W2 = W * W
        a2 = acts[l] ** 2
        vz_a.append(va_a[l] @ W2.T + W.shape[1] * E2 * (a2 @ W2.T) + E2 * b * b)
        vz_w.append(va_w[l] @ W2.T + U2 * (a2 @ W2.T))
        if l < len(layers) - 1:
            g = M.gelu(zs[l])
            gp2 = M.gelu_grad(zs[l]) ** 2
            sz = np.sqrt(vz_a[l] + vz_w[l])
            va_a.append(gp2 * vz_a[l] + U2 * g * g + (1e-6 * (np.abs(zs[l]) + sz)) ** 2)
            va_w.append(gp2 * vz_w[l])
    return out, (vz_a, vz_w), (va_a, va_w), zs, acts


def head_sigma(params, x, norm):
    """Outputs in the target's units (mu = mu'/ys + y0, log sigma^2 = l' - 2 ln ys) with the
    model's standard deviations of mu and log sigma^2 (per row).  For the two outputs the
    first-order variance is summed exactly over the rounding sites, sum_site (d out/d site)^2
    var(site), with the sensitivities from backpropagation: activations and inputs
    (d out/d a_l,j)^2 (u^2/3) a_l,j^2, weights (d out/d z_l,i)^2 a_l,j^2 (u^2/3) W_ij^2, FP32
    sums n_l (2^-24)^2/3 (d out/d z_l,i)^2 sum_j W_ij^2 a_l,j^2, and the FP32 GELU."""
    out, acts, zs = M.forward(params, x, norm, bf=False)
    layers = M.unpack(np.asarray(params, dtype=np.float64))
    B = out.shape[0]
    var = np.zeros((B, 2))
    for k in range(2):
        gz = np.zeros((B, 2))
        gz[:, k] = 1.0  # d out_k / d z_4
        for l in range(len(layers) - 1, -1, -1):
            W, b = layers[l]
            a2 = acts[l] ** 2
            W2 = W * W
            var[:, k] += U2 * np.sum(gz * gz * (a2 @ W2.T), axis=1)              # weights
            var[:, k] += W.shape[1] * E2 * np.sum(gz * gz * (a2 @ W2.T), axis=1)  # FP32 sums
            ga = gz @ W                                                          # d out_k / d a_l
            var[:, k] += U2 * np.sum(ga * ga * a2, axis=1)                       # rounding of a_l
            if l > 0:
                var[:, k] += np.sum((ga * 1e-6 * (np.abs(zs[l - 1]) + 1.0)) ** 2, axis=1)  # FP32 GELU
                gz = ga * M.gelu_grad(zs[l - 1])
    ys = float(norm[13])
    mu = out[:, 0] / ys + float(norm[12])
    lv = out[:, 1] - 2.0 * np.log(ys)
    return mu, lv, np.sqrt(var[:, 0]) / ys, np.sqrt(var[:, 1])


def loss_grad_sigma(params, x, y, norm):
    """(loss, grad, sigma_loss, sigma_grad): the FP64 loss and gradient (params' layout) and the
    model's standard deviations of their BF16 computation.  Per-row parts add in variance over
    the batch; the weight-rounding parts, shared by all rows, add in standard deviation (fully
    correlated, the worst case)."""
    layers = M.unpack(np.asarray(params, dtype=np.float64))
    out, (vz_a, vz_w), (va_a, va_w), zs, acts = forward_sigma(params, x, norm)
    loss, grad = M.loss_and_grad(params, x, y, norm, bf=False)
    B = out.shape[0]
    y0, ys = float(norm[12]), float(norm[13])
    mu, lv = out[:, 0], out[:, 1]
    res = (np.asarray(y, float) - y0) * ys - mu
    w = np.exp(-lv)
    # L = mean(res^2 w + lv)/2: dL/dmu = -res w/B, dL/dlv = (1 - res^2 w)/(2B)
    lm, ll = res * w / B, (1.0 - res * res * w) / (2 * B)
    var_loss = np.sum(lm ** 2 * vz_a[-1][:, 0] + ll ** 2 * vz_a[-1][:, 1])
    # the weights' rounding moves the loss by sum_theta (dL/dtheta) delta theta (first order, exact)
    off = 0
    for (W, b) in layers:
        gW = grad[off:off + W.size]
        var_loss += U2 * np.sum((gW * W.ravel()) ** 2)
        off += W.size + b.size
    # dz_4 = (-res w/B, (1 - res^2 w)/(2B)) and its derivatives with respect to (mu, lv)
    dz = np.stack([-res * w / B, 0.5 * (1.0 - res * res * w) / B], axis=1)
    d00, d01 = w / B, res * w / B
    d10, d11 = res * w / B, 0.5 * res * res * w / B

    def head(v):
        return np.stack([d00 ** 2 * v[:, 0] + d01 ** 2 * v[:, 1], d10 ** 2 * v[:, 0] + d11 ** 2 * v[:, 1]], axis=1)

    vd_a = head(vz_a[-1]) + E2 * dz * dz
    vd_w = head(vz_w[-1])
    sg = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        W2 = W * W
        a2 = acts[l] ** 2
        d2 = dz * dz
        var_gW = (vd_a + U2 * d2).T @ a2 + d2.T @ va_a[l] + B * E2 * (d2.T @ a2)
        # sum over rows of per-row standard deviations (Cauchy-Schwarz gives the bound below
        # cheaply: sum_b sqrt(p_b q_b) <= sqrt(sum_b p_b sum_b q_b) would lose too much, so the
        # per-row terms are summed exactly)
        sd_gW = np.einsum("bi,bj->ij", np.sqrt(vd_w), np.sqrt(a2)) + np.einsum("bi,bj->ij", np.sqrt(d2),
                                                                                np.sqrt(va_w[l]))
        var_gb = vd_a.sum(axis=0) + B * E2 * d2.sum(axis=0)
        sd_gb = np.sqrt(vd_w).sum(axis=0)
        sg[l] = (np.sqrt(var_gW + sd_gW ** 2), np.sqrt(var_gb + sd_gb ** 2))
        if l > 0:
            gp2 = M.gelu_grad(zs[l - 1]) ** 2
            gpp2 = _gelu_second(zs[l - 1]) ** 2
            dzW = dz @ W
            vd_a_next = gp2 * ((vd_a + U2 * d2) @ W2 + W.shape[0] * E2 * (d2 @ W2)) + dzW * dzW * gpp2 * vz_a[l - 1]
            vd_w = gp2 * (vd_w @ W2 + U2 * (d2 @ W2)) + dzW * dzW * gpp2 * vz_w[l - 1]
            vd_a = vd_a_next
            dz = dzW * M.gelu_grad(zs[l - 1])
    flat = np.concatenate([np.concatenate([a.ravel(), c]) for a, c in sg])
    return loss, grad, float(np.sqrt(var_loss)), flat

"""Surrogate network: GPU kernels against the FP64 oracle (forward and gradients), and a reduced
end-to-end run showing what the trained network gains over solving every scan point."""
import time

import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


def _table(n, seed):
    from paper_2512_16889_gb300 import workloads as W
    return W.surrogate_samples(n, seed=seed)


def test_forward_and_gradients_match_oracle():
    """Forward (tensor-memory inference kernel), loss and gradients (training kernels) against the
    plain FP64 network (oracle bf=False, pinned by finite differences), element by element within
    6 standard deviations of the probabilistic BF16 error model of tests/bf16_bounds.py (about
    0.7 % of mu); and, as a secondary check, against the oracle's BF16-rounding network."""
    import torch
    from paper_2512_16889_gb300 import build, surrogate as S, swf
    from tests import bf16_bounds as BB
    build.build()
    t = _table(192, seed=11)
    X = S.features(t)
    y = (-12.0 + 3.0 * np.tanh(X[:, 0] * 5 - 1.0) + 0.5 * X[:, 3] * X[:, 4]).astype(np.float32)
    norm = S.normalisation(X, y)
    p0 = S.init_params(seed=3)
    p0[np.arange(p0.size) % 7 == 0] *= 0.5  # break symmetry of the zero biases' neighbourhood
    sur = swf.Surrogate(p0, norm, max_batch=256)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    out = torch.zeros(len(X), 2, dtype=torch.float32, device="cuda")
    sur.forward(Xd, out)  # 192 rows: one full tile of 128 and a ragged one
    sur.status()
    pf, Xf, yf, nf = p0.astype(float), X.astype(float), y.astype(float), norm.astype(float)
    mu64, lv64, smu, slv = BB.head_sigma(pf, Xf, nf)
    got = out.cpu().numpy().astype(float)
    assert np.all(np.abs(got[:, 0] - mu64) <= BB.K * smu), np.max(np.abs(got[:, 0] - mu64) / smu)
    assert np.all(np.abs(got[:, 1] - lv64) <= BB.K * slv), np.max(np.abs(got[:, 1] - lv64) / slv)
    grad = torch.zeros(swf.Surrogate.param_count(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    sur.gradients(Xd, yd, grad, loss)
    loss64, g64, sl, sg = BB.loss_grad_sigma(pf, Xf, yf, nf)
    g = grad.cpu().numpy().astype(float)
    assert abs(loss.item() - loss64) <= BB.K * sl, (loss.item(), loss64, sl)
    assert np.all(np.abs(g - g64) <= BB.K * sg), np.max(np.abs(g - g64) / sg)
    # secondary: the oracle's network with the kernels' BF16 rounding points
    mu_ref, lv_ref = _heads(M.forward(pf, Xf, nf, bf=True)[0], norm)
    assert np.max(np.abs(got[:, 0] - mu_ref)) <= 1e-2 * max(1.0, np.max(np.abs(mu_ref)))
    assert np.max(np.abs(got[:, 1] - lv_ref)) <= 1e-2 * max(1.0, np.max(np.abs(lv_ref)))
    ref_loss, ref_g = M.loss_and_grad(pf, Xf, yf, nf, bf=True)
    assert abs(loss.item() - ref_loss) <= 1e-3 * abs(ref_loss)
    # the inference kernel (tensor memory) and the training path's forward give the same loss
    r = (y - norm[12]) * norm[13] - (got[:, 0] - norm[12]) * norm[13]
    lvs = got[:, 1] + 2.0 * np.log(norm[13])
    assert abs(0.5 * np.mean(r * r * np.exp(-lvs) + lvs) - loss.item()) <= 1e-3 * abs(loss.item())
    off = 0
    for i, o in zip(M.DIN, M.DOUT):  # per layer, weights and biases
        for size in (i * o, o):
            a, b = g[off:off + size], ref_g[off:off + size]
            assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-12, (off, size)
            off += size
    sur.close()


def _heads(z, norm):
    """Network outputs in the target's units: mu = mu'/ys + y0, log sigma^2 = l' - 2 ln ys."""
    ys = float(norm[13])
    return z[:, 0] / ys + float(norm[12]), z[:, 1] - 2.0 * np.log(ys)


@pytest.mark.parametrize("n_rows", [1, 127, 40000])
def test_inference_tiles_match_oracle(n_rows):
    """The persistent inference kernel on a single row, on one ragged tile, and on 313 tiles
    (more tiles than SMs, so CTAs loop), against the oracle on sampled rows."""
    import torch
    from paper_2512_16889_gb300 import build, surrogate as S, swf
    build.build()
    t = _table(n_rows, seed=21)
    X = S.features(t)
    y = (-9.0 + np.tanh(3 * X[:, 0]) + 0.4 * X[:, 3]).astype(np.float32)
    norm = S.normalisation(X, y) if n_rows > 1 else np.concatenate([np.zeros(6), np.ones(6), [-9.0, 1.0]]).astype(np.float32)
    p0 = S.init_params(seed=5)
    p0[np.arange(p0.size) % 5 == 0] *= -0.7
    sur = swf.Surrogate(p0, norm, max_batch=256)
    out = torch.full((n_rows, 2), float("nan"), dtype=torch.float32, device="cuda")
    sur.forward(torch.from_numpy(X).cuda(), out)
    sur.status()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    rows = np.unique(np.concatenate([np.arange(min(n_rows, 64)), np.arange(max(0, n_rows - 64), n_rows),
                                     np.random.default_rng(1).integers(0, n_rows, 256)]))
    from tests import bf16_bounds as BB
    mu64, lv64, smu, slv = BB.head_sigma(p0.astype(float), X[rows].astype(float), norm.astype(float))
    assert np.all(np.abs(got[rows, 0] - mu64) <= BB.K * smu), np.max(np.abs(got[rows, 0] - mu64) / smu)
    assert np.all(np.abs(got[rows, 1] - lv64) <= BB.K * slv), np.max(np.abs(got[rows, 1] - lv64) / slv)
    mu_ref, lv_ref = _heads(M.forward(p0.astype(float), X[rows].astype(float), norm.astype(float), bf=True)[0], norm)
    assert np.max(np.abs(got[rows, 0] - mu_ref)) <= 1e-2 * max(1.0, np.max(np.abs(mu_ref)))
    assert np.max(np.abs(got[rows, 1] - lv_ref)) <= 1e-2 * max(1.0, np.max(np.abs(lv_ref)))
    sur.close()


def _momentum_scan(n, seed):
    """A momentum scan at the fixed field of the batched workload (E = 0.3, omega = 0.5, lambda = 5)."""
    rng = np.random.default_rng(seed)
    return {"E": np.full(n, 0.3), "omega": np.full(n, 0.5), "lam": np.full(n, 5.0),
            "px": rng.uniform(-1, 1, n), "py": rng.uniform(-1, 1, n), "s": rng.choice([1, -1], n)}


def test_surrogate_screens_a_momentum_scan():
    """Reduced scale (64^2 grid, 200 steps, 2048 training points): train on solver output,
    calibrate the sigma threshold on held-out solver data, then scan; the accepted points need no
    solve and the rest fall back to the solver, so the scan is exact there."""
    from paper_2512_16889_gb300 import build, surrogate as S, swf
    build.build()
    grid = dict(n=64, L=40.0, n_steps=200, t_window=20.0)
    ctx = swf.Context(0)
    tr, ho, sc = _momentum_scan(2048, 4), _momentum_scan(256, 5), _momentum_scan(512, 6)
    y_tr = S.solve_targets(ctx, tr, **grid)
    y_ho = S.solve_targets(ctx, ho, **grid)
    X_tr = S.features(tr)
    sur = swf.Surrogate(S.init_params(0), S.normalisation(X_tr, y_tr), max_batch=512)
    hist = S.train(sur, X_tr, y_tr, epochs=800, batch=256, lr=1e-3)
    assert hist[-1] < hist[0]
    tol = 5e-2  # in ln P (5 % in P): what this training-set size reaches on part of the scan
    thr = S.calibrate(sur, S.features(ho), y_ho, tol, coverage=0.95)
    assert thr > 0
    t0 = time.perf_counter()
    y_all = S.solve_targets(ctx, sc, **grid)  # the method without the network: solve every point
    t_all = time.perf_counter() - t0
    vals, acc, t_net, t_sol = S.screened_scan(sur, ctx, sc, thr, **grid)
    frac = acc.mean()
    err = np.abs(vals - y_all)
    print(f"accepted {frac:.1%} of the scan; screened {t_net + t_sol:.2f} s vs all-solver {t_all:.2f} s; "
          f"accepted within tol: {(err[acc] <= tol).mean():.1%}")
    assert frac > 0.15
    assert (err[acc] <= tol).mean() >= 0.85
    assert np.all(err[~acc] == 0.0)  # the fallback is the solver itself
    assert t_net + t_sol < t_all
    sur.close()
    ctx.close()


def test_train_step_is_one_adam_step_on_the_gradient():
    """The captured training step (one CUDA graph per batch size) applies Adam to the gradient of
    swf_mlp_gradients: first step m = (1 - b1) g, v = (1 - b2) g^2, p -= lr (m/c1)/(sqrt(v/c2) + eps);
    a second batch size and a repeat of the first reuse or capture their own graphs."""
    import torch
    from paper_2512_16889_gb300 import build, surrogate as S, swf
    build.build()
    t = _table(256, seed=31)
    X = S.features(t)
    y = (-11.0 + 2.0 * np.tanh(X[:, 0] * 4) + 0.3 * X[:, 4]).astype(np.float32)
    norm = S.normalisation(X, y)
    p0 = S.init_params(seed=7)
    sur = swf.Surrogate(p0, norm, max_batch=256)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    g = torch.zeros(swf.Surrogate.param_count(), dtype=torch.float32, device="cuda")
    sur.gradients(Xd, yd, g)
    g = g.cpu().numpy().astype(np.float64)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    sur.train_step(Xd, yd, lr, loss)
    p1 = sur.params().astype(np.float64)
    m, v = (1 - b1) * g, (1 - b2) * g * g
    ref = p0.astype(np.float64) - lr * (m / (1 - b1)) / (np.sqrt(v / (1 - b2)) + eps)
    assert np.max(np.abs(p1 - ref)) <= 1e-6 + 1e-5 * np.max(np.abs(ref)), np.max(np.abs(p1 - ref))
    assert np.isfinite(loss.item())
    sur.train_step(Xd[:128].contiguous(), yd[:128].contiguous(), lr, loss)
    sur.train_step(Xd, yd, lr, loss)
    assert np.all(np.isfinite(sur.params()))
    assert np.max(np.abs(sur.params() - p1)) > 0
    sur.close()


def test_activation_matches_the_exact_gelu():
    """The network's GELU (erf by Abramowitz and Stegun's formula 7.1.26, |error| <= 1.5e-7) and
    its derivative against the exact x Phi(x) and Phi(x) + x phi(x) in FP64, over the range the
    hidden layers see and beyond: within 4e-7 absolute (plus FP32 rounding of x Phi(x)), far
    below the bfloat16 rounding (2^-8 relative) applied to its outputs."""
    import torch
    from scipy.special import erf
    from paper_2512_16889_gb300 import build, swf
    build.build()
    x = np.concatenate([np.linspace(-12, 12, 200001), [0.0, -0.0, 1e-30, -1e-30, 60.0, -60.0]]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    g = torch.empty_like(xd)
    dg = torch.empty_like(xd)
    swf.Surrogate.activation(xd, g, dg)
    torch.cuda.synchronize()
    xx = x.astype(np.float64)
    cdf = 0.5 * (1.0 + erf(xx / np.sqrt(2.0)))
    pdf = np.exp(-0.5 * xx * xx) / np.sqrt(2.0 * np.pi)
    gg, dd = g.cpu().numpy().astype(np.float64), dg.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(gg)) and np.all(np.isfinite(dd))
    assert np.max(np.abs(gg - xx * cdf) / np.maximum(1.0, np.abs(xx))) < 4e-7
    assert np.max(np.abs(dd - (cdf + xx * pdf)) / np.maximum(1.0, np.abs(xx))) < 4e-7

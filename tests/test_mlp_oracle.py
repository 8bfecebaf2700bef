"""Pins of the surrogate network's oracle: finite differences of the FP64 loss, GELU against
its definition, and the bfloat16 rounding against the format's definition."""
import numpy as np

from oracle import mlp_oracle as M


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = []
    for i, o in zip(M.DIN, M.DOUT):
        p.append(rng.normal(scale=scale / np.sqrt(i), size=i * o))
        p.append(rng.normal(scale=0.05, size=o))
    return np.concatenate(p)


NORM = np.array([0.3, 0.5, 5.5, 0.0, 0.0, 0.0, 10.0, 3.3, 0.4, 1.7, 1.7, 1.0, -10.0, 0.2])


def test_gelu_and_bf16_definitions():
    x = np.linspace(-4, 4, 101)
    h = 1e-6
    assert np.allclose((M.gelu(x + h) - M.gelu(x - h)) / (2 * h), M.gelu_grad(x), atol=1e-8)
    assert np.isclose(M.gelu(1.0), 0.8413447460685429)  # x Phi(x) at 1
    # bfloat16 keeps 8 significand bits, ties to even
    assert M.bf16(1.0 + 2 ** -8) == 1.0 and M.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert M.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7
    assert M.bf16(-3.0) == -3.0


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    p = _params(1)
    x = np.stack([rng.uniform(0.15, 0.45, 12), rng.uniform(0.2, 0.8, 12), rng.uniform(3, 8, 12),
                  rng.uniform(-1, 1, 12), rng.uniform(-1, 1, 12), rng.choice([-1.0, 1.0], 12)], axis=1)
    y = rng.normal(-10, 3, 12)
    loss, g = M.loss_and_grad(p, x, y, NORM, bf=False)
    idx = rng.choice(p.size, 40, replace=False)
    idx = np.concatenate([idx, [0, 5, p.size - 1, p.size - 2, p.size - 3]])  # first and output layers
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        num = (M.loss_and_grad(p + e, x, y, NORM, bf=False)[0] - M.loss_and_grad(p - e, x, y, NORM, bf=False)[0]) / 2e-6
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, num, g[i])


def test_bf16_error_model_covers_the_oracles_bf16_arithmetic():
    """The probabilistic BF16 error model (tests/bf16_bounds.py) that sets the GPU tolerances,
    checked against one realisation of BF16 arithmetic, the oracle's bf=True network: its
    outputs, loss and every gradient element lie within 6 model standard deviations of the
    plain FP64 network (measured: at most 2.6 sigma forward, 1.7 sigma for the gradients)."""
    from tests import bf16_bounds as BB
    from paper_2512_16889_gb300 import surrogate as S, workloads as W
    t = W.surrogate_samples(192, seed=11)
    X = S.features(t).astype(float)
    y = -12.0 + 3.0 * np.tanh(X[:, 0] * 5 - 1.0) + 0.5 * X[:, 3] * X[:, 4]
    norm = S.normalisation(X.astype(np.float32), y.astype(np.float32)).astype(float)
    p = S.init_params(seed=3).astype(float)
    mu, lv, smu, slv = BB.head_sigma(p, X, norm)
    mir = M.forward(p, X, norm, bf=True)[0]
    ys = norm[13]
    assert np.all(np.abs(mir[:, 0] / ys + norm[12] - mu) <= BB.K * smu)
    assert np.all(np.abs(mir[:, 1] - 2 * np.log(ys) - lv) <= BB.K * slv)
    assert np.max(BB.K * smu / np.abs(mu)) < 1e-2  # the tolerance is below 1 % of the output
    loss, g, sl, sg = BB.loss_grad_sigma(p, X, y, norm)
    ml, mg = M.loss_and_grad(p, X, y, norm, bf=True)
    assert abs(ml - loss) <= BB.K * sl
    assert np.all(np.abs(mg - g) <= BB.K * sg)
    # the tolerance is not vacuous: scaling any one weight matrix by 1.03 moves some output by
    # more than 6 sigma (9 to 17 sigma, depending on the layer)
    off = 0
    for i, o in zip(M.DIN, M.DOUT):
        q = p.copy()
        q[off:off + i * o] *= 1.03
        out_q = M.forward(q, X, norm, bf=False)[0]
        assert np.any(np.abs(out_q[:, 0] / ys + norm[12] - mu) > BB.K * smu), off
        off += i * o + o

"""Pins of the rank-prediction MLP oracle (oracle/mlp.py) against properties
that do not come from the oracle itself: central finite differences of the
loss, a network whose output is known in closed form, the closed form of the
first Adam step, and a fit of a target the network can represent."""
import numpy as np

from oracle import mlp


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = np.column_stack([rng.uniform(3, 9, n), rng.integers(1, 12, n), rng.uniform(0, 2, n),
                         rng.integers(1, 4, n), rng.uniform(0.7, 1.3, n), rng.uniform(0, 0.05, n)])
    t = np.log1p(rng.integers(1, 90, n).astype(float))
    return X, t


def _theta(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0, scale, mlp.NPARAMS)


def test_layout_size():
    assert mlp.NPARAMS == 64 * 6 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 8833
    th = _theta(0)
    assert np.array_equal(mlp.pack(mlp.unpack(th)), th)


def test_gradient_matches_central_differences():
    X, t = _data(40, 1)
    norm = mlp.standardisation(X, t)
    th = _theta(2)
    loss, g = mlp.loss_grad(th, X, t, norm)
    rng = np.random.default_rng(3)
    idx = rng.choice(mlp.NPARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        fd = (mlp.loss_grad(th + e, X, t, norm)[0] - mlp.loss_grad(th - e, X, t, norm)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_closed_form():
    """W1 copies the standardised features into units 0..5, W2 and W3 pass
    units through, W4 sums them: y = sum_i relu(xh_i) + b4."""
    P = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    P["W1"][:6, :6] = np.eye(6)
    P["W2"][:6, :6] = np.eye(6)
    P["W3"][:6, :6] = np.eye(6)
    P["W4"][:6] = 1.0
    P["b4"][0] = 0.25
    X, t = _data(25, 4)
    norm = mlp.standardisation(X, t)
    y, _ = mlp.forward(mlp.pack(P), X, norm)
    Xh = (X - X.mean(axis=0)) / X.std(axis=0)
    assert np.allclose(y, np.maximum(Xh, 0).sum(axis=1) + 0.25, rtol=1e-13, atol=1e-13)


def test_first_adam_step_closed_form():
    th = _theta(5)
    g = np.random.default_rng(6).normal(size=mlp.NPARAMS)
    new, m, v = mlp.adam_step(th, g, np.zeros_like(th), np.zeros_like(th), 1, lr=1e-2)
    # bias correction makes m_hat = g and v_hat = g^2 at step 1
    assert np.allclose(new, th - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_standardisation_and_zero_variance_feature():
    X, t = _data(50, 7)
    X[:, 3] = 2.0
    mu, sd, tmu, tsd = mlp.standardisation(X, t)
    assert sd[3] == 1.0
    Xh = (X - mu) / sd
    assert np.allclose(Xh[:, [0, 1, 2, 4, 5]].mean(axis=0), 0, atol=1e-12)
    assert np.allclose(Xh[:, [0, 1, 2, 4, 5]].std(axis=0), 1, atol=1e-12)
    assert np.isclose(((t - tmu) / tsd).std(), 1)


def test_adam_fits_a_representable_target():
    """t = log(1 + k) with k a smooth function of the features: full-batch
    Adam drives the standardised loss well below its starting value."""
    X, _ = _data(200, 8)
    t = np.log1p(4 + 3 * X[:, 0] + 2 * X[:, 2] * X[:, 3])
    norm = mlp.standardisation(X, t)
    th = _theta(9, 0.2)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    l0 = mlp.loss_grad(th, X, t, norm)[0]
    for s in range(1, 301):
        loss, g = mlp.loss_grad(th, X, t, norm)
        th, m, v = mlp.adam_step(th, g, m, v, s, lr=3e-3)
    assert loss < 0.02 * l0 and loss < 0.02


def test_bf16_rounding_matches_library_conversion():
    """The oracle's bfloat16 rounding equals PyTorch's CPU conversion."""
    import torch
    rng = np.random.default_rng(10)
    a = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 500), [0.0, -0.0, 1.0, 3.0, 1.0 + 2 ** -8]])
    a = a.astype(np.float32)
    ref = torch.as_tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(a), ref)


def test_bf16_forward_close_to_fp64_forward():
    X, t = _data(64, 11)
    norm = mlp.standardisation(X, t)
    th = _theta(12, 0.2)
    y64, _ = mlp.forward(th, X, norm)
    yb = mlp.forward_bf16(th, X, norm)
    assert np.abs(yb - (norm[2] + norm[3] * y64)).max() <= 0.05 * norm[3] * max(1.0, np.abs(y64).max())

"""Pins of the MLP oracle: backpropagation against central finite differences (FP64,
unrounded weights), bfloat16 rounding against torch's conversion, closed-form special
cases of the forward pass."""
import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")


def _setup(L=6, B=37, seed=0):
    rng = np.random.default_rng(seed)
    P = mlp.param_count(L)
    params = rng.normal(size=P) * 0.4
    up = rng.integers(0, 2 ** L, size=B)
    dn = rng.integers(0, 2 ** L, size=B)
    x = mlp.features(up, dn, L, 3.0, round_inputs=False)
    psi = rng.normal(size=B) * 0.2
    psi[3] = 0.0          # a zero amplitude contributes nothing
    return L, params, x, psi


def test_backprop_matches_finite_differences():
    L, params, x, psi = _setup()
    _, g = mlp.loss_and_grad(params, x, psi, 7.0, L, round_weights=False)
    rng = np.random.default_rng(1)
    idx = rng.choice(len(params), size=60, replace=False)
    for i in idx:
        h = 1e-6
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_only(pp, x, psi, 7.0, L, False) - mlp.loss_only(pm, x, psi, 7.0, L, False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-5, 5, size=5000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0]]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(v), ref)


def test_forward_special_cases():
    L = 4
    P = mlp.param_count(L)
    params = np.zeros(P)
    params[-2:] = [-1.5, 0.25]          # b3: a = -1.5, z = 0.25 for every input
    x = mlp.features(np.array([3, 5]), np.array([1, 8]), L, 2.0)
    a, z, _ = mlp.forward(params, x, L)
    assert np.all(a == -1.5) and np.all(z == 0.25)
    assert np.allclose(mlp.predict(params, x, L), np.exp(-1.5))
    # a single input bit through W1 -> h1 -> h2 -> a with unit weights: nested tanh
    W1, b1, W2, b2, W3, b3 = mlp.unpack(params.copy(), L)
    params2 = np.zeros(P)
    o = 0
    params2[o + 0 * mlp.HIDDEN + 0] = 1.0            # W1[0][0]
    o = mlp.n_inputs(L) * mlp.HIDDEN + mlp.HIDDEN
    params2[o + 0 * mlp.HIDDEN + 0] = 1.0            # W2[0][0]
    o += mlp.HIDDEN * mlp.HIDDEN + mlp.HIDDEN
    params2[o + 0] = 1.0                              # W3[0][0]
    a, z, _ = mlp.forward(params2, x, L)
    h1b = float(torch.tensor(np.tanh(1.0), dtype=torch.float32).to(torch.bfloat16))
    assert np.allclose(a, [np.tanh(h1b), np.tanh(h1b)])


def test_features_layout():
    x = mlp.features(np.array([0b0101]), np.array([0b0010]), 4, 4.0)
    assert np.array_equal(x[0], [1, 0, 1, 0, 0, 1, 0, 0, 0.5])
    # U/8 enters rounded to bfloat16: 3.3/8 = 0.4125 -> 0.412109375
    x = mlp.features(np.array([0]), np.array([0]), 4, 3.3)
    assert x[0, -1] == 0.412109375

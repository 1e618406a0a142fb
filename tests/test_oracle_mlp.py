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


def test_forward_weight_layout_off_diagonal():
    """Parameter layout W1 [IN x 64] input-major, W2 [64 x 64] as (from unit, to unit), W3
    [64 x 2]: input bit 2 (up site 2) drives hidden unit 5 of layer one, which drives unit 9
    of layer two, which drives output z only. The two states with that bit set give
    z = tanh(bf16(tanh(1.5))) * 0.75, the others z = 0, and a = 0 throughout."""
    L = 4
    P = mlp.param_count(L)
    n_in, Hd = mlp.n_inputs(L), mlp.HIDDEN
    params = np.zeros(P)
    params[2 * Hd + 5] = 1.5                                   # W1[2][5]
    o2 = n_in * Hd + Hd
    params[o2 + 5 * Hd + 9] = 1.0                              # W2[5][9]
    o3 = o2 + Hd * Hd + Hd
    params[o3 + 9 * 2 + 1] = 0.75                              # W3[9][1]
    up = np.array([0b0100, 0b0011, 0b1100, 0b0000])
    x = mlp.features(up, np.array([0b0100, 0, 0, 0b1111]), L, 2.0)
    a, z, _ = mlp.forward(params, x, L)
    h1b = float(torch.tensor(np.tanh(1.5), dtype=torch.float32).to(torch.bfloat16))
    zz = np.tanh(h1b) * 0.75
    assert np.all(a == 0.0)
    assert np.allclose(z, [zz, 0.0, zz, 0.0], rtol=1e-15, atol=0)


def test_loss_and_output_gradient_worked_example():
    """Constant outputs (all weights zero, b3 = (a0, z0)) give the loss in closed form. With
    a0 = -0.6875 (exact in bfloat16), z0 = 0, psi = (e, -e/2, 0) for e = exp(a0) and
    c = 1 / e^2: the weights c psi^2 are (1, 0.25, 0), the log terms (0, (log 2)^2, -) and
    the sign terms log 2 each, so L = (1.25 log 2 + 0.25 (log 2)^2) / 3,
    dL/da0 = (0.5 log 2) / 3 and dL/dz0 = (-1/2 + 0.25/2) / 3 = -0.125."""
    L = 4
    P = mlp.param_count(L)
    params = np.zeros(P)
    a0 = -0.6875
    params[-2:] = [a0, 0.0]
    x = mlp.features(np.array([1, 2, 4]), np.array([8, 4, 2]), L, 4.0)
    e = np.exp(a0)
    psi = np.array([e, -e / 2, 0.0])
    ln2 = np.log(2.0)
    for rw in (True, False):
        loss, g = mlp.loss_and_grad(params, x, psi, 1.0 / (e * e), L, round_weights=rw)
        assert abs(loss - (1.25 * ln2 + 0.25 * ln2 * ln2) / 3.0) <= 1e-14
        assert abs(g[-2] - 0.5 * ln2 / 3.0) <= 1e-14
        assert abs(g[-1] - (-0.125)) <= 1e-14

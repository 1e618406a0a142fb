"""Ground-state vector (two-pass Lanczos) and the learned start vector: kernels against the
oracle (dense eigenvectors, FP64 backpropagation), and the gain of the trained network
over the random start of Algorithm 1."""
import math

import numpy as np
import pytest

import ed_inputs
from oracle import basis as obasis
from oracle import dense, mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ed():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1511_00863_gb300 as m
    return m


def _dev_view(ptr, n, typestr):
    class V:
        pass
    v = V()
    v.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                  "version": 3, "strides": None}
    return torch.as_tensor(v, device="cuda")


@pytest.mark.parametrize("case", [
    (8, ed_inputs.ring_bonds(8), 3, 3, 1.0, 4.0),
    (7, ed_inputs.ring_bonds(7), 3, 3, 1.0, 2.0),
    (6, ed_inputs.ring_bonds(6), 1, 1, 1.0, 3.0),
])
def test_ground_state_vector_vs_dense(ed, case):
    L, bonds, nu, nd, t, U = case
    E_ref, psi_ref = dense.ground_state(*case)
    w = dense.spectrum(*case)
    assert w[1] - w[0] > 1e-6   # non-degenerate: the vector is unique up to sign
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        dim = ed.ed_basis_dims(b)[2]
        psi = torch.empty(dim, dtype=torch.float64, device="cuda")
        res = ed.ed_lanczos_ground_state(b, t, U, ed.make_opts(max_steps=300, tol=1e-13, seed=3), psi)
    finally:
        ed.ed_basis_destroy(b)
    p = psi.cpu().numpy()
    assert abs(res["E0"] - E_ref) <= 1e-10 * abs(E_ref)
    assert abs(np.linalg.norm(p) - 1.0) <= 1e-12
    assert float(p @ psi_ref) >= 1.0 - 1e-9
    assert np.max(np.abs(p - psi_ref)) <= 1e-5


def _set_params(ed, net, values):
    ptr, n = ed.ed_mlp_params(net)
    dev = _dev_view(ptr, n, "<f4")
    dev.copy_(torch.tensor(values, dtype=torch.float32))
    torch.cuda.synchronize()


def test_mlp_gradient_vs_oracle(ed):
    L, nu, nd, U = 6, 3, 2, 3.0
    b = ed.ed_build_basis(L, ed_inputs.ring_bonds(L), nu, nd)
    net = ed.ed_mlp_create(L, 7)
    try:
        dim = ed.ed_basis_dims(b)[2]
        P = omlp.param_count(L)
        rng = np.random.default_rng(4)
        params = (rng.normal(size=P) * 0.3).astype(np.float32)
        _set_params(ed, net, params)
        n = 517                                   # several tiles and a ragged tail
        idx = rng.integers(0, dim, size=n)
        target = rng.normal(size=n) * 0.05
        target[5] = 0.0
        loss, gptr = ed.ed_mlp_loss_grad(net, b, U, torch.tensor(idx, device="cuda"),
                                         torch.tensor(target, device="cuda"), float(dim))
        g = _dev_view(gptr, P, "<f4").double().cpu().numpy()
        up = obasis.species_states(L, nu)
        dn = obasis.species_states(L, nd)
        x = omlp.features(up[idx // len(dn)], dn[idx % len(dn)], L, U)
        L_ref, g_ref = omlp.loss_and_grad(params.astype(np.float64), x, target, float(dim), L)
        assert abs(loss - L_ref) <= 1e-5 * abs(L_ref)
        assert np.max(np.abs(g - g_ref)) <= 1e-4 * np.max(np.abs(g_ref)), np.max(np.abs(g - g_ref))
    finally:
        ed.ed_mlp_destroy(net)
        ed.ed_basis_destroy(b)


# The inference evaluates tanh on the special-function unit (PTX tanh.approx.f32); the PTX ISA
# states a maximum relative error of about 2^-11 for it. Taken with a factor-2 margin:
EPS_TANH = 2.0 ** -10


@pytest.mark.parametrize("fill", [(3, 4), (3, 0)])
def test_mlp_inference_vs_unrounded_forward(ed, fill):
    """The network evaluated in FP64 with bfloat16 weights, exact tanh and without rounding the
    first layer's output or the U input (the plain definition of the network on rounded
    parameters) against the GPU's tensor-core inference, which feeds the second layer
    bfloat16 activations and bfloat16(U/8) and evaluates tanh with the approximation above:
    the difference must stay inside the bound those roundings (bfloat16: relative 2^-8 at
    most, taken twice as a margin; tanh: EPS_TANH) propagate through the layers (tanh is
    1-Lipschitz), plus FP32 accumulation at every layer. Fill (3, 0) has an empty species."""
    L, U = 8, 2.5
    nu, nd = fill
    b = ed.ed_build_basis(L, ed_inputs.ring_bonds(L), nu, nd)
    net = ed.ed_mlp_create(L, 13)
    try:
        dim = ed.ed_basis_dims(b)[2]
        P = omlp.param_count(L)
        params = (np.random.default_rng(6).normal(size=P) * 0.3).astype(np.float32)
        _set_params(ed, net, params)
        out = torch.empty(dim, dtype=torch.float64, device="cuda")
        ed.ed_mlp_infer(net, b, U, out)
        got = out.cpu().numpy()
    finally:
        ed.ed_mlp_destroy(net)
        ed.ed_basis_destroy(b)
    up = obasis.species_states(L, nu)
    dn = obasis.species_states(L, nd)
    g = np.arange(dim)
    x = omlp.features(up[g // len(dn)], dn[g % len(dn)], L, U, round_inputs=False)
    pr = omlp.bf16_round(params)            # bfloat16 weights, used as given below
    a, z, (_, h1, h2) = omlp.forward(pr, x, L, round_weights=False)
    W1, b1, W2, b2, W3, b3 = omlp.unpack(pr, L)
    u = 2.0 ** -8
    f32 = 1e-5                                                     # FP32 sums
    dh1 = np.abs(W1[2 * L]) * abs(U / 8.0) * u                  # bf16(U/8)
    dh1 = dh1[None, :] + f32 * (np.abs(x) @ np.abs(W1) + np.abs(b1)[None, :])
    dh1 = dh1 + EPS_TANH * (np.abs(h1) + dh1)                    # approximate tanh
    dh1 = dh1 + (np.abs(h1) + dh1) * u                           # bf16(h1)
    dh2 = dh1 @ np.abs(W2) + f32 * (np.abs(h1) @ np.abs(W2) + np.abs(b2)[None, :])
    dh2 = dh2 + EPS_TANH * (np.abs(h2) + dh2)                    # approximate tanh
    acc = f32 * (np.abs(h2) @ np.abs(W3) + np.abs(b3)[None, :])
    da = dh2 @ np.abs(W3[:, 0]) + acc[:, 0]
    dz = dh2 @ np.abs(W3[:, 1]) + acc[:, 1]
    sure = np.abs(z) > dz
    assert sure.mean() > 0.3   # the sign check is not vacuous
    assert np.all(np.sign(got[sure]) == np.where(z[sure] >= 0, 1.0, -1.0))
    err = np.abs(np.log(np.abs(got)) - a)
    assert np.all(err <= da), float(np.max(err / da))
    # the bound adds every rounding with the worst sign; actual roundings are of mixed sign
    assert np.median(err / da) < 0.25
    assert np.median(err) > 0.0   # the roundings are really there: not a tautology


def test_learned_start_saves_iterations(ed):
    """Train on ground states at U = 0, 1, ..., 8 of the L=10 ring at 5/5 (dim 63504), start
    Algorithm 1 from the network's prediction at held-out U: same E0 (oracle tolerance),
    fewer steps than the random start."""
    L, nu, nd = 10, 5, 5
    bonds = ed_inputs.ring_bonds(L)
    b = ed.ed_build_basis(L, bonds, nu, nd)
    net = ed.ed_mlp_create(L, 1)
    try:
        dim = ed.ed_basis_dims(b)[2]
        train_U = [float(u) for u in range(9)]
        psis = []
        for U in train_U:
            psi = torch.empty(dim, dtype=torch.float64, device="cuda")
            ed.ed_lanczos_ground_state(b, 1.0, U, ed.make_opts(max_steps=400, tol=1e-13, seed=2), psi)
            psis.append(psi)
        for step in range(600):
            k = step % len(train_U)
            ed.ed_mlp_train_step(net, b, train_U[k], psis[k], 4096, 3e-3, 1000 + step)
        opts = ed.make_opts(max_steps=400, tol=1e-11, seed=9)
        for U in (2.5, 5.5):
            rnd = ed.ed_lanczos_solve(b, 1.0, U, opts)
            f1 = torch.empty(dim, dtype=torch.float64, device="cuda")
            ed.ed_mlp_infer(net, b, U, f1)
            lrn = ed.ed_lanczos_solve(b, 1.0, U, opts, f1=f1)
            assert abs(lrn["E0"] - rnd["E0"]) <= 1e-10 * abs(rnd["E0"])
            assert lrn["steps"] < 0.8 * rnd["steps"], (U, lrn["steps"], rnd["steps"])
    finally:
        ed.ed_mlp_destroy(net)
        ed.ed_basis_destroy(b)

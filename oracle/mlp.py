"""Learned Lanczos start vector: the small network, its loss and its gradient in FP64.

The paper has no learned component; this is the oracle of the library's MLP (same
definition, written plainly). A basis state s = (up bits, down bits) of an L-site lattice
and the interaction U give the input features
    x = (up bit 0..L-1, down bit 0..L-1, bf16(U / 8))                 (2L + 1 values)
and the network
    h1 = tanh(W1^T x + b1), h2 = tanh(W2^T bf16(h1) + b2), (a, z) = W3^T h2 + b3
with 64 hidden units per layer. The predicted start-vector entry is sign(z) exp(a)
(z >= 0 counts as positive). The forward pass uses the weights rounded to bfloat16
(round to nearest even) and feeds the second layer the first layer's output rounded to
bfloat16 (the operands of the GPU's bfloat16 tensor-core products); it accumulates in FP64
here (FP32 on the GPU). The backward pass treats both roundings as the identity.

Loss over a batch of states s_k with target amplitudes psi_k (samples drawn uniformly,
weight w_k = c psi_k^2 with c = the basis dimension, so that E[w] = 1 for a normalised psi):
    L = (1/B) sum_k w_k [ (a_k - log|psi_k|)^2 + log(1 + exp(-sign(psi_k) z_k)) ]
States with psi_k = 0 contribute nothing. The gradient is taken with respect to the
rounded weights and applied to the FP32 master weights (straight-through).

Parameter layout (flat, FP32): W1 [IN x 64] (input-major), b1 [64], W2 [64 x 64], b2 [64],
W3 [64 x 2], b3 [2], IN = 2L + 1.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64


def n_inputs(n_sites: int) -> int:
    return 2 * n_sites + 1


def param_count(n_sites: int) -> int:
    n_in = n_inputs(n_sites)
    return n_in * HIDDEN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN * 2 + 2


def unpack(params: np.ndarray, n_sites: int):
    n_in = n_inputs(n_sites)
    p = np.asarray(params)
    o = 0
    W1 = p[o:o + n_in * HIDDEN].reshape(n_in, HIDDEN); o += n_in * HIDDEN
    b1 = p[o:o + HIDDEN]; o += HIDDEN
    W2 = p[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = p[o:o + HIDDEN]; o += HIDDEN
    W3 = p[o:o + HIDDEN * 2].reshape(HIDDEN, 2); o += HIDDEN * 2
    b3 = p[o:o + 2]; o += 2
    return W1, b1, W2, b2, W3, b3


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16 (nearest, ties to even), returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def features(up_bits: np.ndarray, dn_bits: np.ndarray, n_sites: int, U: float,
             round_inputs: bool = True) -> np.ndarray:
    up = np.asarray(up_bits, dtype=np.int64)
    dn = np.asarray(dn_bits, dtype=np.int64)
    x = np.zeros((len(up), n_inputs(n_sites)))
    for i in range(n_sites):
        x[:, i] = (up >> i) & 1
        x[:, n_sites + i] = (dn >> i) & 1
    x[:, 2 * n_sites] = bf16_round(np.float32(U / 8.0)) if round_inputs else U / 8.0
    return x


def _weights(params, n_sites, round_weights):
    ws = unpack(params, n_sites)
    return tuple(bf16_round(w) if round_weights else np.asarray(w, dtype=np.float64) for w in ws)


def forward(params, x, n_sites, round_weights=True):
    W1, b1, W2, b2, W3, b3 = _weights(params, n_sites, round_weights)
    h1 = np.tanh(x @ W1 + b1)
    h1b = bf16_round(h1) if round_weights else h1
    h2 = np.tanh(h1b @ W2 + b2)
    out = h2 @ W3 + b3
    return out[:, 0], out[:, 1], (x, h1, h2)


def predict(params, x, n_sites, round_weights=True):
    a, z, _ = forward(params, x, n_sites, round_weights)
    return np.where(z >= 0, 1.0, -1.0) * np.exp(a)


def loss_and_grad(params, x, psi, weight_scale, n_sites, round_weights=True):
    """Loss L and dL/dparams (FP64), by explicit backpropagation through the layers.
    round_weights=False evaluates the same network with unrounded weights (used to check the
    backpropagation against finite differences, which the bfloat16 steps would defeat)."""
    W1, b1, W2, b2, W3, b3 = _weights(params, n_sites, round_weights)
    B = len(psi)
    psi = np.asarray(psi, dtype=np.float64)
    h1 = np.tanh(x @ W1 + b1)
    h1b = bf16_round(h1) if round_weights else h1
    h2 = np.tanh(h1b @ W2 + b2)
    out = h2 @ W3 + b3
    a, z = out[:, 0], out[:, 1]
    live = psi != 0.0
    w = np.where(live, weight_scale * psi * psi, 0.0)
    l = np.where(live, np.log(np.where(live, np.abs(psi), 1.0)), 0.0)
    sg = np.where(psi >= 0, 1.0, -1.0)
    L = np.sum(w * ((a - l) ** 2 + np.logaddexp(0.0, -sg * z))) / B
    da = w * 2.0 * (a - l) / B
    dz = w * (-sg) / (1.0 + np.exp(sg * z)) / B
    dout = np.stack([da, dz], axis=1)
    gW3 = h2.T @ dout
    gb3 = dout.sum(0)
    g2 = (dout @ W3.T) * (1.0 - h2 * h2)
    gW2 = h1b.T @ g2
    gb2 = g2.sum(0)
    g1 = (g2 @ W2.T) * (1.0 - h1 * h1)
    gW1 = x.T @ g1
    gb1 = g1.sum(0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, grad


def loss_only(params, x, psi, weight_scale, n_sites, round_weights=True):
    return loss_and_grad(params, x, psi, weight_scale, n_sites, round_weights)[0]

"""Surrogate initial guess: POD basis and a fully connected network (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Not part of the
paper's method: the paper starts Newton from zero interior velocity with the
Dirichlet data on the boundary (section 2.4).  This module is the plain
reference for the learned initial guess y0 = ybar + Phi diag(sigma) f(x):

* ``pod_basis``: proper orthogonal decomposition of solution snapshots --
  the mean ybar and the leading left singular vectors Phi of the centred
  snapshot matrix, with their singular values (library SVD).
* ``mlp_forward`` / ``mlp_backward``: a fully connected network
  f(x) = W_L h_{L-1} + b_L, h_l = tanh(W_l h_{l-1} + b_l), h_0 = x, and the
  gradient of the loss (1 / 2B) sum_b ||f(x_b) - t_b||^2 by the chain rule,
  layer by layer in reverse.
* ``adam_step``: Adam (Kingma & Ba 2015) with bias correction.

The network inputs come from ``workloads.cases.surrogate_inputs`` (input
encoding, shared with the GPU path).

Row-major conventions shared with the CUDA kernels: a batch is X[B][n_in],
a weight W_l[n_out][n_in] (out x in), so a layer is X W_l^T + b_l.

Pinned by tests/test_oracle_surrogate.py: the backward pass against central
differences of the loss; a network with identity-like tiny weights against
its linearisation; the first Adam step moves every parameter by exactly lr
against the sign of its gradient; the POD basis is orthonormal, reproduces
the snapshots at full rank and orders its energies.
"""
from __future__ import annotations

import numpy as np


# ------------------------------------------------------------------ POD

def pod_basis(snapshots: np.ndarray, k: int):
    """snapshots [S][n] -> (mean [n], Phi [n][k], sigma [k]) of the centred set."""
    Y = np.asarray(snapshots, dtype=np.float64)
    mean = Y.mean(axis=0)
    X = (Y - mean).T                        # [n][S]
    U, s, _ = np.linalg.svd(X, full_matrices=False)
    k = min(k, U.shape[1])
    return mean, U[:, :k], s[:k]


def pod_coefficients(y: np.ndarray, mean: np.ndarray, Phi: np.ndarray, sigma: np.ndarray):
    """Normalised coefficients a = Phi^T (y - mean) / sigma (the network's targets)."""
    return (Phi.T @ (np.asarray(y, dtype=np.float64).reshape(-1) - mean)) / sigma


def pod_reconstruct(a: np.ndarray, mean: np.ndarray, Phi: np.ndarray, sigma: np.ndarray):
    return mean + Phi @ (np.asarray(a) * sigma)


# ------------------------------------------------------------------ network

def mlp_init(sizes, seed: int):
    """Weights ~ U(-1/sqrt(n_in), 1/sqrt(n_in)), biases zero."""
    rng = np.random.default_rng(seed)
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        lim = 1.0 / np.sqrt(n_in)
        params.append((rng.uniform(-lim, lim, size=(n_out, n_in)), np.zeros(n_out)))
    return params


def mlp_forward(params, X):
    """Returns the output and the list of layer inputs h_0 .. h_{L-1}."""
    h = np.asarray(X, dtype=np.float64)
    hs = []
    for l, (W, b) in enumerate(params):
        hs.append(h)
        z = h @ W.T + b
        h = np.tanh(z) if l < len(params) - 1 else z
    return h, hs


def mlp_loss(params, X, T):
    out, _ = mlp_forward(params, X)
    return 0.5 * np.sum((out - T) ** 2) / X.shape[0]


def mlp_backward(params, X, T):
    """Loss and gradients [(dW_l, db_l)] of (1 / 2B) sum ||f(x) - t||^2."""
    out, hs = mlp_forward(params, X)
    B = X.shape[0]
    loss = 0.5 * np.sum((out - T) ** 2) / B
    delta = (out - T) / B                    # dLoss / dz_L
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        h = hs[l]
        grads[l] = (delta.T @ h, delta.sum(axis=0))
        if l > 0:
            # h_l = tanh(z_l): dLoss/dz_{l} = (delta W) * (1 - h_l^2)
            delta = (delta @ W) * (1.0 - hs[l] ** 2)
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state = {"t": int, "m": [...], "v": [...]}."""
    if not state:
        state["t"] = 0
        state["m"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        state["v"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    state["t"] += 1
    t = state["t"]
    new = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for p, g, i in ((W, gW, 0), (b, gb, 1)):
            m = state["m"][l][i]
            v = state["v"][l][i]
            m[...] = beta1 * m + (1 - beta1) * g
            v[...] = beta2 * v + (1 - beta2) * g * g
            mhat = m / (1 - beta1 ** t)
            vhat = v / (1 - beta2 ** t)
            out.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        new.append(tuple(out))
    params[:] = new
    return params

"""Pins of the surrogate reference (oracle/surrogate.py) against properties
that do not restate its formulas: finite differences, linearisation, the
closed-form first Adam step, SVD identities."""
import numpy as np

from oracle import surrogate as sg
from workloads import cases


def _net(seed=0, sizes=(5, 7, 6, 3)):
    return sg.mlp_init(list(sizes), seed)


def test_backward_matches_central_differences():
    params = _net()
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4, 5))
    T = rng.standard_normal((4, 3))
    # non-zero biases so that their gradients are exercised too
    params = [(W, rng.standard_normal(b.shape) * 0.3) for W, b in params]
    _, grads = sg.mlp_backward(params, X, T)
    h = 1e-6
    for l in range(len(params)):
        for which in (0, 1):
            P = params[l][which]
            G = grads[l][which]
            for idx in [tuple(rng.integers(0, s) for s in P.shape) for _ in range(4)]:
                old = P[idx]
                P[idx] = old + h
                lp = sg.mlp_loss(params, X, T)
                P[idx] = old - h
                lm = sg.mlp_loss(params, X, T)
                P[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - G[idx]) <= 1e-7 * max(1.0, abs(fd)), (l, which, idx, fd, G[idx])


def test_tiny_weights_linearise():
    # with weights scaled by eps, tanh(z) = z + O(z^3): the network is the
    # product of its matrices to relative O(eps^2)
    params = _net(seed=3)
    eps = 1e-4
    params = [(W * eps, b) for W, b in params]
    x = np.random.default_rng(2).standard_normal((1, 5))
    out, _ = sg.mlp_forward(params, x)
    lin = x
    for W, _ in params:
        lin = lin @ W.T
    assert np.allclose(out, lin, rtol=1e-7, atol=0)
    # a transposed layer changes the result
    bad = x
    for W, _ in params[:1]:
        bad = bad @ W.T
    assert out.shape == (1, 3) and bad.shape == (1, 7)


def test_first_adam_step_moves_by_lr():
    # after one step m_hat = g and v_hat = g^2, so the move is lr g / (|g| + eps)
    params = _net(seed=4)
    before = [(W.copy(), b.copy()) for W, b in params]
    rng = np.random.default_rng(5)
    grads = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in params]
    state = {}
    sg.adam_step(params, grads, state, lr=0.01, eps=0.0)
    for (W0, b0), (W1, b1), (gW, gb) in zip(before, params, grads):
        assert np.allclose(W0 - W1, 0.01 * np.sign(gW), atol=1e-15)
        assert np.allclose(b0 - b1, 0.01 * np.sign(gb), atol=1e-15)


def test_adam_training_fits_a_smooth_map():
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, size=(64, 3))
    T = np.column_stack([np.sin(X[:, 0]) + X[:, 1] * X[:, 2], np.cos(X[:, 1])])
    params = sg.mlp_init([3, 32, 32, 2], seed=7)
    state = {}
    l0 = sg.mlp_loss(params, X, T)
    for _ in range(1500):
        _, g = sg.mlp_backward(params, X, T)
        sg.adam_step(params, g, state, lr=3e-3)
    assert sg.mlp_loss(params, X, T) < 0.01 * l0


def test_pod_basis_properties():
    rng = np.random.default_rng(8)
    S, n = 12, 40
    Y = rng.standard_normal((S, 3)) @ rng.standard_normal((3, n)) + 0.01 * rng.standard_normal((S, n))
    mean, Phi, sigma = sg.pod_basis(Y, 12)
    assert np.allclose(Phi.T @ Phi, np.eye(Phi.shape[1]), atol=1e-12)
    assert np.all(np.diff(sigma) <= 1e-12)
    # three dominant directions carry almost all the energy
    assert sigma[3] < 0.05 * sigma[2]
    # full rank reproduces every snapshot; the coefficients round-trip
    for y in Y:
        a = sg.pod_coefficients(y, mean, Phi, sigma)
        assert np.allclose(sg.pod_reconstruct(a, mean, Phi, sigma), y, atol=1e-10)
    # the mean is the optimal rank-0 approximation: centred snapshots sum to zero
    assert np.allclose((Y - mean).sum(axis=0), 0.0, atol=1e-12)


def test_encode_inputs_layout():
    U1 = np.array([1.0, 0.1 + 0.2j, -0.3j, 0.05, 0.0, 0.0, 0.0])
    U2 = np.array([1.0, 0.4, 0.0, 0.0, -0.02j, 0.0, 0.0])
    x = cases.surrogate_inputs([U1, U2], Re=800.0, Wo=10.0)
    assert x.shape == (18,)
    assert np.allclose(x[:8], [0.1, 0.2, 0.0, -0.3, 0.05, 0.0, 0.0, 0.0])
    assert np.allclose(x[8:16], [0.4, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -0.02])
    assert np.allclose(x[16:], [1.0, 1.0])

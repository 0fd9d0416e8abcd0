"""Learned initial guess: GPU network, Adam and POD kernels vs the oracle
(oracle/surrogate.py), and what the trained guess gains over the plain
initial guess on seeded pulsatile pipe solves.

Bars: forward within 1e-5 and gradients within 1e-4 relative L2 of the FP64
oracle (FP32 kernels); POD singular values within 1e-4, coefficients within
1e-4 after aligning each basis vector's sign (eigenvectors are unique up to
sign).  Solves from the surrogate reach the same tolerance and the same
field (1e-6) as solves from the plain guess.
"""
import math

import numpy as np
import pytest

from oracle import surrogate as sg
from workloads import cases, meshgen as mg

from gpu_util import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _sur(n_in=18, hidden=70, layers=3, n_out=20, n_dof=100, seed=1):
    import paper_2311_09465_gb300 as ts
    return ts.Surrogate(n_in, hidden, layers, n_out, n_dof, seed=seed)


def _oracle_params(s, flat=None):
    return [(W.astype(np.float64), b.astype(np.float64)) for W, b in s.layers(flat)]


def test_forward_and_gradient_match_oracle(torch):
    s = _sur()
    rng = np.random.default_rng(2)
    flat = s.get_params()
    # non-zero biases so that their paths are exercised
    for W, b in s.layers(flat):
        b[:] = rng.standard_normal(b.shape) * 0.2
    s.set_params(flat)
    B = 37                                    # ragged against the 64-row tile
    X = rng.standard_normal((B, 18))
    T = rng.standard_normal((B, 20))
    params = _oracle_params(s, flat)
    out_ref, _ = sg.mlp_forward(params, X)
    out = to_np(s.forward(to_dev(X, torch.float32)))
    assert rel_l2(out, out_ref) <= 1e-5, rel_l2(out, out_ref)
    loss_ref, grads = sg.mlp_backward(params, X, T)
    loss, g = s.gradient(to_dev(X, torch.float32), to_dev(T, torch.float32))
    g = to_np(g)
    flat_ref = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    assert rel_l2(g, flat_ref) <= 1e-4, rel_l2(g, flat_ref)
    # every layer separately, so a small layer's error is not hidden by a large one
    off = 0
    for gW, gb in grads:
        n = gW.size + gb.size
        assert rel_l2(g[off: off + n], np.concatenate([gW.ravel(), gb])) <= 1e-4
        off += n


def test_adam_steps_match_oracle(torch):
    s = _sur(seed=3)
    rng = np.random.default_rng(4)
    params = _oracle_params(s)
    state = {}
    for it in range(3):
        X = rng.standard_normal((16, 18))
        T = rng.standard_normal((16, 20))
        _, g = s.gradient(to_dev(X, torch.float32), to_dev(T, torch.float32))
        s.adam(g, 1e-2)
        _, grads = sg.mlp_backward(params, X, T)
        sg.adam_step(params, grads, state, lr=1e-2)
    got = s.get_params()
    ref = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)


def test_pod_basis_and_coefficients_match_oracle(torch):
    rng = np.random.default_rng(5)
    S, n = 12, 5003                           # ragged against tiles and split-K chunks
    # eight directions with well separated energies (consecutive singular values
    # differ by >= 25%), so every basis vector is unique up to its sign
    coef = rng.standard_normal((S, 8)) * (4.0 * 0.6 ** np.arange(8))
    Y = coef @ rng.standard_normal((8, n)) + 1e-4 * rng.standard_normal((S, n))
    Y += 3.0
    s = _sur(n_out=8, n_dof=n)
    sigma = s.fit_basis(to_dev(Y, torch.float64))
    mean, Phi, sig_ref = sg.pod_basis(Y, 8)
    assert np.min(sig_ref[:-1] / sig_ref[1:]) > 1.25
    assert len(sigma) == 8
    assert rel_l2(sigma, sig_ref) <= 1e-4
    A = to_np(s.coefficients(to_dev(Y, torch.float64)))
    A_ref = np.stack([sg.pod_coefficients(y, mean, Phi, sig_ref) for y in Y])
    # align signs column by column on the entry of largest magnitude
    for j in range(8):
        k = np.argmax(np.abs(A_ref[:, j]))
        if np.sign(A[k, j]) != np.sign(A_ref[k, j]):
            A[:, j] *= -1
    # the basis is stored in FP32: a coefficient along direction j picks up the
    # FP32 rounding of phi_j along the stronger directions, a relative error of
    # about u32 (sigma_1 / sigma_j); the bar scales with that ratio
    for j in range(8):
        tol = 1e-5 * sig_ref[0] / sig_ref[j]
        assert rel_l2(A[:, j], A_ref[:, j]) <= tol, (j, rel_l2(A[:, j], A_ref[:, j]), tol)


def _pipe_sample(rng, mesh):
    Re = float(rng.uniform(60.0, 140.0))
    U = cases.waveform_random(3, int(rng.integers(0, 2**31)), amp=0.4)
    case = cases.pipe_case(N=3, Re=Re, Wo=5.0, amps=tuple(U), mesh=mesh)
    x = cases.surrogate_inputs([U], Re, 5.0, harmonics=2)
    return case, x


def test_trained_guess_saves_newton_steps(torch):
    """Train on solves of the method, then compare held-out solves from the
    plain guess and from the surrogate: same tolerance, same field, fewer steps."""
    import paper_2311_09465_gb300 as ts
    mesh = mg.pipe(nc=3, nr=2, nz=10)
    rng = np.random.default_rng(6)
    # restart length 100 as in the paper; the pseudo-time step grows at most to 8, which
    # keeps the mass term in the tangent (GMRES(m) can stall on the pure Newton tangent)
    opts = dict(precision=32, tol=1e-8, max_steps=100, krylov=100, eps_ls=0.05, ser=1.0, dt_max=8.0)
    train_x, train_y = [], []
    for _ in range(40):
        case, x = _pipe_sample(rng, mesh)
        g = ts.GLSProblem(case, dt_pseudo=0.5)
        y = to_dev(case.y0, torch.float64)
        rep = g.solve(y, **opts)
        assert rep["status"] == 0
        train_x.append(x)
        train_y.append(y.reshape(-1))
        g.close()
    Y = torch.stack(train_y)
    n_dof = Y.shape[1]
    s = ts.Surrogate(len(train_x[0]), 128, 3, 16, n_dof, seed=7)
    s.fit_basis(Y)
    hist = s.train(np.array(train_x), Y, epochs=800, batch=20, lr=2e-3, seed=8)
    # the training loss falls (the held-out solves below are the real check)
    assert hist[-1] < 0.25 * hist[0], (hist[0], hist[-1])
    steps_plain, steps_sur = [], []
    for _ in range(4):
        case, x = _pipe_sample(rng, mesh)
        g = ts.GLSProblem(case, dt_pseudo=0.5)
        y0 = to_dev(case.y0, torch.float64)
        r_ref = float(g.residual(y0).norm())
        y_plain = y0.clone()
        rp = g.solve(y_plain, r_ref=r_ref, raise_on_noconv=False, **opts)
        y_sur = y0.clone()
        s.guess(g, x, y_sur)
        # Dirichlet data untouched by the guess
        dm = case.dirichlet_mask
        assert np.array_equal(to_np(y_sur)[dm, :3], case.y0[dm, :3])
        rs = g.solve(y_sur, r_ref=r_ref, raise_on_noconv=False, **opts)
        assert rp["status"] == 0, rp["hist"]
        assert rs["status"] == 0, rs["hist"]
        assert rel_l2(to_np(y_sur), to_np(y_plain)) <= 1e-6
        steps_plain.append(rp["steps"])
        steps_sur.append(rs["steps"])
        g.close()
    print(f"pseudo-time steps plain {steps_plain} surrogate {steps_sur}")
    assert sum(steps_sur) < sum(steps_plain)

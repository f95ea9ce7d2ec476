"""Pins of the oracle's surrogate operations (CPU, FP64).

Convolution gradients against central finite differences, the Adam step
against its closed form after one step (|update| = lr), and the
Chapman-Enskog reconstruction against its defining properties: conserved
moments equal the fields, f^eq is recovered for uniform fields, and the
non-equilibrium part of a shear flow carries the Navier-Stokes stress
-rho nu (du_x/dy) with nu = (1/omega - 1/2) theta.
"""
import numpy as np
import pytest

import oracle as O
from oracle import cnn as N


def _rand(shape, rng, s=1.0):
    return s * rng.standard_normal(shape)


def test_conv_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    X = _rand((2, 5, 6, 3), rng)
    W = _rand((3, 3, 3, 4), rng, 0.3)
    b = _rand(4, rng)
    G = _rand((2, 5, 6, 4), rng)  # upstream gradient of L = sum(G * Y)
    L = lambda X_, W_, b_: float(np.sum(G * N.conv3x3(X_, W_, b_)))
    dX = N.conv3x3_grad_input(G, W)
    dW, db = N.conv3x3_grad_weight(X, G)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 4, 5, 2), (0, 2, 3, 1), (1, 0, 5, 0)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[idx] += h
        Xm[idx] -= h
        fd = (L(Xp, W, b) - L(Xm, W, b)) / (2 * h)
        assert abs(fd - dX[idx]) <= 1e-7 * max(1.0, abs(fd))
    for idx in [(0, 0, 0, 0), (2, 2, 2, 3), (1, 0, 1, 2), (0, 2, 2, 1)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += h
        Wm[idx] -= h
        fd = (L(X, Wp, b) - L(X, Wm, b)) / (2 * h)
        assert abs(fd - dW[idx]) <= 1e-7 * max(1.0, abs(fd))
    for o in range(4):
        bp, bm = b.copy(), b.copy()
        bp[o] += h
        bm[o] -= h
        fd = (L(X, W, bp) - L(X, W, bm)) / (2 * h)
        assert abs(fd - db[o]) <= 1e-7 * max(1.0, abs(fd))


def test_network_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    chans = [3, 5, 5, 2]
    params = [(_rand((3, 3, a, c), rng, 0.4), _rand(c, rng, 0.1)) for a, c in zip(chans[:-1], chans[1:])]
    X = _rand((1, 4, 5, 3), rng)
    T = _rand((1, 4, 5, 2), rng)

    def loss(ps):
        out, _ = N.forward(ps, X, relu_layers=2)
        return N.mse(out, T)[0]

    out, acts = N.forward(params, X, relu_layers=2)
    _, dout = N.mse(out, T)
    grads = N.backward(params, acts, dout, relu_layers=2)
    h = 1e-6
    for li, idx in [(0, (1, 1, 0, 2)), (1, (0, 2, 4, 1)), (2, (2, 0, 3, 1)), (1, (1, 1, 1, 1))]:
        ps_p = [(W.copy(), b.copy()) for W, b in params]
        ps_m = [(W.copy(), b.copy()) for W, b in params]
        ps_p[li][0][idx] += h
        ps_m[li][0][idx] -= h
        fd = (loss(ps_p) - loss(ps_m)) / (2 * h)
        assert abs(fd - grads[li][0][idx]) <= 1e-6 * max(1e-3, abs(fd))


def test_adam_first_step_moves_by_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 7.0])
    p1, m, v = N.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=1e-2)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> update = lr * sign(g) (eps aside)
    assert np.allclose(p - p1, 1e-2 * np.sign(g), rtol=1e-4)


V5 = (0, 1, -1, 3, -3)


def _moments(f, v):
    vel = np.array([(a, b) for a in v for b in v], dtype=float)
    rho = f.sum(0)
    jx = np.einsum("q,qhw->hw", vel[:, 0], f)
    jy = np.einsum("q,qhw->hw", vel[:, 1], f)
    e = np.einsum("q,qhw->hw", (vel ** 2).sum(1), f)
    ux, uy = jx / rho, jy / rho
    return rho, ux, uy, (e / rho - ux * ux - uy * uy) / 2


def test_reconstruction_conserves_fields():
    rng = np.random.default_rng(2)
    H, W = 12, 16
    y = np.arange(H)[:, None] * 2 * np.pi / H
    x = np.arange(W)[None, :] * 2 * np.pi / W
    rho = 1 + 0.01 * np.sin(x) * np.cos(y)
    ux = 0.05 * np.sin(y) + 0.01 * np.cos(x)
    uy = 0.03 * np.cos(x + y)
    th = 1 + 0.02 * np.sin(2 * x)
    f = N.reconstruct(V5, 1.3, rho, ux, uy, th)
    r, a, b, t = _moments(f, V5)
    for got, ref in ((r, rho), (a, ux), (b, uy), (t, th)):
        assert np.max(np.abs(got - ref)) < 1e-13


def test_reconstruction_of_uniform_fields_is_equilibrium():
    H, W = 6, 7
    rho = np.full((H, W), 1.02)
    ux = np.full((H, W), 0.05)
    uy = np.full((H, W), -0.02)
    th = np.full((H, W), 0.95)
    f = N.reconstruct(V5, 1.3, rho, ux, uy, th)
    feq = O.feq(2, V5, 1.02, 0.05, -0.02, 0.95)
    assert np.max(np.abs(f - feq[:, None, None])) < 1e-15


def test_reconstruction_carries_navier_stokes_shear_stress():
    # For a shear u_x(y) the only first-order term of sum v_x v_y D_p f^eq is the flux
    # d_y(sum v_x v_y^2 f^eq) = d_y(rho theta u_x), so the stored populations carry
    # sum v_x v_y f = rho u_x u_y - ((1 - omega)/omega) rho theta du_x/dy.
    H, W, omega, theta = 64, 4, 1.3, 1.0
    y = np.arange(H)[:, None]
    ux = 0.01 * np.sin(2 * np.pi * y / H) * np.ones((1, W))
    rho = np.ones((H, W))
    f = N.reconstruct(V5, omega, rho, ux, np.zeros((H, W)), np.full((H, W), theta))
    vel = np.array([(a, b) for a in V5 for b in V5], dtype=float)
    pxy = np.einsum("q,qhw->hw", vel[:, 0] * vel[:, 1], f)
    dudy = 0.5 * (np.roll(ux, -1, axis=0) - np.roll(ux, 1, axis=0))
    expect = -((1 - omega) / omega) * rho * theta * dudy
    assert np.max(np.abs(pxy - expect)) < 1e-10 * np.max(np.abs(expect))


def test_reconstruction_recovers_most_of_the_lbm_nonequilibrium():
    # On a developed LBM state (the double shear layer after 500 steps) the
    # Chapman-Enskog reconstruction from the state's own fields carries the
    # non-equilibrium part: ||f - f_CE|| is a small fraction of ||f - f^eq||
    # (measured 0.014 at 64 x 64; 1.0 without the f^neq term, ~0.3 with
    # (1 - omega) in place of (1 - omega)/omega, 2.0 with the sign flipped).
    from paper_1402_5487_gb300 import inputs as I
    L, omega = 64, 1.3
    lat = O.Lattice(2, V5, omega, L, L, theta0=1.0)
    f = lat.run(lat.init(*I.kh_fields(L)), 500)
    rho, ux, uy, th = lat.moments(f)
    f_ce = N.reconstruct(V5, omega, rho, ux, uy, th)
    f_eq = lat.init(rho, ux, uy, th)
    ratio = np.linalg.norm(f - f_ce) / np.linalg.norm(f - f_eq)
    assert ratio < 0.05, ratio

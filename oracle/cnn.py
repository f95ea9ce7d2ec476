"""FP64 reference of the surrogate network's operations (NumPy).

TEST INFRASTRUCTURE ONLY (part of the oracle).

The surrogate (a 6-layer 3x3 CNN on the fields rho, u_x, u_y, theta of a
periodic lattice) is not part of the paper; these are the textbook definitions
its CUDA kernels must reproduce:

* conv3x3 with circular padding (cross-correlation, NHWC):
  Y[b, y, x, o] = bias[o] + sum_{ky, kx, i} X[b, (y + ky - 1) % H, (x + kx - 1) % W, i] W[ky, kx, i, o]
* its gradients with respect to X, W and bias for an upstream gradient dY;
* ReLU, mean squared error, and one Adam step (Kingma & Ba 2015).

Chapman-Enskog reconstruction of populations from fields (Sec. 2.1 gives the
Navier-Stokes level of the model) is in ``reconstruct``.
"""
from __future__ import annotations

import numpy as np


def conv3x3(X, W, bias=None):
    """X: (B, H, W, Cin), W: (3, 3, Cin, Cout) -> (B, H, W, Cout), circular padding."""
    B, H, Wd, _ = X.shape
    out = np.zeros((B, H, Wd, W.shape[3]))
    for ky in range(3):
        for kx in range(3):
            Xs = np.roll(np.roll(X, -(ky - 1), axis=1), -(kx - 1), axis=2)
            out += Xs @ W[ky, kx]
    if bias is not None:
        out += bias
    return out


def conv3x3_grad_input(dY, W):
    """dL/dX for Y = conv3x3(X, W)."""
    dX = np.zeros(dY.shape[:3] + (W.shape[2],))
    for ky in range(3):
        for kx in range(3):
            g = dY @ W[ky, kx].T  # contribution at the shifted input position
            dX += np.roll(np.roll(g, ky - 1, axis=1), kx - 1, axis=2)
    return dX


def conv3x3_grad_weight(X, dY):
    """dL/dW and dL/dbias for Y = conv3x3(X, W) + bias."""
    Cin, Cout = X.shape[3], dY.shape[3]
    dW = np.zeros((3, 3, Cin, Cout))
    Xf = X.reshape(-1, Cin)
    for ky in range(3):
        for kx in range(3):
            Xs = np.roll(np.roll(X, -(ky - 1), axis=1), -(kx - 1), axis=2).reshape(-1, Cin)
            dW[ky, kx] = Xs.T @ dY.reshape(-1, Cout)
    db = dY.reshape(-1, Cout).sum(axis=0)
    del Xf
    return dW, db


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, X, relu_layers=5):
    """Network forward; params = [(W, b), ...]; returns output and the list of layer inputs."""
    acts = [X]
    h = X
    for i, (W, b) in enumerate(params):
        h = conv3x3(h, W, b)
        if i < relu_layers:
            h = relu(h)
        acts.append(h)
    return h, acts


def backward(params, acts, dOut, relu_layers=5):
    """Gradients of every (W, b) for the upstream gradient dOut of the network output."""
    grads = [None] * len(params)
    g = dOut
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        dW, db = conv3x3_grad_weight(acts[i], g)
        grads[i] = (dW, db)
        if i > 0:
            g = conv3x3_grad_input(g, W)
            if i - 1 < relu_layers:
                g = g * (acts[i] > 0)
    return grads


def mse(pred, target):
    d = pred - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def reconstruct(v, omega, rho, ux, uy, theta, theta0=1.0):
    """Chapman-Enskog populations of the stored (post-collision) state, FP64.

    f_p = f^eq_p - ((1 - omega)/omega) D_p f^eq_p with D_p = d_t + v_p . grad,
    d_t from the Euler equations of p = rho theta in 2D, central differences on
    the periodic grid, then the non-equilibrium part projected off
    span{w0, w0 v_x, w0 v_y, w0 |v|^2} (w0 = f^eq(1, 0, theta0)) so that the
    conserved moments equal the fields.  Returns (q, H, W), p = i q1 + j.
    """
    from . import feq as _feq, vandermonde_inverse
    C = vandermonde_inverse(v)
    q1 = len(v)
    dx = lambda a: 0.5 * (np.roll(a, -1, axis=1) - np.roll(a, 1, axis=1))
    dy = lambda a: 0.5 * (np.roll(a, -1, axis=0) - np.roll(a, 1, axis=0))
    p = rho * theta
    divu = dx(ux) + dy(uy)
    dt = {
        "rho": -(ux * dx(rho) + uy * dy(rho)) - rho * divu,
        "ux": -(ux * dx(ux) + uy * dy(ux)) - dx(p) / rho,
        "uy": -(ux * dx(uy) + uy * dy(uy)) - dy(p) / rho,
        "th": -(ux * dx(theta) + uy * dy(theta)) - theta * divu,
    }
    grads = {"rho": (dx(rho), dy(rho)), "ux": (dx(ux), dy(ux)), "uy": (dx(uy), dy(uy)),
             "th": (dx(theta), dy(theta))}

    def rules(u):
        mu = [np.ones_like(u), u]
        for n in range(1, q1 - 1):
            mu.append(u * mu[n] + n * theta * mu[n - 1])
        r = [sum(C[i, n] * mu[n] for n in range(q1)) for i in range(q1)]
        ru = [sum(C[i, n] * n * mu[n - 1] for n in range(1, q1)) for i in range(q1)]
        rt = [sum(C[i, n] * 0.5 * n * (n - 1) * mu[n - 2] for n in range(2, q1)) for i in range(q1)]
        return r, ru, rt

    rx, rxu, rxt = rules(ux)
    ry, ryu, ryt = rules(uy)
    w0 = _feq(2, v, 1.0, 0.0, 0.0, theta0)
    H, W = rho.shape
    f = np.zeros((q1 * q1, H, W))
    fneq = np.zeros((q1 * q1, H, W))
    coef = (1.0 - omega) / omega
    for i in range(q1):
        for j in range(q1):
            k = i * q1 + j
            D = lambda name: dt[name] + v[i] * grads[name][0] + v[j] * grads[name][1]
            Df = (rx[i] * ry[j] * D("rho") + rho * rxu[i] * ry[j] * D("ux") + rho * rx[i] * ryu[j] * D("uy")
                  + rho * (rxt[i] * ry[j] + rx[i] * ryt[j]) * D("th"))
            fneq[k] = -coef * Df
            f[k] = rho * rx[i] * ry[j]
    vel = np.array([(a, b) for a in v for b in v], dtype=float)
    basis = np.stack([np.ones(len(vel)), vel[:, 0], vel[:, 1], (vel ** 2).sum(1)])  # (4, q)
    G = (basis * w0) @ basis.T
    m = np.einsum("kq,qhw->khw", basis, fneq)
    c = np.einsum("ak,khw->ahw", np.linalg.inv(G), m)
    fneq = fneq - np.einsum("q,aq,ahw->qhw", w0, basis, c)
    return f + fneq

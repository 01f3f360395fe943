"""FP64 reference of the learned-window network (test infrastructure only).

The network maps normalised inputs u = (u_x, u_nu) to four standardised
window targets through three tanh layers of width 64:

    h1 = tanh(W1 u + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3),
    y  = W4 h3 + b4,

with loss L = mean over the batch and the four outputs of (y - t)^2.  The
parameters are one flat float array in the order W1 (64x2), b1, W2 (64x64),
b2, W3 (64x64), b3, W4 (4x64), b4, each W row-major as W[out, in].  Forward
and backward are plain numpy in float64, written from the definitions above
(chain rule; d tanh(a)/da = 1 - tanh(a)^2); the tests check the backward pass
against central finite differences of the forward pass.
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = 64
SHAPES = [(HIDDEN, 2), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,),
          (4, HIDDEN), (4,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)  # 8772

# Input normalisation: log x over [ln 1e-3, ln 140] and nu over [0.05, 20]
# mapped affinely onto [-1, 1].
LOGX_LO, LOGX_HI = math.log(1e-3), math.log(140.0)
NU_LO, NU_HI = 0.05, 20.0


def normalise_inputs(x, nu):
    ux = (np.log(np.asarray(x, dtype=np.float64)) - 0.5 * (LOGX_LO + LOGX_HI)) / (0.5 * (LOGX_HI - LOGX_LO))
    un = (np.asarray(nu, dtype=np.float64) - 0.5 * (NU_LO + NU_HI)) / (0.5 * (NU_HI - NU_LO))
    return np.stack([ux, un], axis=1)


def targets_from_labels(labels):
    """Raw targets (t*, t* - t0, t1 - t*, ln N) from oracle window labels
    (rows t*, t0, t1, g(t*), N, ...)."""
    lab = np.asarray(labels, dtype=np.float64)
    return np.stack([lab[:, 0], lab[:, 0] - lab[:, 1], lab[:, 2] - lab[:, 0], np.log(lab[:, 4])],
                    axis=1)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(p[o:o + k].reshape(s))
        o += k
    return out


def forward(p, U):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    U = np.asarray(U, dtype=np.float64)
    h1 = np.tanh(U @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    h3 = np.tanh(h2 @ W3.T + b3)
    y = h3 @ W4.T + b4
    return y, (U, h1, h2, h3)


def loss_and_grad(p, U, T):
    """Mean squared error and its gradient with respect to the flat parameters."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    y, (U, h1, h2, h3) = forward(p, U)
    T = np.asarray(T, dtype=np.float64)
    B = U.shape[0]
    r = y - T
    loss = float(np.mean(r * r))
    dy = 2.0 * r / (B * 4)
    gW4 = dy.T @ h3
    gb4 = dy.sum(0)
    d3 = (dy @ W4) * (1.0 - h3 * h3)
    gW3 = d3.T @ h2
    gb3 = d3.sum(0)
    d2 = (d3 @ W3) * (1.0 - h2 * h2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    gW1 = d1.T @ U
    gb1 = d1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])
    return loss, g


def loss_only(p, U, T):
    y, _ = forward(p, U)
    r = y - np.asarray(T, dtype=np.float64)
    return float(np.mean(r * r))

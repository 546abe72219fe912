"""Oracle of the learned shape-parameter warm start (not in the paper).

The paper searches eps per stencil (Section 5).  The learned part predicts
that eps from the stencil's tangent-plane geometry and hands it to the
search as a first guess; the search stays the arbiter.  Definitions, in
float64:

Features of a stencil P = (x_1 .. x_n) with unit normal nh at the centre
x_1 (offsets d_j = x_j - x_1, radius r_s = max_j |d_j|):
  * orientation: if sum_j nh . d_j > 0, nh is replaced by -nh (the search is
    blind to the normal's sign, Eq. proj_mat uses nh nh^T);
  * t1 = d_2 - (nh . d_2) nh normalised (d_2 is the nearest neighbour),
    t2 = nh x t1;
  * x = [(t1.d_j, t2.d_j, nh.d_j) / r_s for j = 1..n], length 3n.
Target: log(eps * r_s).

Network: 3n -> 64 -> 64 -> 1, GELU(z) = z/2 (1 + erf(z / sqrt 2)) on both
hidden layers, linear output.  Loss: mean squared error over the batch.
Optimiser: Adam (Kingma & Ba 2015) with bias correction.

Pins: tests/test_oracle_mlp.py (central finite differences of the loss
against the analytic backward pass; features invariant under rigid motion
and normal sign; Adam's first step equals lr * sign(g)).
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = 64


def features(P: np.ndarray, nh: np.ndarray) -> tuple[np.ndarray, float]:
    """(3n feature vector, r_s) of one stencil, as defined above."""
    d = P - P[0]
    r_s = float(np.sqrt(np.max(np.sum(d * d, axis=1))))
    nh = nh / np.linalg.norm(nh)
    if float(np.sum(d @ nh)) > 0.0:
        nh = -nh
    t1 = d[1] - (nh @ d[1]) * nh
    t1 = t1 / np.linalg.norm(t1)
    t2 = np.cross(nh, t1)
    F = np.stack([d @ t1, d @ t2, d @ nh], axis=1) / r_s
    return F.reshape(-1), r_s


def gelu(z):
    return 0.5 * z * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def forward(params: dict, x: np.ndarray):
    """x (B, D) -> (y (B,), cache)."""
    z1 = x @ params["W1"] + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"] + params["b2"]
    h2 = gelu(z2)
    y = h2 @ params["W3"][:, 0] + params["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss_and_grads(params: dict, x: np.ndarray, t: np.ndarray):
    """MSE loss and its gradient with respect to every parameter."""
    B = x.shape[0]
    y, (x, z1, h1, z2, h2) = forward(params, x)
    r = y - t
    loss = float(np.mean(r * r))
    dy = (2.0 / B) * r                       # dL/dy
    g = {}
    g["W3"] = (h2.T @ dy)[:, None]
    g["b3"] = np.array([dy.sum()])
    dz2 = np.outer(dy, params["W3"][:, 0]) * gelu_grad(z2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ params["W2"].T) * gelu_grad(z1)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam_step(params: dict, grads: dict, state: dict, lr=1e-3, b1=0.9,
              b2=0.999, eps=1e-8):
    """One Adam update in place; ``state`` holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = b1 * m + (1.0 - b1) * grads[k]
        v[...] = b2 * v + (1.0 - b2) * grads[k] * grads[k]
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)

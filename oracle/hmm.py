"""Rigidness E-step and depth confidence.

Sec. III-A "Hierarchical Propagation Scheme": in the E-step hidden Markov
chain smoothing is imposed on the rigidness maps along the same 1-D chains,
with the forward-backward algorithm.  Eq. 6: the confidence of the depth map
is the pixel-wise average of the rigidness of all flows and priors used.

Reading fixed here:
  * two states per pixel and flow: 0 = outlier, 1 = rigid (inlier).
  * transition: keep the state with probability gamma, switch with 1 - gamma;
    initial distribution (1/2, 1/2).
  * emissions at the new depth: rigid -> p1(residual) (fisk.residual_density),
    outlier -> P0; a term without observation has both emissions P0, an
    observed term whose point is behind camera t has rigid emission 0.
  * chains are rows for directions 0/2 and columns for 1/3 (the posterior of
    a symmetric chain does not depend on which end it is walked from).
  * the prior's rigidness q_hat is the isolated posterior
    e1_hat / (e1_hat + e0_hat) at the new depth (0 at prior holes).
  * C = (sum_t q_t + q_hat) / (N + 1) with a prior, sum_t q_t / N without.
"""
from __future__ import annotations

import numpy as np

from . import model


def forward_backward(e1, e0, gamma):
    """Posterior P(state = 1) for chains of emissions e1, e0 with shape [L, ...].

    Plain normalised forward and backward recursions along axis 0."""
    e1 = np.asarray(e1, np.float64)
    e0 = np.asarray(e0, np.float64)
    L = e1.shape[0]
    g, h = gamma, 1.0 - gamma
    a0 = np.empty_like(e1)
    a1 = np.empty_like(e1)
    x0, x1 = 0.5 * e0[0], 0.5 * e1[0]
    s = x0 + x1
    a0[0], a1[0] = x0 / s, x1 / s
    for m in range(1, L):
        x0 = (a0[m - 1] * g + a1[m - 1] * h) * e0[m]
        x1 = (a0[m - 1] * h + a1[m - 1] * g) * e1[m]
        s = x0 + x1
        a0[m], a1[m] = x0 / s, x1 / s
    b0 = np.empty_like(e1)
    b1 = np.empty_like(e1)
    b0[L - 1] = 1.0
    b1[L - 1] = 1.0
    for m in range(L - 2, -1, -1):
        y0 = e0[m + 1] * b0[m + 1]
        y1 = e1[m + 1] * b1[m + 1]
        x0 = g * y0 + h * y1
        x1 = h * y0 + g * y1
        s = x0 + x1
        b0[m], b1[m] = x0 / s, x1 / s
    p1 = a1 * b1
    p0 = a0 * b0
    return p1 / (p0 + p1)


def rigidness_estep(P, S: model.State, rho_new, direction, p):
    """Returns (q [N, H, W] float32, q_hat [H, W] float32, C [H, W] float32)."""
    iu, iv = model.pixel_grid(P)
    _, e1, _ = model.flow_terms(P, S.G, iu, iv, rho_new, p)      # [N, H, W]
    e0 = np.full_like(e1, p.outlier_density)
    q = np.empty((P.N, P.H, P.W), np.float32)
    for t in range(P.N):
        if direction in (0, 2):     # rows: chain axis is u (axis 1)
            post = forward_backward(e1[t].T, e0[t].T, p.gamma_stay).T
        else:                       # columns: chain axis is v (axis 0)
            post = forward_backward(e1[t], e0[t], p.gamma_stay)
        q[t] = post.astype(np.float32)
    if P.prior_kind != "none":
        _, e1h, e0h, valid = model.prior_terms(P, iu, iv, rho_new, p)
        qh = np.where(valid, e1h / (e1h + e0h), 0.0)
        qhat = qh.astype(np.float32)
        C = (q.astype(np.float64).sum(0) + qhat) / (P.N + 1)
    else:
        qhat = np.zeros((P.H, P.W), np.float32)
        C = q.astype(np.float64).sum(0) / P.N
    return q, qhat, C.astype(np.float32)

"""Monocular bootstrap: the essential matrix of X_1 by the 8-point method.

VOLDOR+ bootstraps from monocular capture (Sec. I, Sec. III-A); without a
prior the first relative pose comes from the epipolar constraint of the first
flow field.  Textbook linear 8-point estimate (Longuet-Higgins 1981; Hartley &
Zisserman, Alg. 11.1 and Result 9.19) on calibrated rays:
  * every pixel j of frame 0 gives a = K^-1 (u, v, 1), b = K^-1 (u + X_1, v + Y_1, 1)
    and the linear equation b^T E a = 0 in the nine entries of E (row-major);
  * E = the eigenvector of the smallest eigenvalue of M = sum_j r_j r_j^T;
  * E = U diag(s) V^T with det U = det V = +1 gives two rotations U W V^T,
    U W^T V^T and the translation direction +-U[:, 2];
  * flow noise is Fisk distributed (heavy tailed, infinite variance for
    beta <= 2), so the estimate is iteratively re-weighted: IRLS_ITERS rounds
    of the weighted normal matrix M = sum_j w_j r_j r_j^T, with w_j = 1 after
    the first and w_j = 1 / (1 + (d_j / alpha0)^2) from the Sampson distance
    d_j (in pixels, f = sqrt(fx fy)) of the previous E -- the IRLS weight of a
    residual density proportional to (1 + d^2 / alpha^2)^-2, the beta = 2
    case of the residual model;
  * of the four motions, keep the one with most pixels triangulated in front
    of both cameras (first on ties); |tau_1| = 1 fixes the monocular scale.
"""
from __future__ import annotations

import numpy as np

from . import model

WMAT = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])


IRLS_ITERS = 8


def normal_matrix(P: model.Problem):
    iu, iv = model.pixel_grid(P)
    a = P.rays.reshape(-1, 3)
    fx, fy, cx, cy = P.K
    F = P.flow[0].astype(np.float64).reshape(-1, 2)
    u1 = iu.ravel() + F[:, 0]
    v1 = iv.ravel() + F[:, 1]
    b = np.stack([(u1 - cx) / fx, (v1 - cy) / fy, np.ones_like(u1)], axis=1)
    rows = (b[:, :, None] * a[:, None, :]).reshape(-1, 9)
    return rows.T @ rows, a, b


def candidates(E):
    U, _, Vt = np.linalg.svd(E)
    if np.linalg.det(U) < 0:
        U = -U
    if np.linalg.det(Vt) < 0:
        Vt = -Vt
    R1 = U @ WMAT @ Vt
    R2 = U @ WMAT.T @ Vt
    t = U[:, 2]
    return [(R1, t), (R1, -t), (R2, t), (R2, -t)]


def cheirality_count(R, t, a, b):
    """Pixels whose least-squares triangulation lam_b b = lam_a R a + t has
    both depths positive."""
    Ra = a @ R.T
    # normal equations of [Ra, -b] [lam_a, lam_b]^T = -t
    m11 = np.sum(Ra * Ra, 1)
    m12 = -np.sum(Ra * b, 1)
    m22 = np.sum(b * b, 1)
    r1 = -(Ra @ t)
    r2 = b @ t
    det = m11 * m22 - m12 * m12
    with np.errstate(divide="ignore", invalid="ignore"):
        la = (m22 * r1 - m12 * r2) / det
        lb = (m11 * r2 - m12 * r1) / det
    return int(np.sum((la > 0) & (lb > 0)))


def sampson_px(E, a, b, f):
    Ea = a @ E.T
    Etb = b @ E
    num = np.sum(b * Ea, 1)
    den = Ea[:, 0] ** 2 + Ea[:, 1] ** 2 + Etb[:, 0] ** 2 + Etb[:, 1] ** 2
    return f * np.abs(num) / np.sqrt(np.maximum(den, 1e-300))


def essential(P: model.Problem, alpha0):
    """IRLS estimate of E (row-major 3x3, unit Frobenius norm)."""
    _, a, b = normal_matrix(P)
    rows = (b[:, :, None] * a[:, None, :]).reshape(-1, 9)
    f = np.sqrt(P.K[0] * P.K[1])
    w = np.ones(len(rows))
    for _ in range(IRLS_ITERS):
        M = (rows * w[:, None]).T @ rows
        _, V = np.linalg.eigh(M)
        E = V[:, 0].reshape(3, 3)
        d = sampson_px(E, a, b, f)
        w = 1.0 / (1.0 + (d / alpha0) ** 2)
    return E, a, b


def bootstrap_pose(P: model.Problem, alpha0=0.5):
    """Returns (G_1 as [3, 4] with |tau| = 1, the four counts)."""
    E, a, b = essential(P, alpha0)
    cands = candidates(E)
    counts = [cheirality_count(R, t, a, b) for R, t in cands]
    k = int(np.argmax(counts))
    R, t = cands[k]
    return np.concatenate([R, (t / np.linalg.norm(t))[:, None]], axis=1), counts

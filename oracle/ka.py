"""Keyframe alignment: point-to-plane registration of two depth maps in
inverse-depth form, solved by Levenberg-Marquardt (test infrastructure).

Sec. III-C "Keyframe Alignment" (Eq. 9-12): the relative motion T and scale
s between the depth maps theta_1 and theta_2 of two keyframes minimise
E_geo = sum_j C^j psi(<n(theta_1^l), phi(theta_1^l, I) - phi(theta_2^j, T)>
                      / (s theta_1^l phi_z(theta_2^j, T)))
with psi the Cauchy kernel, n the normal of depth map 1, C the confidence
of Eq. 6; s = 1 for depth of absolute scale; the covariance of T is
(J^T J)^-1.  The photometric term (Eq. 11) is optional and not used.

Readings fixed here (the paper leaves them open):
  * T maps keyframe-2 coordinates to keyframe-1 coordinates (3x4); a
    pixel j of keyframe 2 with depth theta_2 is the point
    P2 = R theta_2 r_j + t, r_j = ((u - cx)/fx, (v - cy)/fy, 1); it is
    associated with the nearest pixel l of its projection into keyframe 1
    (floor(x + 1/2), floor(y + 1/2), in front when P2_z > 1e-6, inside the
    image), and the association is redone at every evaluation.
  * keyframe 1's point at l is s theta_1^l r_l: s scales depth map 1, as in
    the inverse-depth difference 1/(s theta_1^l) - 1/phi_z of Eq. 9.
  * occlusion gate: the pair counts only when the depths agree,
    |P2_z - s theta_1^l| <= GATE s theta_1^l (GATE = 0.2).  A point of
    keyframe 2 hidden in keyframe 1 lands on the occluding surface; left to
    the Cauchy kernel alone, such pairs (about 2 % of a street scene) move
    the minimum away from the true pose (1e-2 rad on the driving scene),
    because a pose that pushes them out of the image or onto pixels without
    a normal lowers E.  0.1 rejects too many true pairs from a start whose
    scale is 10 % off; from 0.3 up occluded pairs bias the driving scene
    again (6e-4 rad).
  * the residual r_j = <n_l, s theta_1^l r_l - P2> / (s theta_1^l P2_z).
  * the normal n_l of depth map 1: the cross product of the central
    differences of its points, (P(u+1,v) - P(u-1,v)) x (P(u,v+1) - P(u,v-1)),
    normalised and turned towards the camera (<n, P> < 0); none at the
    border, next to an invalid depth, for a zero cross product, or at a
    depth edge or fold: where a second difference of the points,
    |P(u+1,v) - 2 P(u,v) + P(u-1,v)| (and the same along v), exceeds
    KINK = 0.2 of the central span |P(u+1,v) - P(u-1,v)| (a fold sharper
    than 23 degrees, any depth jump; white pixel-scale depth noise of
    relative size e gives about 1.2 e f of the span, f the focal length in
    pixels, so the maps must be smooth at the pixel scale, as propagated EM
    depth is).  A normal across an edge mixes two surfaces; its residual is
    not zero at the true pose and biases the alignment (1.4e-4 rad on the
    four-plane scene without the test, 1.7e-5 at 0.25, 3e-7 at 0.2).
  * valid depth: finite and > 0; confidence C^j of keyframe 2's pixel j
    (1 without a map).
  * Cauchy kernel psi(r) = (c^2/2) log(1 + r^2/c^2); Gauss-Newton weights
    w = C psi'(r)/r = C / (1 + r^2/c^2).
  * parameters: a left increment xi in se(3) of T (T <- exp(xi) T) and
    sigma = log s (left out with a fixed scale).  Levenberg-Marquardt: with
    H = sum w J J^T and g = sum w J r at the current estimate, the step
    solves (H + lambda diag(H)) delta = -g; it is taken when it lowers E
    (lambda /= 10) and refused otherwise (lambda *= 10); lambda starts at
    1e-3; stop after max_iters evaluations of a step, when |delta| < 1e-10,
    or when lambda > 1e10.
  * covariance: the pose block (6 x 6, rotation first) of H^-1 at the
    estimate.
  * float64.
"""
from __future__ import annotations

import numpy as np

from . import geometry

Z_EPS = 1e-6
KINK = 0.2
GATE = 0.2
LAMBDA0 = 1e-3
STEP_TOL = 1e-10


def rays(W, H, K):
    fx, fy, cx, cy = K
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    return np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=-1)


def valid_depth(theta):
    theta = np.asarray(theta, np.float64)
    with np.errstate(invalid="ignore"):
        return np.isfinite(theta) & (theta > 0)


def normals(theta1, K):
    """(n [H][W][3], ok [H][W]) of depth map 1."""
    H, W = theta1.shape
    ok_d = valid_depth(theta1)
    P = np.where(ok_d[..., None], np.asarray(theta1, np.float64)[..., None] * rays(W, H, K), 0.0)
    n = np.zeros((H, W, 3))
    ok = np.zeros((H, W), bool)
    dx = P[1:-1, 2:] - P[1:-1, :-2]
    dy = P[2:, 1:-1] - P[:-2, 1:-1]
    c = np.cross(dx, dy)
    nrm = np.linalg.norm(c, axis=-1)
    ddx = np.linalg.norm(P[1:-1, 2:] - 2 * P[1:-1, 1:-1] + P[1:-1, :-2], axis=-1)
    ddy = np.linalg.norm(P[2:, 1:-1] - 2 * P[1:-1, 1:-1] + P[:-2, 1:-1], axis=-1)
    smooth = (ddx <= KINK * np.linalg.norm(dx, axis=-1)) & (ddy <= KINK * np.linalg.norm(dy, axis=-1))
    inner = (ok_d[1:-1, 2:] & ok_d[1:-1, :-2] & ok_d[2:, 1:-1] & ok_d[:-2, 1:-1] &
             ok_d[1:-1, 1:-1] & (nrm > 0) & smooth)
    c = np.where(inner[..., None], c / np.where(nrm > 0, nrm, 1.0)[..., None], 0.0)
    flip = np.sum(c * P[1:-1, 1:-1], axis=-1) > 0
    c[flip] *= -1.0
    n[1:-1, 1:-1] = c
    ok[1:-1, 1:-1] = inner
    return n, ok


def residuals(theta1, n1, ok1, theta2, conf2, K, T, s, jac=False, assoc_out=None):
    """Residuals of every associated pixel of keyframe 2, their confidences
    and (with jac) the 7-column Jacobian d r / d(xi, log s); assoc_out (a
    list) receives (pixel index of keyframe 2, l) of every residual."""
    H, W = theta2.shape
    fx, fy, cx, cy = K
    T = np.asarray(T, np.float64)
    ok2 = valid_depth(theta2)
    X2 = np.asarray(theta2, np.float64)[..., None] * rays(W, H, K)
    P2 = X2 @ T[:, :3].T + T[:, 3]
    front = ok2 & (P2[..., 2] > Z_EPS)
    z = np.where(front, P2[..., 2], 1.0)
    x = fx * P2[..., 0] / z + cx
    y = fy * P2[..., 1] / z + cy
    with np.errstate(invalid="ignore"):
        inside = front & (x >= 0) & (x <= W - 1) & (y >= 0) & (y <= H - 1)
    li = np.where(inside, np.floor(y + 0.5), 0).astype(np.int64)
    lj = np.where(inside, np.floor(x + 0.5), 0).astype(np.int64)
    th1 = np.asarray(theta1, np.float64)[li, lj]
    with np.errstate(invalid="ignore"):
        agree = np.abs(P2[..., 2] - s * th1) <= GATE * s * th1
    assoc = inside & ok1[li, lj] & valid_depth(th1) & agree
    idx = np.nonzero(assoc)
    if assoc_out is not None:
        assoc_out.append((idx[0] * W + idx[1], li[idx] * W + lj[idx]))
    P = P2[idx]
    n = n1[li[idx], lj[idx]]
    t1 = th1[idx]
    rl = rays(W, H, K)[li[idx], lj[idx]]
    Z = P[:, 2]
    D = s * t1
    A = np.sum(n * rl, axis=1)                      # <n, r_l>
    B = np.sum(n * P, axis=1)                       # <n, P2>
    r = A / Z - B / (D * Z)                         # = <n, D r_l - P2> / (D Z)
    C = np.ones(len(r)) if conf2 is None else np.asarray(conf2, np.float64)[idx]
    if not jac:
        return r, C, None
    # d r / d P2 = -n / (D Z) + e_z (B - A D) / (D Z^2); d P2 / d xi = [-[P2]x | I]
    drdP = -n / (D * Z)[:, None]
    drdP[:, 2] += (B - A * D) / (D * Z * Z)
    J = np.zeros((len(r), 7))
    J[:, :3] = np.cross(P, drdP)                    # (-[P]x)^T g = P x g
    J[:, 3:6] = drdP
    J[:, 6] = B / (D * Z)                           # d r / d log s
    return r, C, J


def cauchy(r, c):
    return 0.5 * c * c * np.log1p((r / c) ** 2)


def energy(theta1, n1, ok1, theta2, conf2, K, T, s, c):
    r, C, _ = residuals(theta1, n1, ok1, theta2, conf2, K, T, s)
    return float(np.sum(C * cauchy(r, c))), len(r)


def normal_equations(theta1, n1, ok1, theta2, conf2, K, T, s, c, fix_scale):
    r, C, J = residuals(theta1, n1, ok1, theta2, conf2, K, T, s, jac=True)
    if fix_scale:
        J = J[:, :6]
    w = C / (1.0 + (r / c) ** 2)
    Hm = (J * w[:, None]).T @ J
    g = J.T @ (w * r)
    return float(np.sum(C * cauchy(r, c))), Hm, g, len(r)


def align(theta1, theta2, K, T0, s0=1.0, conf2=None, c=0.01, fix_scale=False, max_iters=50):
    """dict(T, s, cov (6x6), energy, iterations, n_valid)."""
    n1, ok1 = normals(theta1, K)
    T = np.array(T0, np.float64)
    s = 1.0 if fix_scale else float(s0)
    lam = LAMBDA0
    E, Hm, g, n = normal_equations(theta1, n1, ok1, theta2, conf2, K, T, s, c, fix_scale)
    it = 0
    while it < max_iters and lam <= 1e10 and n > 0:
        it += 1
        A = Hm + lam * np.diag(np.diag(Hm))
        try:
            delta = -np.linalg.solve(A, g)
        except np.linalg.LinAlgError:
            lam *= 10.0
            continue
        Tn = geometry.compose(geometry.se3_exp(delta[:6]), T)
        sn = s if fix_scale else s * np.exp(delta[6])
        En, Hn, gn, nn = normal_equations(theta1, n1, ok1, theta2, conf2, K, Tn, sn, c, fix_scale)
        if nn > 0 and En < E:
            T, s, E, Hm, g, n = Tn, sn, En, Hn, gn, nn
            lam /= 10.0
        else:
            lam *= 10.0
        if np.linalg.norm(delta) < STEP_TOL:
            break
    cov = np.linalg.inv(Hm)[:6, :6] if n > 0 else np.full((6, 6), np.nan)
    return dict(T=T, s=s, cov=cov, energy=E, iterations=it, n_valid=n)

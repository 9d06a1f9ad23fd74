"""Camera geometry for the oracle: projection, bilinear flow sampling, SE(3).

Conventions: pixel (u, v) with u the column; ray r = ((u-cx)/fx, (v-cy)/fy, 1);
absolute pose G_t = (R_t, tau_t) maps frame-0 coordinates to frame t.  A point
of reference pixel j with inverse depth rho is X_0 = r_j / rho, so its frame-t
image is pi(K (R_t r_j + rho tau_t)) -- the homogeneous form that needs no
division by rho (Sec. III-A: the rigid flow implied by depth and pose).
"""
from __future__ import annotations

import math

import numpy as np

Z_EPS = 1e-6   # a homogeneous z at or below this is "behind the camera"


def rays(W, H, K):
    fx, fy, cx, cy = K
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    return np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=-1)


def project_h(K, G, r, rho):
    """Homogeneous image point h = K (R r + rho tau) for rays r[..., 3], rho[...]."""
    fx, fy, cx, cy = K
    R, tau = G[:, :3], G[:, 3]
    X = r @ R.T + np.asarray(rho, np.float64)[..., None] * tau
    return np.stack([fx * X[..., 0] + cx * X[..., 2], fy * X[..., 1] + cy * X[..., 2], X[..., 2]],
                    axis=-1)


def dehom(h):
    """(x, y, front) with front = h_z > Z_EPS; x, y are NaN when not in front."""
    front = h[..., 2] > Z_EPS
    with np.errstate(divide="ignore", invalid="ignore"):
        x = np.where(front, h[..., 0] / h[..., 2], np.nan)
        y = np.where(front, h[..., 1] / h[..., 2], np.nan)
    return x, y, front


def inside(x, y, W, H):
    """Sample position inside the image: 0 <= x <= W-1 and 0 <= y <= H-1."""
    with np.errstate(invalid="ignore"):
        return (x >= 0) & (x <= W - 1) & (y >= 0) & (y <= H - 1)


def bilinear(F, x, y):
    """Bilinear sample of F[H, W, C] at (x, y); positions must be inside.

    The taps are (x0, y0) .. (x0+1, y0+1) with x0 = min(floor(x), W-2), so the
    last row/column is reached with weight 1 and no tap leaves the image."""
    H, W = F.shape[:2]
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    x0 = np.minimum(np.floor(x), W - 2).astype(np.int64)
    y0 = np.minimum(np.floor(y), H - 2).astype(np.int64)
    ax = (x - x0)[..., None]
    ay = (y - y0)[..., None]
    F = F.astype(np.float64)
    f00 = F[y0, x0]
    f01 = F[y0, x0 + 1]
    f10 = F[y0 + 1, x0]
    f11 = F[y0 + 1, x0 + 1]
    return (1 - ay) * ((1 - ax) * f00 + ax * f01) + ay * ((1 - ax) * f10 + ax * f11)


# ----------------------------------------------------------------------------
# SE(3): poses as [3, 4] = [R | tau]; tangent vectors xi = (omega, v)
# ----------------------------------------------------------------------------
def hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def so3_exp(w):
    th = float(np.linalg.norm(w))
    Kx = hat(w)
    if th < 1e-8:
        return np.eye(3) + Kx + 0.5 * Kx @ Kx
    return np.eye(3) + math.sin(th) / th * Kx + (1 - math.cos(th)) / th ** 2 * Kx @ Kx


def so3_log(R):
    c = (np.trace(R) - 1.0) / 2.0
    v = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]]) / 2.0
    s = float(np.linalg.norm(v))
    th = math.atan2(s, c)
    if s < 1e-8:
        if c > 0:
            return v * (1.0 + th * th / 6.0)
        # rotation by pi: axis from the symmetric part
        B = (R + np.eye(3)) / 2.0
        k = int(np.argmax(np.diag(B)))
        a = B[:, k] / math.sqrt(max(B[k, k], 1e-300))
        return a * math.pi
    return v * (th / s)


def _V(w):
    th = float(np.linalg.norm(w))
    Kx = hat(w)
    if th < 1e-6:
        return np.eye(3) + 0.5 * Kx + Kx @ Kx / 6.0
    return (np.eye(3) + (1 - math.cos(th)) / th ** 2 * Kx
            + (th - math.sin(th)) / th ** 3 * Kx @ Kx)


def se3_exp(xi):
    w, v = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    return np.concatenate([so3_exp(w), (_V(w) @ v)[:, None]], axis=1)


def se3_log(T):
    w = so3_log(T[:, :3])
    v = np.linalg.solve(_V(w), T[:, 3])
    return np.concatenate([w, v])


def compose(A, B):
    """A o B (apply B first)."""
    return np.concatenate([A[:, :3] @ B[:, :3], (A[:, :3] @ B[:, 3] + A[:, 3])[:, None]], axis=1)


def inverse(T):
    Rt = T[:, :3].T
    return np.concatenate([Rt, (-Rt @ T[:, 3])[:, None]], axis=1)


IDENTITY = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)

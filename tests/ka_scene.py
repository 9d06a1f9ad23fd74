"""Depth maps rendered analytically from a scene of planes, for the
keyframe-alignment tests (test infrastructure: no alignment arithmetic)."""
import numpy as np

from oracle import geometry

W, H = 160, 120
K = (120.0, 120.0, 80.0, 60.0)
# planes n . X = d in keyframe-1 coordinates (y points down): floor, back
# wall, left and right walls.  Three planes leave the scale unobservable (a
# scaled set of three planes is a translated one: n_i . t = (s - 1) d_i has a
# solution); the fourth, parallel to the third, fixes it.
PLANES = [(np.array([0.0, 1.0, 0.0]), 1.2), (np.array([0.0, 0.0, 1.0]), 9.0),
          (np.array([1.0, 0.0, 0.0]), -4.0), (np.array([1.0, 0.0, 0.0]), 3.0)]


def rays(W, H, K):
    fx, fy, cx, cy = K
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    return np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=-1)


def render(T, W=W, H=H, K=K):
    """Depth map of the camera whose coordinates map to keyframe 1's by T."""
    R, t = T[:, :3], T[:, 3]
    r = rays(W, H, K)
    theta = np.full((H, W), np.inf)
    for n, d in PLANES:
        nc, dc = R.T @ n, d - n @ t          # the plane in this camera's coordinates
        den = r @ nc
        with np.errstate(divide="ignore", invalid="ignore"):
            th = np.where(den != 0, dc / den, np.inf)
        th = np.where(th > 1e-6, th, np.inf)
        theta = np.minimum(theta, th)
    theta[~np.isfinite(theta)] = np.nan
    return theta


def T_true():
    return geometry.se3_exp(np.array([0.01, -0.025, 0.008, 0.2, -0.05, 0.4]))


def start(T, rng, rot=0.02, trans=0.05):
    xi = np.concatenate([rng.normal(size=3) * rot, rng.normal(size=3) * trans])
    return geometry.compose(geometry.se3_exp(xi), T)


def pose_err(A, B):
    d = geometry.se3_log(geometry.compose(geometry.inverse(A), B))
    return np.abs(d[:3]).max(), np.abs(d[3:]).max()

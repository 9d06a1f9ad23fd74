"""Visibility-coverage (VC) score, VO stride and keyframe test (test infrastructure).

Sec. III-B "VO Stride and Keyframe Selection" (Eq. 8): for a pair of frames
with known poses where only the first has a depth map, the visibility is the
fraction of the first frame's depth pixels whose projection falls inside the
second frame's image, the coverage is the fraction of the second frame's
image area that these projections cover, and VC is their harmonic mean.  The
next batch starts at the first frame whose VC with the reference frame is
below tau_stride; the reference frame becomes a keyframe when its VC with the
latest keyframe is below tau_keyframe.

Readings fixed here (the paper leaves them open):
  * depth pixels: reference pixels with a finite inverse depth rho > 0.
  * projection of pixel (u, v) into a frame with pose T = [R | tau]
    (reference -> frame) and intrinsics (fx, fy, cx, cy): with
    r = ((u - cx) / fx, (v - cy) / fy, 1), h = R r + rho tau (the point
    r / rho scaled by rho > 0, which leaves the image point and the sign of
    its depth unchanged); in front when h_z > 1e-6; image point
    x = fx (h_x / h_z) + cx, y = fy (h_y / h_z) + cy; inside when in front and
    0 <= x <= W - 1, 0 <= y <= H - 1 (the second frame has the first's size).
  * coverage: the image area is the W x H grid of pixel cells; a projection
    covers the cell of its nearest pixel (floor(x + 1/2), floor(y + 1/2)).
  * VC = 2 V C / (V + C), 0 when V or C is 0.
  * stride: the first frame t = 1..N with VC < tau_stride; N when there is
    none.
  * precision: the projections decide integers (inside or not, which cell),
    so they are taken in float32, one rounding per operation in the order
    written below (R, tau, intrinsics rounded to float32 once), on both
    sides; the counts are then exact.
"""
from __future__ import annotations

import numpy as np

Z_EPS = np.float32(1e-6)


def project_f32(rho, K, T, W, H):
    """(x, y, inside) of every reference pixel; rho float32 [H][W]."""
    f32 = np.float32
    fx, fy, cx, cy = (f32(k) for k in K)
    R = np.asarray(T, np.float64)[:, :3].astype(f32)
    tau = np.asarray(T, np.float64)[:, 3].astype(f32)
    rho = np.asarray(rho, f32)
    v, u = np.mgrid[0:H, 0:W]
    rx = (u.astype(f32) - cx) / fx
    ry = (v.astype(f32) - cy) / fy
    h = [((R[i, 0] * rx + R[i, 1] * ry) + R[i, 2]) + rho * tau[i] for i in range(3)]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        front = h[2] > Z_EPS
        x = fx * (h[0] / h[2]) + cx
        y = fy * (h[1] / h[2]) + cy
        inside = front & (x >= f32(0)) & (x <= f32(W - 1)) & (y >= f32(0)) & (y <= f32(H - 1))
    return x, y, inside


def counts(rho, K, T, W, H):
    """(depth pixels, depth pixels inside the frame, pixel cells covered)."""
    rho = np.asarray(rho, np.float32)
    with np.errstate(invalid="ignore"):
        valid = np.isfinite(rho) & (rho > 0)
    x, y, inside = project_f32(rho, K, T, W, H)
    vis = valid & inside
    with np.errstate(invalid="ignore"):
        cx = np.floor(x[vis] + np.float32(0.5)).astype(np.int64)
        cy = np.floor(y[vis] + np.float32(0.5)).astype(np.int64)
    covered = np.zeros((H, W), bool)
    covered[cy, cx] = True
    return int(valid.sum()), int(vis.sum()), int(covered.sum())


def harmonic(v, c):
    """VC = 2 V C / (V + C) (Eq. 8), 0 when either is 0."""
    return 0.0 if v <= 0.0 or c <= 0.0 else 2.0 * v * c / (v + c)


def scores(rho, K, T, W, H):
    """(visibility, coverage, VC) of the depth map rho in the frame of pose T."""
    n_depth, n_vis, n_cov = counts(rho, K, T, W, H)
    v = n_vis / n_depth if n_depth else 0.0
    c = n_cov / (W * H)
    return v, c, harmonic(v, c)


def window_scores(rho, K, G, W, H):
    """VC of the reference depth in every frame t = 1..N of a window with
    absolute poses G[t] (reference -> frame t)."""
    return [scores(rho, K, G[t], W, H) for t in range(1, len(G))]


def stride(vc, tau_stride):
    """The next batch's reference: the first t (1-based) with VC < tau_stride,
    len(vc) when there is none."""
    for t, s in enumerate(vc, start=1):
        if s < tau_stride:
            return t
    return len(vc)


def is_keyframe(vc_to_last_keyframe, tau_keyframe):
    return vc_to_last_keyframe < tau_keyframe

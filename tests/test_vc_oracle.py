"""Pins of the VC oracle (oracle/vc.py) against closed forms, exact
rational arithmetic and a scalar brute force.

The cases use a power-of-two focal length and integer principal points, so
that the float32 projections of the oracle are exact and the expected
counts follow from the geometry alone."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import vc

W, H = 96, 40
K = (256.0, 256.0, 40.0, 17.0)     # power-of-two focal length: exact projections


def _pose(R=None, t=(0.0, 0.0, 0.0)):
    T = np.zeros((3, 4))
    T[:, :3] = np.eye(3) if R is None else R
    T[:, 3] = t
    return T


def _plane(rho):
    return np.full((H, W), rho, np.float32)


def test_identity_pose_sees_and_covers_everything():
    assert vc.counts(_plane(0.3), K, _pose(), W, H) == (W * H, W * H, W * H)
    assert vc.scores(_plane(0.3), K, _pose(), W, H) == (1.0, 1.0, 1.0)


@pytest.mark.parametrize("shift", [8, -5])
def test_sideways_translation_over_a_plane(shift):
    # plane at depth 4 (rho = 1/4), translation tau_x: every point moves by
    # fx rho tau_x = shift pixels; the pixels pushed past the border leave
    rho = 0.25
    tx = shift / (K[0] * rho)
    n_depth, n_vis, n_cov = vc.counts(_plane(rho), K, _pose(t=(tx, 0, 0)), W, H)
    assert n_depth == W * H
    assert n_vis == (W - abs(shift)) * H
    assert n_cov == (W - abs(shift)) * H
    v, c, s = vc.scores(_plane(rho), K, _pose(t=(tx, 0, 0)), W, H)
    assert v == c == s == (W - abs(shift)) / W


def test_two_projections_in_one_nearest_pixel_cell():
    # tau_x = 1/fx moves a point by rho pixels: pixel 3 (rho 5/8) lands on
    # x = 3.625 and pixel 4 (rho 1/4) on x = 4.25, both nearest to pixel 4:
    # two visible depth pixels, one covered cell
    rho = np.full((H, W), np.nan, np.float32)
    rho[5, 3], rho[5, 4] = 0.625, 0.25
    x, y, inside = vc.project_f32(rho, K, _pose(t=(1.0 / K[0], 0, 0)), W, H)
    assert x[5, 3] == 3.625 and x[5, 4] == 4.25 and y[5, 3] == 5.0
    assert vc.counts(rho, K, _pose(t=(1.0 / K[0], 0, 0)), W, H) == (2, 2, 1)


def test_camera_past_the_plane_sees_nothing():
    # h_z = 1 + rho tau_z = 1 - 2 < 0 for every pixel
    assert vc.counts(_plane(0.25), K, _pose(t=(0, 0, -8.0)), W, H) == (W * H, 0, 0)
    assert vc.scores(_plane(0.25), K, _pose(t=(0, 0, -8.0)), W, H) == (0.0, 0.0, 0.0)


def test_invalid_depths_are_not_depth_pixels():
    rho = _plane(0.25)
    rho[::2] = np.nan
    rho[1::4, :10] = -1.0
    rho[3::4, 10:20] = 0.0
    valid = int(np.sum(np.isfinite(rho) & (rho > 0)))
    n_depth, n_vis, n_cov = vc.counts(rho, K, _pose(), W, H)
    assert n_depth == valid and n_vis == valid and n_cov == valid
    # no depth pixel at all: visibility 0 by definition
    assert vc.scores(np.full((H, W), np.nan, np.float32), K, _pose(), W, H) == (0.0, 0.0, 0.0)


def test_coverage_is_a_fraction_of_the_image_not_of_the_depth_pixels():
    # only the left half has depth: all of it is visible and covers half of
    # the second image (V = 1, C = 1/2, VC = 2/3)
    rho = np.full((H, W), np.nan, np.float32)
    rho[:, :W // 2] = 0.25
    assert vc.scores(rho, K, _pose(), W, H) == (1.0, 0.5, pytest.approx(2.0 / 3.0))


def test_receding_camera_contracts_the_image():
    # tau_z = +2 on a plane at depth 4: h = (r, 1.5); every point lands at
    # c + (p - c) / 1.5.  Coverage counted with exact rationals (no ties:
    # the fractional parts are 0, 1/3, 2/3).
    rho = 0.25
    cover = set()
    for v in range(H):
        for u in range(W):
            x = Fraction(int(K[2])) + Fraction(u - int(K[2])) / Fraction(3, 2)
            y = Fraction(int(K[3])) + Fraction(v - int(K[3])) / Fraction(3, 2)
            cover.add((int(np.floor(x + Fraction(1, 2))), int(np.floor(y + Fraction(1, 2)))))
    assert vc.counts(_plane(rho), K, _pose(t=(0, 0, 2.0)), W, H) == (W * H, W * H, len(cover))


def test_vectorised_projection_equals_a_scalar_loop():
    rng = np.random.default_rng(0)
    w, h = 13, 7
    Kr = (97.3, 101.1, 6.2, 3.4)
    rho = rng.uniform(0.05, 1.0, (h, w)).astype(np.float32)
    rho[2, 3] = np.nan
    a = rng.normal(size=3) * 0.05
    th = np.linalg.norm(a)
    A = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]]) / th
    R = np.eye(3) + np.sin(th) * A + (1 - np.cos(th)) * A @ A
    T = _pose(R, rng.normal(size=3) * 0.3)
    x, y, inside = vc.project_f32(rho, Kr, T, w, h)
    f = np.float32
    fx, fy, cx, cy = (f(k) for k in Kr)
    Rf, tf = T[:, :3].astype(f), T[:, 3].astype(f)
    for v in range(h):
        for u in range(w):
            rx = (f(u) - cx) / fx
            ry = (f(v) - cy) / fy
            hh = [((Rf[i, 0] * rx + Rf[i, 1] * ry) + Rf[i, 2]) + rho[v, u] * tf[i] for i in range(3)]
            if not np.isfinite(rho[v, u]):
                continue
            xs = fx * (hh[0] / hh[2]) + cx
            ys = fy * (hh[1] / hh[2]) + cy
            assert xs == x[v, u] and ys == y[v, u]
            ins = bool(hh[2] > f(1e-6) and 0 <= xs <= w - 1 and 0 <= ys <= h - 1)
            assert ins == bool(inside[v, u])


def test_harmonic_mean_stride_and_keyframe():
    assert vc.harmonic(0.5, 1.0) == pytest.approx(2.0 / 3.0)
    assert vc.harmonic(0.8, 0.8) == pytest.approx(0.8)
    assert vc.harmonic(0.0, 0.7) == 0.0 and vc.harmonic(0.7, 0.0) == 0.0
    assert vc.stride([0.95, 0.81, 0.62, 0.4], 0.7) == 3
    assert vc.stride([0.95, 0.81], 0.7) == 2            # none below: the last frame
    assert vc.stride([0.5, 0.9], 0.7) == 1
    assert vc.stride([0.9, 0.7, 0.5], 0.7) == 3       # equal is not below
    assert vc.is_keyframe(0.49, 0.5) and not vc.is_keyframe(0.5, 0.5)


def test_window_scores_follow_the_poses():
    rho = 0.25
    G = [_pose(), _pose(t=(2 / (K[0] * rho), 0, 0)), _pose(t=(16 / (K[0] * rho), 0, 0))]
    s = vc.window_scores(_plane(rho), K, G, W, H)
    assert [x[0] for x in s] == [(W - 2) / W, (W - 16) / W]
    assert vc.stride([x[2] for x in s], 0.9) == 2


def test_direction_of_translation_and_rotation():
    # T maps reference coordinates to the frame's: a point moves by
    # +fx rho tau_x, and a rotation about y by a moves the principal point
    # to cx + fx tan(a) (R, not its transpose)
    rho = 0.25
    x, y, inside = vc.project_f32(_plane(rho), K, _pose(t=(8 / (K[0] * rho), 0, 0)), W, H)
    assert x[0, 0] == 8.0 and y[5, 0] == 5.0
    assert inside[0, W - 9] and not inside[0, W - 8]
    a = 0.05
    R = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    x, y, _ = vc.project_f32(_plane(rho), K, _pose(R), W, H)
    u, v = int(K[2]), int(K[3])
    assert x[v, u] == pytest.approx(K[2] + K[0] * np.tan(a), abs=1e-3)
    assert y[v, u] == pytest.approx(K[3], abs=1e-4)

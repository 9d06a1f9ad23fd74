"""Pose M-step: Monte-Carlo P3P sampling, dense scoring and mean-shift (Eq. 7).

Sec. III-A "Uncertainty-aware Pose Estimation": with depth and rigidness
fixed, the posterior of each camera pose is approximated by S samples, each a
P3P solution; every sample is a Gaussian N(T_g, Sigma) with a fixed Sigma, and
the pose is the mode of this mixture, found by mean-shift with a Gaussian
kernel in the Lie algebra.

Reading fixed here:
  * poses are absolute G_t (frame 0 -> frame t); frames are updated in order
    t = 1..N, each using the already updated G_{t-1}.
  * rigid set R_t: pixels j (in row-major order) with q_t^j > 0.5 (float32
    compare), x_{t-1} = pi(G_{t-1} X_j) in front of camera t-1 and inside the
    image (always true for t = 1), and X_j in front of the current camera t.
    These tests are taken in float64.
  * correspondence of j: world point X_j = r_j / rho_j and the observed frame-t
    pixel x_obs = x_{t-1} + X_t(x_{t-1}).
  * sample g draws 3 indices into R_t from Philox(g + 65536 t, iteration code,
    TAG_POSE, attempt) words 0..2 as (word * |R_t|) >> 32; a draw with a
    repeated index is retried with the next attempt (at most 8), else void.
  * each P3P root is scored by E = sum_{j in R_t} q_t^j l(|x_obs - pi(G X_j)|)
    (l = L_BEHIND behind the camera); the sample keeps its lowest-energy root
    (roots ordered by (rotation vector, translation) first; ties: first).
  * mean-shift starts at the lowest-energy sample and iterates
    x <- x exp(sum_g w_g d_g / sum_g w_g), d_g = log(x^-1 T_g),
    w_g = exp(-d_g^T Sigma^-1 d_g / 2), until |step| < 1e-12: the pose is
    the mode of the approximated posterior (Sec. III-A, the paragraph after
    Eq. 7), the iteration's fixed point, so it runs to convergence; the
    linear rate approaches 1 where the mode is flat (a few samples in the
    kernel's reach, as after the bootstrap), and MS_MAX_ITERS is only a
    safeguard.  Sigma = diag(s_r^2 (x3), s_t^2 (x3)), s_t = rel |tau_start| + abs.
  * fewer than 3 rigid pixels, or no valid sample: the pose is kept and the
    step reports a degenerate frame.
"""
from __future__ import annotations

import math

import numpy as np

from . import fisk, geometry, model, p3p, philox

MS_TOL = 1e-12
MS_MAX_ITERS = 100000
MAX_ATTEMPTS = 8


def rigid_set(P: model.Problem, S: model.State, t, p: model.Params):
    """Ordered rigid pixel set of frame t and its correspondences (float64)."""
    iu, iv = model.pixel_grid(P)
    rho = S.rho.astype(np.float64)
    r = P.rays
    if t == 1:
        xp = iu.astype(np.float64)
        yp = iv.astype(np.float64)
        ok = np.ones((P.H, P.W), bool)
        F = P.flow[0].astype(np.float64)
    else:
        xp, yp, front = geometry.dehom(geometry.project_h(P.K, S.G[t - 1], r, rho))
        ok = front & geometry.inside(xp, yp, P.W, P.H)
        F = geometry.bilinear(P.flow[t - 1], np.where(ok, xp, 0.0), np.where(ok, yp, 0.0))
    _, _, front_t = geometry.dehom(geometry.project_h(P.K, S.G[t], r, rho))
    ok = ok & front_t & (S.q[t - 1] > np.float32(0.5))
    j = np.flatnonzero(ok.ravel())
    vv, uu = np.divmod(j, P.W)
    X = r[vv, uu] / rho[vv, uu][:, None]
    xobs = np.stack([xp[vv, uu] + F[vv, uu, 0], yp[vv, uu] + F[vv, uu, 1]], axis=1)
    w = S.q[t - 1][vv, uu].astype(np.float64)
    alpha = p.fisk_alpha0 + p.fisk_alpha1 * np.hypot(F[vv, uu, 0], F[vv, uu, 1])
    return dict(j=j, X=X, xobs=xobs, w=w, alpha=alpha)


def draw_triplet(n, g, t, it_code, p):
    """Three distinct indices into a set of size n, or None (void sample)."""
    k0, k1 = philox.seed_key(p.seed)
    for b in range(MAX_ATTEMPTS):
        w = philox.philox4x32_10(g + 65536 * t, it_code, philox.TAG_POSE, b, k0, k1)
        idx = [int(philox.index_pick(w[m], n)) for m in range(3)]
        if len(set(idx)) == 3:
            return idx
    return None


def score(P, G, rs, p):
    """E(G) = sum_j q_j l(|x_obs - pi(G X_j)|) over the rigid set (float64)."""
    fx, fy, cx, cy = P.K
    Xc = rs["X"] @ G[:, :3].T + G[:, 3]
    front = Xc[:, 2] > geometry.Z_EPS
    z = np.where(front, Xc[:, 2], 1.0)
    x = fx * Xc[:, 0] / z + cx
    y = fy * Xc[:, 1] / z + cy
    rr = np.hypot(rs["xobs"][:, 0] - x, rs["xobs"][:, 1] - y)
    ell = np.where(front, fisk.inlier_energy(rr, rs["alpha"], p.fisk_beta, p.outlier_density),
                   fisk.L_BEHIND)
    return float(np.sum(rs["w"] * ell))


def root_key(G):
    w = geometry.so3_log(G[:, :3])
    return tuple(w) + tuple(G[:, 3])


def meanshift(samples, start, p):
    st = p.pose_sigma_trans_rel * float(np.linalg.norm(start[:, 3])) + p.pose_sigma_trans_abs
    inv_var = np.array([1 / p.pose_sigma_rot ** 2] * 3 + [1 / st ** 2] * 3)
    x = start.copy()
    n_it = 0
    for n_it in range(1, MS_MAX_ITERS + 1):
        xi = geometry.inverse(x)
        d = np.stack([geometry.se3_log(geometry.compose(xi, T)) for T in samples])
        w = np.exp(-0.5 * np.sum(d * d * inv_var, axis=1))
        step = (w[:, None] * d).sum(0) / w.sum()
        x = geometry.compose(x, geometry.se3_exp(step))
        if np.linalg.norm(step) < MS_TOL:
            break
    return x, n_it


def pose_mstep_frame(P, S: model.State, t, it, p, detail=False):
    """Update S.G[t] in place; returns a dict of intermediate results."""
    it_code = philox.ITER_BOOT if it < 0 else int(it)
    rs = rigid_set(P, S, t, p)
    n = len(rs["j"])
    out = dict(n_rigid=n, degenerate=False, samples=[], scores=[], roots=[], root_scores=[],
               tri_X=[], tri_bear=[])
    if n < 3:
        out["degenerate"] = True
        return out
    fx, fy, cx, cy = P.K
    samples, sample_E = [], []
    for g in range(p.n_pose_samples):
        tri = draw_triplet(n, g, t, it_code, p)
        if tri is None:
            out["roots"].append([])
            out["root_scores"].append([])
            out["tri_X"].append(None)
            out["tri_bear"].append(None)
            continue
        X3 = rs["X"][tri]
        xo = rs["xobs"][tri]
        bear = np.stack([(xo[:, 0] - cx) / fx, (xo[:, 1] - cy) / fy, np.ones(3)], axis=1)
        roots = sorted(p3p.solve(bear, X3), key=root_key)
        if detail:
            out["roots"].append(roots)
            out["tri_X"].append(X3)
            out["tri_bear"].append(bear)
        Es = [score(P, G, rs, p) for G in roots]
        if detail:
            out["root_scores"].append(Es)
        if not roots:
            continue
        k = int(np.argmin(Es))
        samples.append(roots[k])
        sample_E.append(Es[k])
    out["samples"], out["scores"] = samples, sample_E
    if not samples:
        out["degenerate"] = True
        return out
    start = samples[int(np.argmin(sample_E))]
    x, n_it = meanshift(samples, start, p)
    out["ms_iters"] = n_it
    S.G[t] = x
    return out


def pose_mstep(P, S, it, p):
    return [pose_mstep_frame(P, S, t, it, p) for t in range(1, P.N + 1)]

"""The generalised-EM schedule over one window (Sec. III-A).

Iteration i (0-based), chain direction d = i mod 4:
  1. depth M-step (depth.depth_mstep): candidates, argmin, propagation along d;
  2. rigidness E-step (hmm.rigidness_estep) on the chains of d at the new depth;
  3. pose M-step (pose.pose_mstep) for t = 1..N in order.

Bootstrap before iteration 0 (VOLDOR+ bootstraps from priors where it has
them, Sec. I and III-A):
  * with a depth prior: rho = clamped prior inverse depth (random draw at prior
    holes), q = 1, q_hat = 1, poses as given (identity by default), then one
    pose M-step;
  * monocular: G_1 from the 8-point method (|tau_1| = 1), G_t = G_1 composed t
    times; rho drawn uniformly from [rho_min, rho_max] (Philox, TAG_INIT,
    word 0 of counter (j, ITER_BOOT, TAG_INIT, 0)); a depth M-step along
    direction 0 with only X_1 weighted (q_1 = 1, q_t = 0 for t > 1); then
    q = 1 and one pose M-step.
Both bootstrap steps use the iteration code ITER_BOOT for their draws.
"""
from __future__ import annotations

import numpy as np

from . import depth, eightpoint, geometry, hmm, model, philox, pose


def initial_rho(P: model.Problem, p: model.Params):
    iv, iu = np.mgrid[0:P.H, 0:P.W]
    j = (iv * P.W + iu).astype(np.uint64)
    k0, k1 = philox.seed_key(p.seed)
    w = philox.philox4x32_10(j, philox.ITER_BOOT, philox.TAG_INIT, 0, k0, k1)[0]
    u = philox.u24_float(w)
    rmin, rmax = p.f32("rho_min"), p.f32("rho_max")
    rho = rmin + np.float32(u * np.float32(rmax - rmin))
    prho = P.prior_rho()
    if prho is not None:
        rho = np.where(np.isfinite(prho), np.clip(prho, rmin, rmax), rho)
    return rho.astype(np.float32)


def bootstrap(P: model.Problem, p: model.Params, G_init=None):
    G = np.stack([geometry.IDENTITY] * (P.N + 1)) if G_init is None else np.array(G_init, np.float64)
    S = model.State(rho=initial_rho(P, p), q=np.ones((P.N, P.H, P.W), np.float32),
                    qhat=np.ones((P.H, P.W), np.float32), G=G)
    info = {}
    if P.prior_kind == "none":
        G1, counts = eightpoint.bootstrap_pose(P, p.fisk_alpha0)
        info["eight_point_counts"] = counts
        S.G[0] = geometry.IDENTITY
        S.G[1] = G1
        for t in range(2, P.N + 1):
            S.G[t] = geometry.compose(G1, S.G[t - 1])
        S.q[1:] = 0.0
        rho_new, _, _, _ = depth.depth_mstep(P, S, -1, 0, p)
        S.rho = rho_new
        S.q[:] = 1.0
    info["pose"] = pose.pose_mstep(P, S, -1, p)
    return S, info


def iteration(P, S: model.State, it, p):
    d = it % 4
    rho_new, E_new, rho_star, E_star = depth.depth_mstep(P, S, it, d, p)
    S.rho = rho_new
    S.q, S.qhat, S.C = hmm.rigidness_estep(P, S, rho_new, d, p)
    info = pose.pose_mstep(P, S, it, p)
    return dict(E=E_new, pose=info)


def run(P, p, n_iters, S=None):
    infos = []
    if S is None:
        S, binfo = bootstrap(P, p)
        infos.append(binfo)
    for it in range(n_iters):
        infos.append(iteration(P, S, it, p))
    return S, infos


def relative_poses(G):
    """T_t = G_t G_{t-1}^-1, t = 1..N (frame t-1 -> t)."""
    return np.stack([geometry.compose(G[t], geometry.inverse(G[t - 1])) for t in range(1, len(G))])

"""Shared helpers of the GPU parity tests: build a library context from a
synthetic window, and the oracle objects for the same window and state."""
import numpy as np

import synth
from oracle import model as omodel

# Tolerances.  Rigidness and poses use the bounds of the method statement
# (1e-4 absolute on rigidness, 1e-4 rad / 1e-4 relative on poses).  Where
# float arithmetic decides a discrete choice (the argmin over hypotheses, a
# propagation step), a choice that differs from the oracle's counts as
# correct when the oracle's own float64 energies of the two choices are
# within the energy tie band: the float32 energy differs from the float64 one
# by the rounding of the projected positions (|x| * 2^-23 per coordinate,
# amplified by dl/dr <= ~0.7 per px and summed over N flows) plus the MUFU
# log2 error (~2^-22 absolute per term).
RIGID_TOL = 1e-4
POSE_ROT_TOL = 1e-4
POSE_TRANS_TOL = 1e-4


def tie_band(P, E):
    xmax = max(P.W, P.H) + 200.0
    per_term = 0.7 * 4 * xmax * 2.0 ** -23 + 4 * 2.0 ** -22
    return P.N * per_term + 2e-6 * np.abs(E)


def params_for(win, **kw):
    pr = win.params
    d = dict(fisk_alpha0=pr["fisk_alpha0"], rho_min=pr["rho_min"], rho_max=pr["rho_max"],
             n_hyp=pr["n_hyp"])
    d.update(kw)
    return d


def make_ctx(V, win, prior="auto", **pkw):
    params = V.vd_params_default(**params_for(win, **pkw))
    ctx = V.vd_create(win.W, win.H, win.N, win.intrinsics, params)
    for t in range(1, win.N + 1):
        V.vd_push_flow(ctx, t, win.flow[t - 1])
    P = omodel.problem_from_window(win, prior=prior)
    if P.prior_kind == "stereo":
        V.vd_push_stereo_prior(ctx, win.stereo_disp, win.stereo_baseline)
    elif P.prior_kind == "rgbd":
        V.vd_push_depth_prior(ctx, win.depth_prior)
    return ctx, P, omodel.Params(**params_for(win, **pkw))


def noisy_state(win, P, rng, rel=0.05, qmode="random"):
    """A plausible mid-EM state: true depth with multiplicative noise, random
    rigidness, true poses (in the window's depth units)."""
    s = win.params["scale"]
    G = win.G.copy()
    G[:, :, 3] /= s
    rho = (s / win.depth0 * (1 + rel * rng.standard_normal(win.depth0.shape))).astype(np.float32)
    rho = np.clip(rho, np.float32(win.params["rho_min"]), np.float32(win.params["rho_max"]))
    if qmode == "random":
        q = rng.uniform(0.0, 1.0, size=(P.N, P.H, P.W)).astype(np.float32)
    else:
        q = np.ones((P.N, P.H, P.W), np.float32)
    qhat = rng.uniform(0.2, 1.0, size=(P.H, P.W)).astype(np.float32)
    return omodel.State(rho=rho, q=q, qhat=qhat, G=G)


def push_state(V, ctx, S):
    V.vd_set_poses(ctx, S.G.reshape(-1, 12))
    V.vd_set_state(ctx, S.rho, S.q, S.qhat)


def window(name, seed=0, **kw):
    return synth.make_window(name, seed, **kw)

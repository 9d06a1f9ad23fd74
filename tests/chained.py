"""Chained stage-wise replay of whole EM runs against the float64 oracle.

The library runs a window's bootstrap and iterations one stage at a time
through the C ABI (8-point pose, depth M-step, rigidness E-step, pose M-step
of each frame).  Before every stage the oracle is handed the library's state
at that point (inverse depth, rigidness, poses), runs the same stage from it,
and the two results are compared element by element at the method's bounds:

  * depth M-step (Eq. 5, propagation paragraph of Sec. III-A): the GPU's
    candidates are the oracle's float32 candidates bit for bit; each pixel's
    choice, and each propagation step, is the oracle's or one whose float64
    energy lies within the tie band of the oracle's best (several choices
    are correct there); a float32 decision at an image border or at the
    camera plane may flip a term (see `term_ranges`), which widens a
    choice's energy to the range of its possible terms;
  * rigidness E-step (Sec. III-A, forward-backward on the chains): every
    posterior within 1e-4 of the oracle's, except on a chain holding a term
    whose observability is decided within float32 rounding of a threshold:
    that chain must match, within 1e-4 everywhere, the oracle's posterior
    under one of the possible decisions of those terms;
  * pose M-step (Eq. 7): the rigid set is the oracle's (same size), every
    sample keeps the oracle's root (ill-conditioned P3P instances excepted,
    as the stage tests state), and the pose is within 1e-4 rad and 1e-4
    relative translation of the oracle's.

The GPU is never fed anything but its own state, so the chained GPU run is
the uninterrupted one: `replay` ends by checking that vd_bootstrap +
vd_run_em on a fresh context reach bit for bit the same depth, rigidness and
poses.  Every stage of the real run is thus compared with the oracle started
from the same state, and a float32 near-tie cannot cascade into a drift that
no single stage shows.
"""
from __future__ import annotations

import time

import numpy as np

from oracle import depth as odepth
from oracle import eightpoint as oeight
from oracle import em as oem
from oracle import fisk as ofisk
from oracle import geometry as ogeo
from oracle import hmm as ohmm
from oracle import model as omodel
from oracle import pose as opose

from gpu_common import POSE_ROT_TOL, POSE_TRANS_TOL, RIGID_TOL, tie_band

# A float32 decision is "within rounding of a threshold" when the float64
# value is this close to it: image borders in px, the camera plane in units
# of the homogeneous z (the float32 positions are good to ~1e-3 px and z to
# ~1e-6 at these sizes; the margins are ten to a hundred times that).
BORDER_MARGIN_PX = 1e-2
ZPLANE_MARGIN = 1e-4
# The same for the double-float positions of the rigidness emissions (good
# to ~1e-11 px in the image and z to ~1e-14; again a hundred times that and
# more, plus the position's own error bound, `_df_proj_err`, where it is
# larger).
BORDER_MARGIN_DF_PX = 1e-8
ZPLANE_MARGIN_DF = 1e-10


def pose_err(A, B):
    d = ogeo.se3_log(ogeo.compose(ogeo.inverse(A), B))
    rot = float(np.linalg.norm(d[:3]))
    trans = float(np.linalg.norm(A[:, 3] - B[:, 3]) / max(np.linalg.norm(A[:, 3]), 1e-9))
    return rot, trans


def crop_problem(win, cw, ch):
    """The centred cw x ch crop of a window: flows and intrinsics of the crop."""
    u0, v0 = (win.W - cw) // 2, (win.H - ch) // 2
    fx, fy, cx, cy = win.intrinsics
    flow = np.ascontiguousarray(win.flow[:, v0:v0 + ch, u0:u0 + cw])
    return flow, (fx, fy, cx - u0, cy - v0), (u0, v0)


# ----------------------------------------------------------------- GPU state
def read_state(V, ctx, P):
    rho = np.zeros((P.H, P.W), np.float32)
    q = np.zeros((P.N, P.H, P.W), np.float32)
    qh = np.zeros((P.H, P.W), np.float32)
    V.vd_get_inv_depth(ctx, rho)
    V.vd_get_rigidness(ctx, q)
    V.vd_get_prior_rigidness(ctx, qh)
    G = V.vd_get_poses(ctx, P.N)
    return omodel.State(rho=rho, q=q, qhat=qh, G=np.array(G, np.float64))


# ----------------------------------------------------------------- terms
def _lin_pos_err(c, W):
    """Bound on the float32 error of a projected coordinate c (px): a few
    roundings of numbers of magnitude |c| + W (the homogeneous products and
    the division)."""
    return 2.0 ** -21 * (np.abs(np.nan_to_num(c, nan=0.0)) + W)


def _df_proj_err(h, S):
    """Bounds on the errors of the double-float positions x = h_x / h_z,
    y = h_y / h_z (px), given the homogeneous point h and S, the sums of the
    absolute values of the products that form h (the projection of |R|,
    |tau| and |r|): the compensated sums are good to a few 2^-48 S, the
    double-float rows and rays to 2^-47, and the quotient adds the error of
    h_z times |x|; 2^-42 leaves a wide margin.  Near the camera plane
    (small h_z) the bound grows with 1 / h_z."""
    with np.errstate(invalid="ignore", divide="ignore"):
        iz = 1.0 / np.abs(h[..., 2])
        x = np.abs(h[..., 0]) * iz
        y = np.abs(h[..., 1]) * iz
        ex = 2.0 ** -42 * (S[..., 0] + x * S[..., 2]) * iz
        ey = 2.0 ** -42 * (S[..., 1] + y * S[..., 2]) * iz
    return np.nan_to_num(ex, nan=0.0, posinf=0.0), np.nan_to_num(ey, nan=0.0, posinf=0.0)


def _tap_gradient(F, x, y):
    """Largest difference between neighbouring bilinear taps of F around
    (x, y) (px of flow per px of position, both components)."""
    H, W = F.shape[:2]
    x0 = np.minimum(np.floor(x), W - 2).astype(np.int64)
    y0 = np.minimum(np.floor(y), H - 2).astype(np.int64)
    F = F.astype(np.float64)
    f00, f01 = F[y0, x0], F[y0, x0 + 1]
    f10, f11 = F[y0 + 1, x0], F[y0 + 1, x0 + 1]
    g = np.maximum.reduce([np.abs(f01 - f00), np.abs(f11 - f10), np.abs(f10 - f00),
                           np.abs(f11 - f01)])
    return g.max(-1)


def _fisk_interval(fn, rr, dr):
    """min and max of fn over [rr - dr, rr + dr] (ends and centre)."""
    vals = [fn(np.maximum(rr - dr, 0.0)), fn(rr), fn(rr + dr)]
    return np.minimum.reduce(vals), np.maximum.reduce(vals)


# absolute error of one float32 log / exp chain of the library (a few
# MUFU-approximated log2 / exp2 steps)
MUFU_ERR = 8 * 2.0 ** -22


def term_ranges(P, G, iu, iv, rho, p, positions="f32"):
    """Per flow term of pixels (iu, iv) at inverse depth rho: the values a
    float32 evaluation of the same definition may give.

    Two effects are bounded.  Rounding: the projected positions carry a
    few roundings (`_lin_pos_err`, or `_df_proj_err` with
    positions="df", the rigidness emissions), which move the residual by
    at most the position errors of x_{t-1} and x_t plus the error of
    x_{t-1} times the flow's tap gradient there (steep at a depth edge of
    the flow field); the float32 bilinear weights, flow sample and
    residual add a few roundings of the flow's magnitude and gradient.
    Decisions: a term whose observability (inside the image, in front of
    camera t-1) or camera-plane test at t lies within rounding of its
    threshold may take either side.

    Returns dict of [N, ...] arrays: l_lo, l_hi (the energy term), e1_lo,
    e1_hi (the rigid emission), e1 (the oracle's emission), flipped (a
    decision is within rounding) and steep (the flow changes by more than
    4 px between neighbouring taps)."""
    df = positions == "df"
    if df:
        border, zmargin = BORDER_MARGIN_DF_PX, ZPLANE_MARGIN_DF
    else:
        border, zmargin = BORDER_MARGIN_PX, ZPLANE_MARGIN
    iu = np.asarray(iu)
    iv = np.asarray(iv)
    rho = np.asarray(rho, np.float64)
    r = P.rays[iv, iu]
    W, H = P.W, P.H
    xp = iu.astype(np.float64)
    yp = iv.astype(np.float64)
    zp = np.ones(iu.shape)
    exp_ = np.zeros(iu.shape)   # error bounds of the previous position
    eyp = np.zeros(iu.shape)
    out = {k: [] for k in ("l_lo", "l_hi", "e1_lo", "e1_hi", "e1", "flipped", "steep")}
    big = np.inf
    for t in range(1, P.N + 1):
        h = ogeo.project_h(P.K, G[t], r, rho)
        hz = h[..., 2]
        if df:
            ex, ey = _df_proj_err(h, ogeo.project_h(P.K, np.abs(G[t]), np.abs(r), np.abs(rho)))
        else:
            ex = ey = None   # after the dehomogenisation below
        front = hz > ogeo.Z_EPS
        amb_front = np.abs(hz - ogeo.Z_EPS) < zmargin
        if t == 1:
            obs = np.ones(iu.shape, bool)
            amb_obs = np.zeros(iu.shape, bool)
            F = P.flow[0][iv, iu].astype(np.float64)
            e_prev = np.zeros(iu.shape)
            grad = np.zeros(iu.shape)
        else:
            fprev = zp > ogeo.Z_EPS
            with np.errstate(invalid="ignore"):
                ins = ogeo.inside(xp, yp, W, H)
                bd = border + np.maximum(exp_, eyp)
                near = (np.minimum.reduce([np.abs(xp), np.abs(xp - (W - 1)), np.abs(yp),
                                           np.abs(yp - (H - 1))]) < bd)
                loose = ((xp >= -bd) & (xp <= W - 1 + bd) &
                         (yp >= -bd) & (yp <= H - 1 + bd))
            near = np.where(np.isfinite(xp) & np.isfinite(yp), near, False)
            obs = fprev & ins
            amb_obs = (np.abs(zp - ogeo.Z_EPS) < zmargin) | (fprev & near & loose)
            xs = np.clip(np.nan_to_num(xp), 0.0, W - 1)
            ys = np.clip(np.nan_to_num(yp), 0.0, H - 1)
            F = ogeo.bilinear(P.flow[t - 1], xs, ys)
            e_prev = exp_ + eyp
            grad = _tap_gradient(P.flow[t - 1], xs, ys)
        hz_f = np.where(hz > ogeo.Z_EPS, hz, ogeo.Z_EPS * (1 + 1e-9))
        x = h[..., 0] / hz_f
        y = h[..., 1] / hz_f
        if not df:
            ex, ey = _lin_pos_err(x, W), _lin_pos_err(y, W)
        rr = np.hypot(F[..., 0] - (x - xp), F[..., 1] - (y - yp))
        rr = np.where(np.isfinite(rr), rr, 1e30)
        with np.errstate(invalid="ignore"):
            fsz = (np.abs(F).sum(-1) + np.abs(np.nan_to_num(x - xp)) +
                   np.abs(np.nan_to_num(y - yp)))
        dr = (e_prev * (1.0 + grad) + ex + ey + 2.0 ** -21 * (fsz + 2.0 * grad))
        alpha = p.fisk_alpha0 + p.fisk_alpha1 * np.hypot(F[..., 0], F[..., 1])
        with np.errstate(over="ignore", divide="ignore"):
            l_lo, l_hi = _fisk_interval(
                lambda z: ofisk.inlier_energy(z, alpha, p.fisk_beta, p.outlier_density), rr, dr)
            e_lo, e_hi = _fisk_interval(
                lambda z: ofisk.residual_density(z, alpha, p.fisk_beta), rr, dr)
        l_lo, l_hi = l_lo - MUFU_ERR, l_hi + MUFU_ERR
        e_lo, e_hi = e_lo * (1 - MUFU_ERR), e_hi * (1 + MUFU_ERR)
        can_obs = obs | amb_obs
        can_unobs = ~obs | amb_obs
        can_front = can_obs & (front | amb_front)
        can_behind = can_obs & (~front | amb_front)
        out["l_lo"].append(np.minimum.reduce([np.where(can_unobs, 0.0, big),
                                              np.where(can_front, l_lo, big),
                                              np.where(can_behind, ofisk.L_BEHIND, big)]))
        out["l_hi"].append(np.maximum.reduce([np.where(can_unobs, 0.0, -big),
                                              np.where(can_front, l_hi, -big),
                                              np.where(can_behind, ofisk.L_BEHIND, -big)]))
        P0 = p.outlier_density
        out["e1_lo"].append(np.minimum.reduce([np.where(can_unobs, P0, big),
                                               np.where(can_front, e_lo, big),
                                               np.where(can_behind, 0.0, big)]))
        out["e1_hi"].append(np.maximum.reduce([np.where(can_unobs, P0, -big),
                                               np.where(can_front, e_hi, -big),
                                               np.where(can_behind, 0.0, -big)]))
        with np.errstate(over="ignore", divide="ignore"):
            e_pt = ofisk.residual_density(rr, alpha, p.fisk_beta)
        out["e1"].append(np.where(obs & front, e_pt, np.where(obs, 0.0, P0)))
        out["flipped"].append(amb_obs | (can_obs & amb_front))
        out["steep"].append(can_front & (grad > 4.0))
        xp, yp, zp = x, y, hz
        exp_, eyp = ex, ey
        # positions behind the camera are not positions: NaN, as the oracle
        xp = np.where(front, xp, np.nan)
        yp = np.where(front, yp, np.nan)
    return {k: np.stack(v) for k, v in out.items()}


def energy_range(P, S, iu, iv, rho, p):
    """(E_lo, E_hi): the energy of Eq. 5 over every float32 evaluation that
    `term_ranges` allows (plus the float32 sum and the prior term, relative
    2e-6)."""
    tr = term_ranges(P, S.G, iu, iv, rho, p)
    q = S.q[:, iv, iu].astype(np.float64)
    E_lo = np.sum(q * tr["l_lo"], axis=0)
    E_hi = np.sum(q * tr["l_hi"], axis=0)
    if P.prior_kind != "none":
        lh, _, _, _ = omodel.prior_terms(P, iu, iv, rho, p)
        wp = omodel.prior_weight(P, S, iu, iv) * lh
        E_lo = E_lo + wp
        E_hi = E_hi + wp
    return E_lo - 2e-6 * np.abs(E_lo), E_hi + 2e-6 * np.abs(E_hi)


# ----------------------------------------------------------------- report
class Report:
    def __init__(self, name):
        self.name = name
        self.rows = []
        self.discrete = 0        # pose stages that differ through a float32 choice
        self.t0 = time.perf_counter()

    def add(self, stage, **kw):
        self.rows.append(dict(stage=stage, **kw))

    def summary(self):
        lines = [f"chained replay {self.name}: {len(self.rows)} stages, "
                 f"{time.perf_counter() - self.t0:.0f} s"]
        for r in self.rows:
            lines.append("  " + " ".join(f"{k}={v}" for k, v in r.items()))
        return "\n".join(lines)


# ----------------------------------------------------------------- stages
def check_argmin(P, S, it, p, rs, es, label):
    """Step A of the depth M-step: candidates bit for bit, each choice the
    oracle's or within the tie band.  Returns (oracle energy of the GPU's
    choices, tie band, fraction identical, number of flipped-term choices)."""
    iu, iv = omodel.pixel_grid(P)
    cands = odepth.hypotheses(P, S.rho, it, p)
    member = (cands == rs[None]).any(0)
    assert member.all(), f"{label}: {(~member).sum()} GPU choices outside the oracle's candidates"
    ro, eo, _ = odepth.argmin_candidates(P, S, cands, p)
    e_g = omodel.energy(P, S, iu, iv, rs, p)
    band = tie_band(P, eo)
    n_e = check_energy(P, S, rs, es, e_g, band, p, label)
    same = rs == ro
    ok = same | (e_g - eo <= band)
    n_flip = 0
    if not ok.all():
        # outside the fixed band: the choice is valid if some float32
        # evaluation of the definition (`term_ranges`) ranks it first, i.e.
        # its lowest value is below every candidate's highest
        fv, fu = np.nonzero(~ok)
        lo_g, _ = energy_range(P, S, fu, fv, rs[fv, fu], p)
        best_hi = np.full(len(fu), np.inf)
        for k in range(cands.shape[0]):
            _, hi_k = energy_range(P, S, fu, fv, cands[k][fv, fu], p)
            best_hi = np.minimum(best_hi, hi_k)
        okf = lo_g <= best_hi
        assert okf.all(), (f"{label}: {(~okf).sum()} argmin choices outside the tie band: "
                           f"excess {(e_g - eo)[fv, fu][~okf][:5]}")
        n_flip = len(fu)
    return e_g, band, float(same.mean()), n_flip, n_e


def check_energy(P, S, rho, e_gpu, e_o, band, p, label):
    """The GPU's float32 energies against the float64 ones at the same rho."""
    bad = ~(np.abs(e_gpu.astype(np.float64) - e_o) <= band)
    if bad.any():
        iu, iv = omodel.pixel_grid(P)
        lo, hi = energy_range(P, S, iu[bad], iv[bad], rho[bad], p)
        eg = e_gpu[bad].astype(np.float64)
        ok = (eg >= lo) & (eg <= hi)
        assert ok.all(), (f"{label}: GPU energy off by {np.abs(e_gpu - e_o)[bad][~ok][:5]} "
                          f"(band {band[bad][~ok][:5]}, float32 range "
                          f"{np.stack([lo, hi], 1)[~ok][:3].tolist()})")
    return int(bad.sum())


def check_propagation(P, S, d, p, rs, new, e_g, band, label, chains=None):
    """Step B: every GPU step along the chains of direction d is a valid
    step of the sequential pass from the GPU's rho* (the oracle's float64
    energies, within the tie band; a flipped term widens them to its range).
    chains: optional indices of the chains to walk (all by default).
    Returns the number of steps decided inside the band the other way."""
    cu, cv = odepth.chain_coords(P, d)
    if chains is not None:
        cu, cv = cu[:, chains], cv[:, chains]
    prev = new[cv[0], cu[0]]
    assert np.array_equal(prev, rs[cv[0], cu[0]]), f"{label}: a chain's first pixel moved"
    n_tie = 0
    for m in range(1, cu.shape[0]):
        u, v = cu[m], cv[m]
        g = new[v, u]
        assert np.all((g == rs[v, u]) | (g == prev)), f"{label}: value from nowhere at step {m}"
        Ep = omodel.energy(P, S, u, v, prev, p)
        Eo = e_g[v, u]
        bd = band[v, u]
        took = (g == prev) & (g != rs[v, u])
        kept = (g == rs[v, u]) & (g != prev)
        badt = took & ~(Ep < Eo + bd)
        badk = kept & ~(Ep >= Eo - bd)
        if badt.any() or badk.any():
            sel = badt | badk
            lo_p, hi_p = energy_range(P, S, u[sel], v[sel], prev[sel], p)
            lo_o, hi_o = energy_range(P, S, u[sel], v[sel], rs[v, u][sel], p)
            tk = took[sel]
            okp = np.where(tk, lo_p < hi_o, hi_p >= lo_o)
            assert okp.all(), (f"{label}: propagation step {m} outside the tie band "
                               f"({(~okp).sum()} chains)")
        n_tie += int(np.sum(took & (Ep >= Eo)) + np.sum(kept & (Ep < Eo)))
        prev = g
    return n_tie


def depth_stage(V, ctx, P, S, it, d, p, rep, label):
    """Depth M-step `it` along direction d from state S (the GPU's)."""
    V.vd_depth_mstep(ctx, it, d)
    rs = np.zeros((P.H, P.W), np.float32)
    es = np.zeros((P.H, P.W), np.float32)
    V.vd_get_depth_candidates(ctx, rs, es)
    new = np.zeros((P.H, P.W), np.float32)
    V.vd_get_inv_depth(ctx, new)
    e_g, band, same, n_flip, n_e = check_argmin(P, S, it, p, rs, es, label)
    n_tie = check_propagation(P, S, d, p, rs, new, e_g, band, label)
    ro_new, _ = odepth.propagate(P, S, rs, e_g, d, p)
    rigid = S.q.max(0) > 0.5
    rel = np.abs(new.astype(np.float64) - ro_new) / ro_new
    rep.add(label, argmin_same=round(same, 5), argmin_slow=n_flip, energy_slow=n_e,
            prop_same=round(float((new == ro_new).mean()), 5), prop_tie_steps=n_tie,
            rho_1e4_rigid=round(float(np.mean(rel[rigid] <= 1e-4)), 5))
    return new


def _chain_view(a, d):
    """[..., H, W] -> [..., chains, L] along the chains of direction d."""
    return a if d in (0, 2) else np.swapaxes(a, -1, -2)


def estep_stage(V, ctx, P, S, d, p, rep, label):
    """Rigidness E-step along direction d from state S (the GPU's, with the
    new depth).  Every posterior within 1e-4 of the oracle's; where one is
    not, its whole chain must lie within 1e-4 of the interval that the
    emissions of `term_ranges` allow (double-float positions, float32 flow
    samples and Fisk ratios): the posterior of a two-state
    chain with gamma >= 1/2 increases with every rigid emission (a
    ferromagnetic chain), so the interval's ends are the oracle's
    forward-backward at all-lowest and at all-highest emissions."""
    V.vd_rigidness_estep(ctx, d)
    q = np.zeros((P.N, P.H, P.W), np.float32)
    qh = np.zeros((P.H, P.W), np.float32)
    C = np.zeros((P.H, P.W), np.float32)
    V.vd_get_rigidness(ctx, q)
    V.vd_get_prior_rigidness(ctx, qh)
    V.vd_get_confidence(ctx, C)
    qo, qho, Co = ohmm.rigidness_estep(P, S, S.rho, d, p)
    err = np.abs(q.astype(np.float64) - qo)
    n_slow, widths, worst = 0, [], 0.0
    kinds = {"flipped": 0, "steep": 0, "other": 0}
    if (err > RIGID_TOL).any():
        iu, iv = omodel.pixel_grid(P)
        tr = term_ranges(P, S.G, iu, iv, S.rho, p, positions="df")
        for t in range(P.N):
            errc = _chain_view(err[t], d)
            chains = np.nonzero((errc > RIGID_TOL).any(1))[0]
            if not len(chains):
                continue
            # entries whose float32 emission is known to 2e-4 relative (a
            # posterior moves by a quarter of that at most) keep the
            # oracle's value; the ill-conditioned ones span their interval
            e1p = tr["e1"][t]
            calm = ~tr["flipped"][t] & (tr["e1_hi"][t] - tr["e1_lo"][t] <= 2e-4 * e1p)
            lo = _chain_view(np.where(calm, e1p, tr["e1_lo"][t]), d)[chains].T   # [L, n]
            hi = _chain_view(np.where(calm, e1p, tr["e1_hi"][t]), d)[chains].T
            e0 = np.full_like(lo, p.outlier_density)
            post_lo = ohmm.forward_backward(lo, e0, p.gamma_stay).T
            post_hi = ohmm.forward_backward(hi, e0, p.gamma_stay).T
            qg = _chain_view(q[t], d)[chains].astype(np.float64)
            ok = (qg >= post_lo - RIGID_TOL) & (qg <= post_hi + RIGID_TOL)
            assert ok.all(), (
                f"{label}: flow {t + 1}: {(~ok).sum()} posteriors outside the float32 interval "
                f"(off the oracle by up to {float(errc[chains].max()):.2e})")
            n_slow += int((errc[chains] > RIGID_TOL).sum())
            widths.append(float((post_hi - post_lo).max()))
            worst = max(worst, float(errc[chains].max()))
            fl = _chain_view(tr["flipped"][t], d)[chains].any(1)
            st = _chain_view(tr["steep"][t], d)[chains].any(1)
            kinds["flipped"] += int(fl.sum())
            kinds["steep"] += int((st & ~fl).sum())
            kinds["other"] += int((~st & ~fl).sum())
    if P.prior_kind != "none":
        assert np.abs(qh.astype(np.float64) - qho).max() <= RIGID_TOL, f"{label}: prior rigidness"
    # Eq. 6 from the GPU's own posteriors
    Cg = (q.astype(np.float64).sum(0) + (qh if P.prior_kind != "none" else 0.0)) / \
        (P.N + (1 if P.prior_kind != "none" else 0))
    assert np.abs(C - Cg).max() <= 1e-6, f"{label}: confidence"
    rep.add(label, q_1e4=round(float(np.mean(err <= RIGID_TOL)), 6), q_slow=n_slow,
            slow_chains=kinds, slow_max_err=f"{worst:.1e}",
            max_interval=f"{max(widths, default=0.0):.1e}")
    return q, qh


def score_range(P, G, rs, p):
    """(E_lo, E_hi): the pose score of Eq. 7's samples (oracle.pose.score)
    over every float32 evaluation: the rounded observation and projection
    move each residual by a few roundings of the coordinates, a point within
    rounding of the camera plane may take either side, and the float32 /
    float64 sums add 2e-6 relative."""
    fx, fy, cx, cy = P.K
    Xc = rs["X"] @ G[:, :3].T + G[:, 3]
    z = Xc[:, 2]
    front = z > ogeo.Z_EPS
    amb = np.abs(z - ogeo.Z_EPS) < ZPLANE_MARGIN
    zf = np.where(front, z, ogeo.Z_EPS * (1 + 1e-9))
    x = fx * Xc[:, 0] / zf + cx
    y = fy * Xc[:, 1] / zf + cy
    rr = np.hypot(rs["xobs"][:, 0] - x, rs["xobs"][:, 1] - y)
    rr = np.where(np.isfinite(rr), rr, 1e30)
    dr = (_lin_pos_err(x, P.W) + _lin_pos_err(y, P.W) + _lin_pos_err(rs["xobs"][:, 0], P.W) +
          _lin_pos_err(rs["xobs"][:, 1], P.W))
    with np.errstate(over="ignore", divide="ignore"):
        l_lo, l_hi = _fisk_interval(
            lambda r: ofisk.inlier_energy(r, rs["alpha"], p.fisk_beta, p.outlier_density), rr, dr)
    l_lo, l_hi = l_lo - MUFU_ERR, l_hi + MUFU_ERR
    can_f = front | amb
    can_b = ~front | amb
    lo = np.minimum(np.where(can_f, l_lo, np.inf), np.where(can_b, ofisk.L_BEHIND, np.inf))
    hi = np.maximum(np.where(can_f, l_hi, -np.inf), np.where(can_b, ofisk.L_BEHIND, -np.inf))
    E_lo = float(np.sum(rs["w"] * np.maximum(lo, 0.0)))
    E_hi = float(np.sum(rs["w"] * hi))
    return E_lo * (1 - 2e-6), E_hi * (1 + 2e-6)


def pose_stage(V, ctx, P, S, it, t, p, rep, label):
    """Pose M-step of frame t from state S (the GPU's); returns the GPU pose."""
    So = S.copy()
    out = opose.pose_mstep_frame(P, So, t, it, p, detail=True)
    st = V.vd_pose_mstep(ctx, it, t)
    poses, en, n = V.vd_get_pose_samples(ctx, p.n_pose_samples)
    assert n == out["n_rigid"], f"{label}: rigid set {n} vs {out['n_rigid']}"
    Gg = np.array(V.vd_get_poses(ctx, P.N), np.float64)
    if out["degenerate"]:
        assert st == V.VD_WARN_DEGENERATE, f"{label}: degenerate on the oracle only"
        assert np.array_equal(Gg[t], S.G[t])
        rep.add(label, n_rigid=n, degenerate=True)
        return Gg[t]
    assert st == V.VD_OK, f"{label}: status {st}"
    mism = 0
    rs, n_e_slow, e_worst = None, 0, 0.0
    for g in range(p.n_pose_samples):
        roots, Es = out["roots"][g], out["root_scores"][g]
        if not roots:
            assert not np.isfinite(en[g]), f"{label}: sample {g} void on the oracle only"
            continue
        k = int(np.argmin(Es))
        srt = np.sort(Es)
        if len(Es) > 1 and srt[1] - srt[0] < 1e-4 * abs(srt[0]):
            continue                   # float32 near-tie between two roots
        dmax = np.abs(poses[g] - roots[k]).max()
        if dmax >= 1e-7:
            mism += 1
            continue
        rel_e = abs(en[g] - Es[k]) / max(abs(Es[k]), 1e-30)
        if rel_e > 2e-5:
            if rs is None:
                rs = opose.rigid_set(P, S, t, p)
            lo_e, hi_e = score_range(P, roots[k], rs, p)
            assert lo_e <= en[g] <= hi_e, (f"{label}: sample {g} energy {en[g]!r} vs {Es[k]!r} "
                                           f"(float32 range {lo_e!r} .. {hi_e!r})")
            n_e_slow += 1
        e_worst = max(e_worst, rel_e)
    assert mism <= max(2, p.n_pose_samples // 8), f"{label}: {mism} samples differ"
    # K6 on its own inputs: the float64 mean-shift (oracle.pose.meanshift)
    # over the GPU's samples from the GPU's start must give the GPU's pose
    fin = np.isfinite(en)
    g0 = int(np.argmin(np.where(fin, en, np.inf)))
    gs = [poses[g] for g in range(p.n_pose_samples) if fin[g]]
    xg, itg = opose.meanshift(gs, poses[g0], p)
    rot_ms, trans_ms = pose_err(xg, Gg[t])
    assert rot_ms < POSE_ROT_TOL and trans_ms < POSE_TRANS_TOL, \
        (f"{label}: mean-shift off by {rot_ms:.2e} rad, {trans_ms:.2e} relative "
         f"on the GPU's own samples ({itg} float64 steps)")
    # against the oracle's own run: equal unless one of the method's discrete
    # choices went the other way within its float32 band -- the start (the
    # best-scoring sample, Eq. 7) or a sample's root -- and then the check
    # above has already held the mean-shift to the bounds on those inputs
    rot, trans = pose_err(So.G[t], Gg[t])
    o_idx = [g for g in range(p.n_pose_samples) if out["roots"][g]]
    og0 = o_idx[int(np.argmin(out["scores"]))]
    o_pose = {g: out["samples"][k] for k, g in enumerate(o_idx)}
    n_diff = sum(1 for g in range(p.n_pose_samples)
                 if (g in o_pose) != bool(fin[g])
                 or (g in o_pose and np.abs(poses[g] - o_pose[g]).max() >= 1e-7))
    start_tie = False
    if og0 != g0:
        if rs is None:
            rs = opose.rigid_set(P, S, t, p)
        a = score_range(P, o_pose[og0], rs, p)
        b = score_range(P, poses[g0], rs, p)
        start_tie = a[0] <= b[1] and b[0] <= a[1]
        assert start_tie or n_diff > 0, \
            (f"{label}: start sample {g0} on the GPU, {og0} on the oracle, float32 "
             f"energy ranges {a} and {b} apart")
    if not (rot < POSE_ROT_TOL and trans < POSE_TRANS_TOL):
        assert start_tie or n_diff > 0, \
            (f"{label}: pose off by {rot:.2e} rad, {trans:.2e} relative with the same "
             f"start and samples (oracle {out.get('ms_iters')} steps, {itg} on the GPU's)")
        rep.discrete += 1
    rep.add(label, n_rigid=n, samples=len(out["samples"]), root_mism=mism,
            energy_rel=f"{e_worst:.1e}", energy_slow=n_e_slow,
            rot=f"{rot:.1e}", trans=f"{trans:.1e}", ms_iters=out.get("ms_iters"),
            ms_own=f"{max(rot_ms, trans_ms):.1e}", start_tie=int(start_tie),
            samples_differ=n_diff)
    return Gg[t]


# ----------------------------------------------------------------- replay
def replay(V, make_ctx_fn, P, p, n_iters, name, check_run=True):
    """Bootstrap and n_iters EM iterations, stage by stage, each compared with
    the oracle from the GPU's state.  make_ctx_fn() returns a fresh context
    with the window's flows and prior pushed.  Returns the report."""
    rep = Report(name)
    ctx = make_ctx_fn()
    try:
        G0 = np.stack([ogeo.IDENTITY] * (P.N + 1))
        rho0 = oem.initial_rho(P, p)
        if P.prior_kind == "none":
            # 8-point pose of X_1 (|tau_1| = 1), then G_t = G_1^t
            T1 = np.array(V.vd_eight_point(ctx), np.float64).reshape(3, 4)
            G1o, _ = oeight.bootstrap_pose(P, p.fisk_alpha0)
            rot, trans = pose_err(G1o, T1)
            assert rot < POSE_ROT_TOL and trans < POSE_TRANS_TOL, \
                f"boot 8-point: {rot:.2e} rad {trans:.2e}"
            rep.add("boot/8pt", rot=f"{rot:.1e}", trans=f"{trans:.1e}")
            G = G0.copy()
            G[1] = T1
            for t in range(2, P.N + 1):
                G[t] = ogeo.compose(T1, G[t - 1])
            q = np.zeros((P.N, P.H, P.W), np.float32)
            q[0] = 1.0
            S = omodel.State(rho=rho0, q=q, qhat=np.ones((P.H, P.W), np.float32), G=G)
            V.vd_set_poses(ctx, G.reshape(-1, 12))
            V.vd_set_state(ctx, S.rho, S.q, S.qhat)
            S.rho = depth_stage(V, ctx, P, S, -1, 0, p, rep, "boot/depth")
            S.q = np.ones((P.N, P.H, P.W), np.float32)
            V.vd_set_state(ctx, S.rho, S.q, S.qhat)
        else:
            S = omodel.State(rho=rho0, q=np.ones((P.N, P.H, P.W), np.float32),
                             qhat=np.ones((P.H, P.W), np.float32), G=G0.copy())
            V.vd_set_state(ctx, S.rho, S.q, S.qhat)
            V.vd_set_poses(ctx, S.G.reshape(-1, 12))
        for t in range(1, P.N + 1):
            S.G[t] = pose_stage(V, ctx, P, S, -1, t, p, rep, f"boot/pose{t}")
        for it in range(n_iters):
            d = it % 4
            S.rho = depth_stage(V, ctx, P, S, it, d, p, rep, f"it{it}/depth(d{d})")
            S.q, S.qhat = estep_stage(V, ctx, P, S, d, p, rep, f"it{it}/estep")
            for t in range(1, P.N + 1):
                S.G[t] = pose_stage(V, ctx, P, S, it, t, p, rep, f"it{it}/pose{t}")
        final = read_state(V, ctx, P)
    finally:
        V.vd_destroy(ctx)
    if check_run:
        # the uninterrupted run reaches the chained GPU state bit for bit
        ctx2 = make_ctx_fn()
        try:
            V.vd_bootstrap(ctx2)
            V.vd_run_em(ctx2, n_iters)
            run = read_state(V, ctx2, P)
        finally:
            V.vd_destroy(ctx2)
        assert np.array_equal(run.rho, final.rho), "vd_run_em depth differs from the chained run"
        assert np.array_equal(run.q, final.q), "vd_run_em rigidness differs from the chained run"
        assert np.array_equal(run.G, final.G), "vd_run_em poses differ from the chained run"
        rep.add("run", identical_to_chained=True)
    rep.final = final
    return rep

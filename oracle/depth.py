"""Depth M-step: hypothesis sampling, per-pixel argmin and chain propagation.

Sec. III-A "Hierarchical Propagation Scheme": the image is cut into 1-D
chains whose direction alternates between iterations; in the M-step depth
values are randomly sampled and propagated along each chain (PatchMatch
style).  Eq. 5 selects, per pixel, the candidate with the lowest
flow + prior energy.

Reading fixed here (the sampling distribution is not printed):
  * K candidates per pixel and iteration.  Slot 0 is the current value; slot 1
    is the prior's inverse depth where the prior is valid; every other slot
    k >= 1 draws the 32-bit word k-1 of the Philox stream
    (counter = (c0, iteration code, TAG_DEPTH, (k-1) >> 2), word (k-1) & 3)
    with c0 = j - (u mod share) (share = 1: one stream per pixel).
    Slots 1 .. floor((K-1)/2) are uniform in [rho_min, rho_max]; the rest are
    local perturbations rho_j (1 + s_i (2u - 1)), s_i = max(0.5 * 2^-i, 1/64).
    Every candidate is clamped to [rho_min, rho_max].  These values are formed
    in float32 with one rounding per operation, exactly as stored.
  * Step A (parallel): rho*_j = argmin_k E_j(c_k), lowest slot on ties.
  * Step B (sequential per chain): walking the chain in its direction,
    rho_new = rho*_j unless E_j(predecessor's rho_new) < E_j(rho*_j).  This
    equals sequential propagation over the whole candidate set, because an
    argmin over a set does not depend on evaluation order.
  * Directions: d = i mod 4 with 0: left->right (rows), 1: top->bottom
    (columns), 2: right->left, 3: bottom->top.
  * Hierarchical option (Sec. III-A, 3x speed-up claim): a global pass on a
    coarse grid of representative pixels (s*uc, s*vc), then every pixel
    compares its rho* with its cell's coarse value, then propagation restarts
    at every multiple of `window` along the chain.
"""
from __future__ import annotations

import numpy as np

from . import model, philox


def perturb_scale(it):
    """s_i; the bootstrap (it < 0) uses the iteration-0 scale."""
    if it < 0:
        it = 0
    return np.float32(max(0.5 * 2.0 ** (-it), 1.0 / 64.0))


def iter_code(it):
    return philox.ITER_BOOT if it < 0 else int(it)


def hypotheses(P: model.Problem, rho_cur, it, p: model.Params, iu=None, iv=None):
    """Candidate inverse depths, float32 [K, H, W] (or [K, n] for the pixels
    (iu, iv) when given; rho_cur is then the [n] current values)."""
    K = p.n_hyp
    if iu is None:
        iv, iu = np.mgrid[0:P.H, 0:P.W]
    iu = np.asarray(iu)
    iv = np.asarray(iv)
    rho_cur = np.asarray(rho_cur, np.float32)
    j = (iv.astype(np.int64) * P.W + iu).astype(np.uint64)
    c0 = j - (iu % p.sample_share).astype(np.uint64)
    k0, k1 = philox.seed_key(p.seed)
    rmin, rmax = p.f32("rho_min"), p.f32("rho_max")
    rng = np.float32(rmax - rmin)
    s = perturb_scale(it)
    n_unif = (K - 1) // 2
    cands = np.empty((K,) + iu.shape, np.float32)
    cands[0] = np.clip(rho_cur, rmin, rmax)
    words = None
    for k in range(1, K):
        w = k - 1
        if w % 4 == 0:
            words = philox.philox4x32_10(c0, iter_code(it), philox.TAG_DEPTH, w >> 2, k0, k1)
        u = philox.u24_float(words[w % 4])
        if k <= n_unif:
            c = rmin + np.float32(u * rng)
        else:
            a = np.float32(np.float32(2.0) * u) - np.float32(1.0)
            c = rho_cur * np.float32(np.float32(1.0) + np.float32(s * a))
        cands[k] = np.clip(c.astype(np.float32), rmin, rmax)
    prho = P.prior_rho()
    if prho is not None and K > 1:
        pr = prho[iv, iu]
        ok = np.isfinite(pr)
        cands[1] = np.where(ok, np.clip(pr, rmin, rmax), cands[1])
    return cands


def argmin_candidates(P, S: model.State, cands, p):
    """Step A: per-pixel argmin over the candidate slots (ties: lowest slot)."""
    iu, iv = model.pixel_grid(P)
    best_E = np.full((P.H, P.W), np.inf)
    best = np.zeros((P.H, P.W), np.float32)
    best_k = np.zeros((P.H, P.W), np.int32)
    for k in range(cands.shape[0]):
        E = model.energy(P, S, iu, iv, cands[k], p)
        take = E < best_E
        best_E = np.where(take, E, best_E)
        best = np.where(take, cands[k], best)
        best_k = np.where(take, k, best_k)
    return best, best_E, best_k


def chain_coords(P, direction):
    """Pixel coordinates of every chain, ordered along the chain.

    Returns iu, iv of shape [L, M]: position m along chain, chain index."""
    H, W = P.H, P.W
    if direction in (0, 2):       # rows
        iu = np.repeat(np.arange(W)[:, None], H, axis=1)
        iv = np.repeat(np.arange(H)[None, :], W, axis=0)
    else:                         # columns
        iv = np.repeat(np.arange(H)[:, None], W, axis=1)
        iu = np.repeat(np.arange(W)[None, :], H, axis=0)
    if direction in (2, 3):
        iu, iv = iu[::-1], iv[::-1]
    return iu, iv


def propagate(P, S: model.State, rho_star, E_star, direction, p, restart=None):
    """Step B: sequential propagation along the chains of `direction`.

    restart: optional chain length after which propagation starts afresh
    (position m with m % restart == 0 takes its own candidate)."""
    iu, iv = chain_coords(P, direction)
    L = iu.shape[0]
    new = rho_star.copy()
    E_new = E_star.copy()
    cur = rho_star[iv[0], iu[0]].copy()
    for m in range(1, L):
        u, v = iu[m], iv[m]
        if restart is not None and m % restart == 0:
            cur = rho_star[v, u].copy()
            continue
        E_c = model.energy(P, S, u, v, cur, p)
        take = E_c < E_star[v, u]
        cur = np.where(take, cur, rho_star[v, u]).astype(np.float32)
        new[v, u] = cur
        E_new[v, u] = np.where(take, E_c, E_star[v, u])
    return new, E_new


def hierarchical(P, S, rho_star, E_star, direction, p):
    """Hierarchical propagation: coarse global pass + local windows."""
    s = p.hier_scale
    Wc, Hc = (P.W + s - 1) // s, (P.H + s - 1) // s
    ru = np.minimum(np.arange(Wc) * s, P.W - 1)
    rv = np.minimum(np.arange(Hc) * s, P.H - 1)
    # 1) global propagation on the representative pixels
    cu, cv = np.meshgrid(ru, rv)
    coarse = rho_star[cv, cu].copy()
    coarse_E = E_star[cv, cu].copy()
    if direction in (0, 2):
        order = range(Wc) if direction == 0 else range(Wc - 1, -1, -1)
        order = list(order)
        cur = coarse[:, order[0]].copy()
        for m in order[1:]:
            E_c = model.energy(P, S, cu[:, m], cv[:, m], cur, p)
            take = E_c < coarse_E[:, m]
            cur = np.where(take, cur, coarse[:, m]).astype(np.float32)
            coarse[:, m] = cur
    else:
        order = range(Hc) if direction == 1 else range(Hc - 1, -1, -1)
        order = list(order)
        cur = coarse[order[0], :].copy()
        for m in order[1:]:
            E_c = model.energy(P, S, cu[m, :], cv[m, :], cur, p)
            take = E_c < coarse_E[m, :]
            cur = np.where(take, cur, coarse[m, :]).astype(np.float32)
            coarse[m, :] = cur
    # 2) every pixel compares its own candidate with its cell's coarse value
    iu, iv = model.pixel_grid(P)
    up = coarse[iv // s, iu // s]
    E_up = model.energy(P, S, iu, iv, up, p)
    take = E_up < E_star
    mid = np.where(take, up, rho_star).astype(np.float32)
    mid_E = np.where(take, E_up, E_star)
    # 3) local propagation in windows of hier_window pixels
    return propagate(P, S, mid, mid_E, direction, p, restart=p.hier_window)


def depth_mstep(P, S: model.State, it, direction, p):
    """One depth M-step; returns (rho_new, E_new, rho_star, E_star)."""
    cands = hypotheses(P, S.rho, it, p)
    rho_star, E_star, _ = argmin_candidates(P, S, cands, p)
    if p.hierarchical:
        rho_new, E_new = hierarchical(P, S, rho_star, E_star, direction, p)
    else:
        rho_new, E_new = propagate(P, S, rho_star, E_star, direction, p)
    return rho_new, E_new, rho_star, E_star

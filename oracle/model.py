"""Problem, parameters, state and the per-pixel energy of the VOLDOR+ model.

Sec. III-A, Eq. 1-2: observed flows X_1..X_N of a window, poses T, the
reference-frame depth theta and rigidness maps W; optional depth priors
theta_hat with their own rigidness W_hat.  Here inverse depth rho = 1/theta
is the per-pixel unknown.

Energy of pixel j at candidate inverse depth c (Eq. 5 = flow term + Eq. 4):
    E_j(c) = sum_t q_t^j l_t^j(c) + w_hat^j l_hat^j(c)
  * l_t^j: maximum-inlier energy of the flow residual of X_t (fisk.py).  The
    track of j starts at x_0 = j; x_t = pi(K (R_t r_j + c tau_t)).  X_t is
    sampled bilinearly at x_{t-1}; the residual is X_t(x_{t-1}) - (x_t - x_{t-1}).
    The term has no observation (l = 0) if x_{t-1} is outside the image or
    behind camera t-1; an observed term whose point is behind camera t costs
    l = L_BEHIND (fisk.py).
  * l_hat^j: prior term.  Stereo (Sec. III-A last paragraph of "Geometric
    Priors" and Sec. IV): the disparity d_hat is the x-flow of a rectified pair
    with baseline b, so its residual |d_hat - fx b c| uses the same Fisk model
    as flow.  RGB-D (Eq. 3): Gaussian-uniform mixture on 1/theta_hat - c with
    sigma = c_sigma rho_hat and uniform density 1/(w rho_hat); with T_hat = I
    the reprojected pixel is j itself and phi_z = 1/c.
  * w_hat^j = q_hat^j * C_prior^j (Sec. III-A "Depth Map Confidence": the prior's
    confidence multiplies its rigidness weight); 0 at prior holes.

State storage precision follows the library: rho, q, q_hat, C are float32
maps, poses are float64.  All arithmetic here is float64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import fisk, geometry


@dataclasses.dataclass
class Params:
    fisk_alpha0: float = 0.5
    fisk_alpha1: float = 0.0
    fisk_beta: float = 2.0
    outlier_density: float = 1e-3      # P0, per px^2
    gamma_stay: float = 0.95           # HMM probability of keeping the rigidness state
    rho_min: float = 0.01
    rho_max: float = 1.0
    n_hyp: int = 64                    # K, hypotheses per pixel per iteration
    n_pose_samples: int = 64           # S, P3P samples per frame
    pose_sigma_rot: float = 0.01       # mean-shift kernel, rad
    pose_sigma_trans_rel: float = 0.01 # mean-shift kernel, fraction of |tau|
    pose_sigma_trans_abs: float = 1e-3
    sample_share: int = 1              # pixels of a row segment that share depth draws
    prior_c_sigma: float = 0.01
    prior_w_uniform: float = 2.0
    hierarchical: int = 0
    hier_scale: int = 4
    hier_window: int = 32
    seed: int = 0

    def f32(self, name):
        return np.float32(getattr(self, name))


@dataclasses.dataclass
class Problem:
    W: int
    H: int
    N: int
    K: tuple                     # (fx, fy, cx, cy)
    flow: np.ndarray             # [N, H, W, 2] float32
    prior_kind: str = "none"     # "none" | "stereo" | "rgbd"
    prior_value: np.ndarray | None = None  # stereo: disparity (px); rgbd: depth (m); float32, NaN = hole
    prior_conf: np.ndarray | None = None   # optional confidence of the prior, float32 [H, W]
    baseline: float = 0.0

    def __post_init__(self):
        self.rays = geometry.rays(self.W, self.H, self.K)

    @property
    def fxb32(self):
        """fx * b rounded to float32 (the stereo prior's scale, as stored)."""
        return np.float32(self.K[0] * self.baseline)

    def prior_rho(self):
        """Inverse depth of the prior as float32, NaN at holes."""
        if self.prior_kind == "none":
            return None
        v = self.prior_value.astype(np.float32)
        with np.errstate(invalid="ignore", divide="ignore"):
            ok = np.isfinite(v) & (v > 0)
            if self.prior_kind == "stereo":
                r = v / self.fxb32
            else:
                r = np.float32(1.0) / v
        return np.where(ok, r, np.float32(np.nan)).astype(np.float32)


@dataclasses.dataclass
class State:
    rho: np.ndarray      # [H, W] float32
    q: np.ndarray        # [N, H, W] float32
    qhat: np.ndarray     # [H, W] float32
    G: np.ndarray        # [N+1, 3, 4] float64, G[0] = identity
    C: np.ndarray | None = None

    def copy(self):
        return State(self.rho.copy(), self.q.copy(), self.qhat.copy(), self.G.copy(),
                     None if self.C is None else self.C.copy())


def problem_from_window(win, prior="auto"):
    """Build a Problem from a synth.Window."""
    kind, val, b = "none", None, 0.0
    if prior in ("auto", "stereo") and win.stereo_disp is not None:
        kind, val, b = "stereo", win.stereo_disp, win.stereo_baseline
    elif prior in ("auto", "rgbd") and win.depth_prior is not None:
        kind, val = "rgbd", win.depth_prior
    return Problem(win.W, win.H, win.N, win.intrinsics, win.flow, kind, val, None, b)


def flow_terms(P: Problem, G, iu, iv, rho, p: Params):
    """Per-flow energy l_t and inlier emission p1 for pixels (iu, iv) at rho.

    iu, iv: integer arrays (same shape S); rho: float array of shape S.
    Returns (ell[N, *S], e1[N, *S], ok[N, *S])."""
    iu = np.asarray(iu)
    iv = np.asarray(iv)
    rho = np.asarray(rho, np.float64)
    r = P.rays[iv, iu]
    xp = iu.astype(np.float64)
    yp = iv.astype(np.float64)
    front_prev = np.ones(iu.shape, bool)
    ells, e1s, oks = [], [], []
    for t in range(1, P.N + 1):
        x, y, front = geometry.dehom(geometry.project_h(P.K, G[t], r, rho))
        if t == 1:
            F = P.flow[0][iv, iu].astype(np.float64)
            obs = np.ones(iu.shape, bool)
        else:
            obs = front_prev & geometry.inside(xp, yp, P.W, P.H)
            F = geometry.bilinear(P.flow[t - 1], np.where(obs, xp, 0.0), np.where(obs, yp, 0.0))
        ok = obs & front
        with np.errstate(invalid="ignore"):
            dx = F[..., 0] - (x - xp)
            dy = F[..., 1] - (y - yp)
        rr = np.sqrt(np.where(ok, dx * dx + dy * dy, 0.0))
        alpha = p.fisk_alpha0 + p.fisk_alpha1 * np.hypot(F[..., 0], F[..., 1])
        ell = np.where(ok, fisk.inlier_energy(rr, alpha, p.fisk_beta, p.outlier_density),
                       np.where(obs, fisk.L_BEHIND, 0.0))
        e1 = np.where(ok, fisk.residual_density(rr, alpha, p.fisk_beta),
                      np.where(obs, 0.0, p.outlier_density))
        ells.append(ell)
        e1s.append(e1)
        oks.append(ok)
        xp, yp, front_prev = x, y, front
    return np.stack(ells), np.stack(e1s), np.stack(oks)


def prior_terms(P: Problem, iu, iv, rho, p: Params):
    """Prior energy l_hat, inlier emission e1_hat, outlier emission e0_hat, valid mask."""
    rho = np.asarray(rho, np.float64)
    shape = np.broadcast(np.asarray(iu), rho).shape
    if P.prior_kind == "none":
        z = np.zeros(shape)
        return z, z, z, np.zeros(shape, bool)
    rhat32 = P.prior_rho()[iv, iu]
    valid = np.isfinite(rhat32)
    rhat = np.where(valid, rhat32.astype(np.float64), 1.0)
    if P.prior_kind == "stereo":
        d = np.where(valid, P.prior_value[iv, iu].astype(np.float64), 0.0)
        rr = np.abs(d - float(P.fxb32) * rho)
        ell = fisk.inlier_energy(rr, p.fisk_alpha0, p.fisk_beta, p.outlier_density)
        e1 = fisk.residual_density(rr, p.fisk_alpha0, p.fisk_beta)
        e0 = np.full(shape, p.outlier_density)
    else:
        res = rhat - rho
        sig = p.prior_c_sigma * rhat
        logk = math.log(math.sqrt(2 * math.pi) * p.prior_c_sigma / p.prior_w_uniform)
        z = res * res / (2 * sig * sig) + logk
        ell = np.logaddexp(0.0, z)                       # log(1 + exp(z))
        e1 = np.exp(-res * res / (2 * sig * sig)) / (math.sqrt(2 * math.pi) * sig)
        e0 = 1.0 / (p.prior_w_uniform * rhat)
    return (np.where(valid, ell, 0.0), np.where(valid, e1, 0.0), np.where(valid, e0, 1.0), valid)


def prior_weight(P: Problem, S: State, iu, iv):
    if P.prior_kind == "none":
        return np.zeros(np.asarray(iu).shape)
    w = S.qhat[iv, iu].astype(np.float64)
    if P.prior_conf is not None:
        w = w * P.prior_conf[iv, iu].astype(np.float64)
    valid = np.isfinite(P.prior_rho()[iv, iu])
    return np.where(valid, w, 0.0)


def energy(P: Problem, S: State, iu, iv, rho, p: Params):
    """E_j(rho) at pixels (iu, iv) (Eq. 5 criterion, float64)."""
    ell, _, _ = flow_terms(P, S.G, iu, iv, rho, p)
    q = S.q[:, iv, iu].astype(np.float64)
    E = np.sum(q * ell, axis=0)
    if P.prior_kind != "none":
        lh, _, _, _ = prior_terms(P, iu, iv, rho, p)
        E = E + prior_weight(P, S, iu, iv) * lh
    return E


def pixel_grid(P: Problem):
    iv, iu = np.mgrid[0:P.H, 0:P.W]
    return iu, iv

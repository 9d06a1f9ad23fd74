"""Pose covariance from the P3P samples (test infrastructure).

Sec. III-A "Uncertainty-aware Pose Estimation": the uncertainty Sigma_t of
each camera pose is estimated by starting from the mean-shift result and
iteratively fitting a Gaussian to the pose samples, discarding the samples
outside 3 sigma and keeping every eigenvalue of Sigma_t above an epsilon.

Readings fixed here (the paper names the steps, not these details):
  * samples: the kept root of every sample of the frame's last pose M-step
    that has one (finite energy); poses are absolute (reference -> frame).
  * the Gaussian lives in the tangent space at its mean mu: a sample's
    coordinates are d = log(mu^-1 T) in se(3) (rotation vector, then the
    translation part, the convention of geometry.se3_log).
  * start: mu = the mean-shift mode; Sigma = the mean-shift kernel's
    covariance there, diag(s_rot^2 x3, s_t^2 x3) with
    s_t = s_rel |tau_mode| + s_abs.
  * one round: d for every sample; inliers: d^T Sigma^-1 d <= 9 (3 sigma);
    if the inlier set equals the previous round's, stop (converged); with
    fewer than 7 inliers (a 6-D covariance needs 7), stop and report the
    frame degenerate, keeping the last fit; else mu <- the Frechet mean of
    the inliers (mu <- mu exp(mean of the inliers' d) until the step is below
    1e-12, at most MEAN_ITERS times), Sigma <- (1/n) sum d d^T over the
    inliers with d taken at that mu (the maximum-likelihood fit), every
    eigenvalue raised to eps.  At most MAX_ROUNDS rounds.
  * float64 throughout.
"""
from __future__ import annotations

import numpy as np

from . import geometry

MAX_ROUNDS = 50
MEAN_ITERS = 50
MEAN_TOL = 1e-12
MIN_INLIERS = 7


def kernel_covariance(mode, sigma_rot, sigma_rel, sigma_abs):
    st = sigma_rel * float(np.linalg.norm(mode[:, 3])) + sigma_abs
    return np.diag([sigma_rot ** 2] * 3 + [st ** 2] * 3)


def floor_eigenvalues(S, eps):
    S = 0.5 * (S + S.T)
    w, V = np.linalg.eigh(S)
    return (V * np.maximum(w, eps)) @ V.T


def _coords(mu, samples):
    mi = geometry.inverse(mu)
    return np.array([geometry.se3_log(geometry.compose(mi, T)) for T in samples])


def fit(samples, mode, sigma0, eps, max_rounds=MAX_ROUNDS):
    """(mu, Sigma, n_inliers, rounds, degenerate) for the list of sample poses."""
    mu = np.array(mode, np.float64)
    S = floor_eigenvalues(np.array(sigma0, np.float64), eps)
    samples = [np.asarray(T, np.float64) for T in samples]
    if len(samples) < MIN_INLIERS:
        return mu, S, len(samples), 0, True
    prev = None
    n_in = 0
    for r in range(1, max_rounds + 1):
        d = _coords(mu, samples)
        m = np.einsum("gi,ij,gj->g", d, np.linalg.inv(S), d)
        inl = m <= 9.0
        n_in = int(inl.sum())
        if prev is not None and np.array_equal(inl, prev):
            return mu, S, n_in, r, False
        if n_in < MIN_INLIERS:
            return mu, S, n_in, r, True
        kept = [T for T, k in zip(samples, inl) if k]
        dn = d[inl]
        for _ in range(MEAN_ITERS):
            step = dn.mean(axis=0)
            mu = geometry.compose(mu, geometry.se3_exp(step))
            dn = _coords(mu, kept)
            if np.linalg.norm(step) < MEAN_TOL:
                break
        S = floor_eigenvalues(dn.T @ dn / n_in, eps)
        prev = inl
    return mu, S, n_in, max_rounds, False

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
  * start: mu = the mean-shift mode; Sigma = a robust diagonal fit of all
    the samples there, diag(s_i^2) with s_i = 1.4826 median_g |d_gi| (the
    median absolute deviation from the mode, which equals sigma_i for a
    Gaussian and ignores up to half of the samples as outliers).  The
    mean-shift kernel's covariance is not a usable start: the P3P samples of
    early iterations spread far wider than the kernel, and a 3-sigma window
    of the kernel then holds only the mode's own sample.
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


def robust_start(samples, mode):
    """diag((1.4826 median_g |d_gi|)^2), d_g = log(mode^-1 T_g)."""
    d = _coords(np.asarray(mode, np.float64), samples)
    s = 1.4826 * np.median(np.abs(d), axis=0)
    return np.diag(s * s)


def floor_eigenvalues(S, eps):
    S = 0.5 * (S + S.T)
    w, V = np.linalg.eigh(S)
    return (V * np.maximum(w, eps)) @ V.T


def _coords(mu, samples):
    if not len(samples):
        return np.zeros((0, 6))
    mi = geometry.inverse(mu)
    return np.array([geometry.se3_log(geometry.compose(mi, T)) for T in samples])


def fit(samples, mode, eps, sigma0=None, max_rounds=MAX_ROUNDS):
    """(mu, Sigma, n_inliers, rounds, degenerate) for the list of sample
    poses; sigma0 replaces the robust start when given."""
    mu = np.array(mode, np.float64)
    samples = [np.asarray(T, np.float64) for T in samples]
    if len(samples) < MIN_INLIERS:
        S0 = np.zeros((6, 6)) if sigma0 is None else np.array(sigma0, np.float64)
        return mu, floor_eigenvalues(S0, eps), len(samples), 0, True
    S0 = robust_start(samples, mu) if sigma0 is None else np.array(sigma0, np.float64)
    S = floor_eigenvalues(S0, eps)
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

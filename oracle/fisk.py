"""Fisk (log-logistic) residual model and the maximum-inlier energy.

Sec. III-A ("VOLDOR+"): the end-point error (EPE) between an observed flow
vector and the rigid flow implied by depth and pose follows a Fisk
distribution; depth and pose are scored in a maximum-inlier form (Eq. 4 shows
the form for depth priors: minus the log of the inlier likelihood over the sum
of inlier and outlier likelihoods, weighted by the rigidness posterior).

Readings fixed here (the paper defers the exact expressions to VOLDOR):
  * EPE r = |d| of the 2-D residual vector d.  r ~ Fisk(alpha, beta) with a
    uniform direction, so the density of the residual VECTOR is
        p1(d) = f_Fisk(|d|) / (2 pi |d|)
              = beta / (2 pi alpha^2) * s^(beta-2) / (1 + s^beta)^2,  s = |d|/alpha.
    (Using the scalar Fisk pdf of |d| directly would make a zero residual
    impossible for beta > 1 and bias every estimate away from exact flow.)
    For beta != 2, s is floored at 1e-6 / alpha to keep s^(beta-2) finite.
  * scale alpha = alpha0 + alpha1 * |observed flow|.
  * outliers have a constant density P0 (per px^2) over the residual plane.
  * energy of one term: l = -log(p1 / (p1 + P0)) = log(1 + P0 / p1).
  * a term of X_t exists only if the track's frame t-1 position x_{t-1} is in
    front of camera t-1 and inside the image (always for t = 1, x_0 = j):
      - no observation: the term contributes l = 0, and in the E-step both
        emissions equal P0 (the rigidness there comes from the chain alone);
      - observed, but the candidate puts the point behind camera t: the rigid
        model cannot explain the observation, l = L_BEHIND (a large constant)
        and the rigid emission is 0;
      - otherwise the Fisk terms above.
"""
from __future__ import annotations

import math

import numpy as np

LOG2 = math.log(2.0)
R_FLOOR = 1e-6
L_BEHIND = 64.0


def fisk_pdf(x, alpha, beta):
    """Fisk density of a non-negative scalar x."""
    x = np.asarray(x, np.float64)
    z = x / alpha
    return (beta / alpha) * z ** (beta - 1) / (1.0 + z ** beta) ** 2


def fisk_cdf(x, alpha, beta):
    x = np.asarray(x, np.float64)
    with np.errstate(divide="ignore"):
        return 1.0 / (1.0 + (x / alpha) ** (-beta))


def residual_density(r, alpha, beta):
    """p1: density of a 2-D residual vector of length r (see module doc)."""
    r = np.asarray(r, np.float64)
    if beta != 2.0:
        r = np.maximum(r, R_FLOOR)
    s = r / alpha
    return beta / (2.0 * math.pi * alpha * alpha) * s ** (beta - 2.0) / (1.0 + s ** beta) ** 2


def inlier_energy(r, alpha, beta, p0):
    """l = log(1 + P0 / p1(r)) for observed (in-view) terms."""
    return np.log1p(p0 / residual_density(r, alpha, beta))


def inlier_posterior(r, alpha, beta, p0):
    """p1 / (p1 + P0): posterior of 'inlier' for one isolated observation."""
    p1 = residual_density(r, alpha, beta)
    return p1 / (p1 + p0)

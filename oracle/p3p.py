"""Minimal 3-point absolute pose (P3P).

Eq. 7 samples pose hypotheses from P3P instances (the paper uses the AP3P
solver of Ke & Roumeliotis; any exact P3P solver returns the same set of
solutions, so this oracle uses the older distance formulation of Grunert as
reviewed by Haralick et al., IJCV 1994).

Given unit bearings f_i in the camera and world points P_i, the camera-frame
distances s_i satisfy the law of cosines on each pair.  With s2 = u s1 and
s3 = v s1 the ratios of these equations give two conics in (u, v); their
resultant in u is a polynomial of degree <= 4 in v.  Every real positive root
v with its common u and s1 = b / sqrt(1 + v^2 - 2 v cos(beta)) gives camera
points Q_i = s_i f_i, and the rigid motion Q = R P + tau follows from the three
point pairs (Kabsch / Procrustes via an SVD).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import polynomial as Pl


def _resultant_quadratics(p, q):
    """Resultant of p2 u^2 + p1 u + p0 and q2 u^2 + q1 u + q0 (coefficients are
    polynomials in v, low order first): (p2 q0 - p0 q2)^2 - (p2 q1 - p1 q2)(p1 q0 - p0 q1)."""
    p2, p1, p0 = p
    q2, q1, q0 = q
    m = Pl.polymul
    s = Pl.polysub
    A = s(m(p2, q0), m(p0, q2))
    B = s(m(p2, q1), m(p1, q2))
    C = s(m(p1, q0), m(p0, q1))
    return s(m(A, A), m(B, C))


def kabsch(P, Q):
    """R, tau minimising sum |Q_i - (R P_i + tau)|^2 (proper rotation)."""
    Pm, Qm = P.mean(0), Q.mean(0)
    Hm = (P - Pm).T @ (Q - Qm)
    U, _, Vt = np.linalg.svd(Hm)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(Vt.T @ U.T))])
    R = Vt.T @ D @ U.T
    return R, Qm - R @ Pm


def solve(bearings, points, imag_tol=1e-7):
    """All P3P solutions as a list of [3, 4] poses (world -> camera)."""
    f = np.asarray(bearings, np.float64)
    f = f / np.linalg.norm(f, axis=1, keepdims=True)
    X = np.asarray(points, np.float64)
    a2 = float(np.sum((X[1] - X[2]) ** 2))
    b2 = float(np.sum((X[0] - X[2]) ** 2))
    c2 = float(np.sum((X[0] - X[1]) ** 2))
    ca, cb, cg = float(f[1] @ f[2]), float(f[0] @ f[2]), float(f[0] @ f[1])
    if min(a2, b2, c2) <= 0:
        return []
    # conic from (2)/(3): -b2 u^2 + 2 b2 cg u + c2 (1 + v^2 - 2 v cb) - b2 = 0
    p = ([-b2], [2 * b2 * cg], [c2 - b2, -2 * c2 * cb, c2])
    # conic from (1)/(2): b2 u^2 - 2 b2 ca v u + b2 v^2 - a2 (1 + v^2 - 2 v cb) = 0
    q = ([b2], [0.0, -2 * b2 * ca], [-a2, 2 * a2 * cb, b2 - a2])
    res = np.trim_zeros(_resultant_quadratics(p, q), "b")
    if len(res) < 2:
        return []
    roots = np.roots(res[::-1])
    sols = []
    for v in roots:
        if abs(v.imag) > imag_tol * (1 + abs(v.real)):
            continue
        v = float(v.real)
        # two Newton steps on the resultant polish the companion-matrix root
        dres = Pl.polyder(res)
        for _ in range(2):
            dv = Pl.polyval(v, dres)
            if dv != 0.0:
                v = v - Pl.polyval(v, res) / dv
        if v <= 0:
            continue
        p0 = c2 * (1 + v * v - 2 * v * cb) - b2
        q1 = -2 * b2 * ca * v
        q0 = b2 * v * v - a2 * (1 + v * v - 2 * v * cb)
        den = b2 * (2 * b2 * cg) - (-b2) * q1
        if abs(den) < 1e-300:
            continue
        u = ((-b2) * q0 - b2 * p0) / den
        if u <= 0:
            continue
        d = 1 + v * v - 2 * v * cb
        if d <= 0:
            continue
        s1 = np.sqrt(b2 / d)
        Q = np.stack([s1 * f[0], u * s1 * f[1], v * s1 * f[2]])
        R, tau = kabsch(X, Q)
        sols.append(np.concatenate([R, tau[:, None]], axis=1))
    return sols

"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test ties one oracle function to a published value, a closed form, an
invariant, a brute-force enumeration or a special case, chosen so that a
plausible slip (a dropped term, a wrong sign or index) fails.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import depth, eightpoint, em, fisk, geometry, hmm, model, p3p, philox, pose

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(v[0], v[1], v[2], v[3], v[4], v[5])
        assert [int(o) for o in out] == v[6:10]


def test_philox_u24_and_pick_are_exact():
    w = np.array([0, 255, 256, 0xFFFFFFFF], np.uint32)
    u = philox.u24_float(w)
    assert u.dtype == np.float32
    assert list(u) == [0.0, 0.0, 2.0 ** -24, (2 ** 24 - 1) * 2.0 ** -24]
    assert int(philox.index_pick(0xFFFFFFFF, 7)) == 6
    assert int(philox.index_pick(0, 7)) == 0
    # (x * n) >> 32 hits every bucket of [0, n) with the right multiplicity
    n = 5
    xs = np.arange(0, 2 ** 32, 2 ** 20, dtype=np.uint64)
    counts = np.bincount(philox.index_pick(xs, n).astype(np.int64), minlength=n)
    assert counts.sum() == len(xs) and counts.min() >= len(xs) // n - 1


# ---------------------------------------------------------------- Fisk model
@pytest.mark.parametrize("alpha,beta", [(0.5, 2.0), (1.0, 2.0), (0.7, 1.5), (2.0, 3.0)])
def test_fisk_pdf_normalises_and_cdf_closed_form(alpha, beta):
    tot, err = integrate.quad(lambda x: fisk.fisk_pdf(x, alpha, beta), 0, np.inf, limit=200)
    assert abs(tot - 1.0) < 1e-10
    for x in [0.1 * alpha, alpha, 3.7 * alpha]:
        c, _ = integrate.quad(lambda s: fisk.fisk_pdf(s, alpha, beta), 0, x)
        assert abs(c - fisk.fisk_cdf(x, alpha, beta)) < 1e-10
    assert abs(fisk.fisk_cdf(alpha, alpha, beta) - 0.5) < 1e-15      # median = alpha


@pytest.mark.parametrize("alpha,beta", [(0.5, 2.0), (1.0, 2.0), (0.8, 2.5)])
def test_residual_density_is_a_planar_density(alpha, beta):
    # integral over the plane in polar coordinates: int p1(r) 2 pi r dr = 1
    tot, _ = integrate.quad(lambda r: fisk.residual_density(r, alpha, beta) * 2 * math.pi * r,
                            0, np.inf, limit=200)
    assert abs(tot - 1.0) < 1e-9
    # and p1(r) 2 pi r is the Fisk pdf of the radius
    r = np.array([0.3, 1.0, 4.0])
    assert np.allclose(fisk.residual_density(r, alpha, beta) * 2 * math.pi * r,
                       fisk.fisk_pdf(r, alpha, beta), rtol=1e-13)


def test_inlier_energy_beta2_closed_form():
    a, p0 = 0.5, 1e-3
    r = np.array([0.0, 0.2, 1.0, 5.0, 50.0])
    # beta = 2: p1(r) = 1 / (pi a^2 (1 + r^2/a^2)^2)
    want = np.log1p(p0 * math.pi * a * a * (1 + (r / a) ** 2) ** 2)
    assert np.allclose(fisk.inlier_energy(r, a, 2.0, p0), want, rtol=1e-14, atol=0)
    post = fisk.inlier_posterior(r, a, 2.0, p0)
    assert np.allclose(-np.log(post), want, rtol=1e-12)
    assert np.all(np.diff(want) > 0)           # monotone in the residual


# ---------------------------------------------------------------- geometry
def test_se3_exp_log_roundtrip_and_compose():
    rng = np.random.default_rng(3)
    for _ in range(50):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        xi = np.concatenate([ax * rng.choice([1e-9, 1e-3, 0.5, 3.0]), rng.normal(size=3)])
        T = geometry.se3_exp(xi)
        assert abs(np.linalg.det(T[:, :3]) - 1) < 1e-12
        assert np.allclose(geometry.se3_log(T), xi, atol=1e-10)
        I = geometry.compose(T, geometry.inverse(T))
        assert np.allclose(I, geometry.IDENTITY, atol=1e-12)
    # rotation about z by 90 deg moves x to y
    R = geometry.so3_exp(np.array([0, 0, math.pi / 2]))
    assert np.allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_se3_exp_equals_the_matrix_exponential():
    """exp of the 4x4 twist matrix [[w^, v], [0, 0]] (a library routine, not
    the closed form the oracle uses), from the series branch to large angles."""
    from scipy.linalg import expm
    rng = np.random.default_rng(5)
    for mag in [1e-7, 1e-4, 0.3, 1.5, 3.0]:
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        w, v = ax * mag, rng.normal(size=3)
        Xi = np.zeros((4, 4))
        Xi[:3, :3] = [[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]]
        Xi[:3, 3] = v
        assert np.allclose(geometry.se3_exp(np.concatenate([w, v])), expm(Xi)[:3], atol=1e-12)


def test_bilinear_reproduces_affine_fields_and_grid_values():
    H, W = 7, 9
    v, u = np.mgrid[0:H, 0:W]
    F = np.stack([0.3 * u - 0.2 * v + 1.0, 0.1 * u + 0.5 * v - 2.0], -1).astype(np.float32)
    xs = np.array([0.0, 3.25, 8.0, 7.999, 4.5])
    ys = np.array([0.0, 2.5, 6.0, 0.001, 6.0])
    got = geometry.bilinear(F, xs, ys)
    want = np.stack([0.3 * xs - 0.2 * ys + 1.0, 0.1 * xs + 0.5 * ys - 2.0], -1)
    assert np.allclose(got, want, atol=1e-6)
    assert np.array_equal(geometry.bilinear(F, np.array([2.0]), np.array([5.0]))[0], F[5, 2])
    assert geometry.inside(np.array([8.0, 8.0001]), np.array([6.0, 0.0]), W, H).tolist() == [True, False]


# ---------------------------------------------------------------- forward-backward
def _brute_posterior(e1, e0, gamma):
    L = len(e1)
    num = np.zeros(L)
    tot = 0.0
    for states in itertools.product([0, 1], repeat=L):
        p = 0.5
        for m, s in enumerate(states):
            if m > 0:
                p *= gamma if s == states[m - 1] else 1 - gamma
            p *= e1[m] if s else e0[m]
        tot += p
        num += p * np.array(states)
    return num / tot


@pytest.mark.parametrize("L", [1, 2, 5, 12])
def test_forward_backward_matches_enumeration(L):
    rng = np.random.default_rng(L)
    for gamma in [0.95, 0.7, 0.5]:
        e1 = rng.uniform(0, 2, size=L) * rng.choice([1, 1e-3], size=L)
        e0 = np.full(L, 1e-3) * rng.uniform(0.5, 2, size=L)
        got = hmm.forward_backward(e1[:, None], e0[:, None], gamma)[:, 0]
        assert np.allclose(got, _brute_posterior(e1, e0, gamma), atol=1e-12, rtol=0)


def test_forward_backward_invariants():
    rng = np.random.default_rng(0)
    e1 = rng.uniform(0, 1, size=(40, 3))
    e0 = rng.uniform(0, 1, size=(40, 3))
    post = hmm.forward_backward(e1, e0, 0.9)
    # a symmetric chain with a uniform start has the same posteriors walked backwards
    assert np.allclose(hmm.forward_backward(e1[::-1], e0[::-1], 0.9)[::-1], post, atol=1e-13)
    # gamma = 1/2: neighbours carry no information
    assert np.allclose(hmm.forward_backward(e1, e0, 0.5), e1 / (e1 + e0), atol=1e-13)
    # gamma = 1: one shared state per chain
    g1 = hmm.forward_backward(e1, e0, 1.0)
    l1 = np.exp(np.log(e1).sum(0))
    l0 = np.exp(np.log(e0).sum(0))
    assert np.allclose(g1, (l1 / (l1 + l0))[None, :], atol=1e-12)


# ---------------------------------------------------------------- P3P
def test_p3p_exact_correspondences():
    rng = np.random.default_rng(11)
    errs = []
    for _ in range(300):
        R = geometry.so3_exp(rng.normal(size=3) * 0.5)
        X = rng.normal(size=(3, 3))
        tau = rng.normal(size=3)
        tau[2] += 5 - (X @ R.T + tau)[:, 2].min()
        Xc = X @ R.T + tau
        sols = p3p.solve(Xc, X)
        assert 1 <= len(sols) <= 4
        G = np.concatenate([R, tau[:, None]], 1)
        errs.append(min(np.abs(s - G).max() for s in sols))
        for s in sols:      # every root reprojects the three points exactly
            Y = X @ s[:, :3].T + s[:, 3]
            assert np.allclose(Y / np.linalg.norm(Y, axis=1, keepdims=True),
                               Xc / np.linalg.norm(Xc, axis=1, keepdims=True), atol=1e-6)
    errs = np.array(errs)
    assert np.percentile(errs, 90) < 1e-9
    assert errs.max() < 1e-5


# ---------------------------------------------------------------- 8-point
def test_eight_point_noise_free_two_planes_is_exact():
    win = synth.make_window("planes160", 0, noisy=False)
    P = model.problem_from_window(win)
    G1, counts = eightpoint.bootstrap_pose(P, 0.5)
    Gt = win.G[1].copy()
    Gt[:, 3] /= np.linalg.norm(Gt[:, 3])
    # limited by the float32 storage of the flow (ulp ~ 1e-6 px)
    assert np.abs(G1[:, :3] - Gt[:, :3]).max() < 1e-9
    assert np.abs(G1[:, 3] - Gt[:, 3]).max() < 1e-7
    assert max(counts) == P.W * P.H
    # E = [t]x R up to scale and sign
    E, _, _ = eightpoint.essential(P, 0.5)
    Et = geometry.hat(Gt[:, 3]) @ Gt[:, :3]
    Et /= np.linalg.norm(Et)
    assert min(np.abs(E - Et).max(), np.abs(E + Et).max()) < 1e-7


def test_essential_decomposition_and_cheirality():
    """Every candidate of E = [t]x R is a proper rotation and one of them is
    (R, t/|t|) up to the sign of t, whatever signs the SVD picks; on the
    noise-free two-plane flow only the true motion puts the points in front
    of both cameras (the other three fail for at least half of them)."""
    rng = np.random.default_rng(9)
    for _ in range(60):
        R = geometry.so3_exp(rng.normal(size=3) * 0.3)
        t = rng.normal(size=3)
        t /= np.linalg.norm(t)
        E = geometry.hat(t) @ R * rng.choice([-1.0, 1.0])
        cands = eightpoint.candidates(E)
        assert all(abs(np.linalg.det(Rc) - 1.0) < 1e-12 for Rc, _ in cands)
        assert min(np.abs(Rc - R).max() + min(np.abs(tc - t).max(), np.abs(tc + t).max())
                   for Rc, tc in cands) < 1e-9
    win = synth.make_window("planes160", 0, noisy=False)
    P = model.problem_from_window(win)
    G1, counts = eightpoint.bootstrap_pose(P, 0.5)
    c = sorted(counts)
    assert c[-1] == P.W * P.H and c[-2] <= 0.5 * P.W * P.H


def test_eight_point_single_plane_is_degenerate():
    win = synth.make_window("planes160", 0, noisy=False)
    # replace the scene by one fronto-parallel plane at 4 m: a homography, E is not unique
    P = model.problem_from_window(win)
    fx, fy, cx, cy = P.K
    r = P.rays
    X = r * 4.0
    G1 = win.G[1]
    Y = X @ G1[:, :3].T + G1[:, 3]
    u, v = np.meshgrid(np.arange(P.W), np.arange(P.H))
    flow = np.stack([fx * Y[..., 0] / Y[..., 2] + cx - u, fy * Y[..., 1] / Y[..., 2] + cy - v], -1)
    P.flow = np.concatenate([flow[None].astype(np.float32), P.flow[1:]])
    M, _, _ = eightpoint.normal_matrix(P)
    w = np.linalg.eigvalsh(M)
    # a planar scene leaves (at least) a 3-dimensional null space (H&Z Sec. 11.9)
    assert w[2] < 1e-6 * w[-1]


# ---------------------------------------------------------------- depth step
def _truth_state(win, P, q=1.0):
    s = win.params["scale"]
    G = win.G.copy()
    G[:, :, 3] /= s
    rho = (s / win.depth0).astype(np.float32)
    return model.State(rho=rho, q=np.full((P.N, P.H, P.W), q, np.float32),
                       qhat=np.zeros((P.H, P.W), np.float32), G=G)


def _params(win, **kw):
    pr = win.params
    d = dict(fisk_alpha0=pr["fisk_alpha0"], rho_min=pr["rho_min"], rho_max=pr["rho_max"],
             n_hyp=pr["n_hyp"])
    d.update(kw)
    return model.Params(**d)


def test_energy_minimum_at_true_depth_noise_free():
    win = synth.make_window("planes160", 0, noisy=False)
    P = model.problem_from_window(win)
    S = _truth_state(win, P)
    p = _params(win)
    iu, iv = model.pixel_grid(P)
    E_true = model.energy(P, S, iu, iv, S.rho, p)
    # the flow term at the true depth is l(~0) per observed flow
    l0 = fisk.inlier_energy(0.0, p.fisk_alpha0, 2.0, p.outlier_density)
    ell, _, ok = model.flow_terms(P, S.G, iu, iv, S.rho, p)
    assert np.all(ok[0])
    assert np.allclose(ell[0], l0, atol=1e-6)
    # every perturbed candidate costs more where all flows are observed
    allobs = ok.all(0)
    for f in [0.9, 0.97, 1.03, 1.1]:
        rf = S.rho * np.float32(f)
        E = model.energy(P, S, iu, iv, rf, p)
        sel = allobs & model.flow_terms(P, S.G, iu, iv, rf, p)[2].all(0)
        assert sel.mean() > 0.8
        assert np.all(E[sel] > E_true[sel])
    # K = 1: the step reduces to evaluating the current depth
    p1 = _params(win, n_hyp=1)
    c = depth.hypotheses(P, S.rho, 0, p1)
    rho_star, E_star, k = depth.argmin_candidates(P, S, c, p1)
    assert np.array_equal(rho_star, np.clip(S.rho, p1.f32("rho_min"), p1.f32("rho_max")))
    assert np.allclose(E_star, model.energy(P, S, iu, iv, rho_star, p1), rtol=0, atol=0)


def test_behind_camera_and_unobserved_terms():
    """The three cases of a flow term: observed and in front (Fisk energy),
    observed but behind camera t (the constant L_BEHIND, rigid emission 0),
    not observed because x_{t-1} left the image (energy 0, both emissions
    P0)."""
    win = synth.make_window("planes160", 0, noisy=False)
    P = model.problem_from_window(win)
    p = _params(win)
    G = np.stack([geometry.IDENTITY] * (P.N + 1))
    iu, iv = model.pixel_grid(P)
    rho = np.full((P.H, P.W), 0.5)
    # camera 1 moves 10 units forward: z = 1 + 0.5 * (-10) < 0 for every pixel
    G[1] = geometry.IDENTITY.copy()
    G[1][2, 3] = -10.0
    ell, e1, ok = model.flow_terms(P, G, iu, iv, rho, p)
    assert not ok[0].any()
    assert np.all(ell[0] == fisk.L_BEHIND) and np.all(e1[0] == 0.0)
    # frame 1 behind: flow 2 has no observation at x_1
    assert np.all(ell[1] == 0.0) and np.all(e1[1] == p.outlier_density)
    # camera 1 shifted sideways by 1000 px: x_1 leaves the image, flow 2 unobserved
    G[1] = geometry.IDENTITY.copy()
    G[1][0, 3] = 1000.0 / (P.K[0] * 0.5)
    ell, e1, ok = model.flow_terms(P, G, iu, iv, rho, p)
    assert np.all(ok[0]) and np.all(ell[0] > 0)
    assert np.all(ell[1] == 0.0) and np.all(e1[1] == p.outlier_density)


def test_argmin_finds_true_depth_among_candidates():
    win = synth.make_window("planes160", 1, noisy=False)
    P = model.problem_from_window(win)
    S = _truth_state(win, P)
    p = _params(win, n_hyp=16)
    c = depth.hypotheses(P, S.rho, 0, p)
    assert np.array_equal(c[0], S.rho)               # slot 0 keeps the current value
    rho_star, _, k = depth.argmin_candidates(P, S, c, p)
    iu, iv = model.pixel_grid(P)
    _, _, ok = model.flow_terms(P, S.G, iu, iv, S.rho, p)
    sel = ok.all(0)
    assert np.mean(rho_star[sel] == S.rho[sel]) > 0.999


def test_hypotheses_distribution_and_sharing():
    win = synth.make_window("planes160", 0, noisy=False)
    P = model.problem_from_window(win)
    p = _params(win, n_hyp=9, rho_min=0.1, rho_max=0.5)
    rho = np.full((P.H, P.W), 0.3, np.float32)
    c = depth.hypotheses(P, rho, 2, p)
    assert c.dtype == np.float32 and c.shape == (9, P.H, P.W)
    assert np.all((c >= np.float32(0.1)) & (c <= np.float32(0.5)))
    # slots 1..4 uniform in [0.1, 0.5] (KS distance of the pooled draws)
    from scipy import stats
    uni = c[1:5].ravel().astype(np.float64)
    assert stats.kstest((uni - 0.1) / 0.4, "uniform").statistic < 0.01
    # slots 5..8 perturb the current value by at most s_2 = 1/8
    loc = c[5:].astype(np.float64)
    assert np.all(np.abs(loc / 0.3 - 1) <= 0.125 + 1e-6)
    assert stats.kstest((loc.ravel() / 0.3 - 1) / 0.125 * 0.5 + 0.5, "uniform").statistic < 0.01
    # share = 8: a row segment of 8 aligned pixels draws the same numbers
    p8 = _params(win, n_hyp=9, rho_min=0.1, rho_max=0.5, sample_share=8)
    c8 = depth.hypotheses(P, rho, 2, p8)
    seg = c8[:, :, :8]
    assert np.all(seg == seg[:, :, :1])
    assert not np.all(c8[:, :, 8] == c8[:, :, 0])


def _naive_patchmatch(P, S, cands, direction, p):
    """Sequential propagation written the direct way: walking each chain, pixel
    m takes the argmin over its own K candidates and, last, the value just
    chosen at its predecessor (strict improvement needed)."""
    iu, iv = depth.chain_coords(P, direction)
    out = np.zeros((P.H, P.W), np.float32)
    for c in range(iu.shape[1]):
        prev = None
        for m in range(iu.shape[0]):
            u, v = iu[m, c], iv[m, c]
            best, bestE = None, np.inf
            for k in range(cands.shape[0]):
                E = model.energy(P, S, np.array([u]), np.array([v]), np.array([cands[k, v, u]]), p)[0]
                if E < bestE:
                    best, bestE = cands[k, v, u], E
            if prev is not None:
                E = model.energy(P, S, np.array([u]), np.array([v]), np.array([prev]), p)[0]
                if E < bestE:
                    best, bestE = prev, E
            out[v, u] = best
            prev = best
    return out


@pytest.mark.parametrize("direction", [0, 1, 2, 3])
def test_split_propagation_equals_naive_sequential(direction):
    win = synth.make_window("planes160", 2, noisy=True)
    P = model.problem_from_window(win)
    # crop to a small window so the naive walk stays cheap
    P = model.Problem(12, 9, P.N, P.K, np.ascontiguousarray(P.flow[:, :9, :12]))
    S = model.State(rho=np.full((9, 12), 0.05, np.float32), q=np.ones((P.N, 9, 12), np.float32),
                    qhat=np.zeros((9, 12), np.float32), G=_truth_state(win, model.problem_from_window(win)).G)
    p = _params(win, n_hyp=6)
    c = depth.hypotheses(P, S.rho, 0, p)
    rho_star, E_star, _ = depth.argmin_candidates(P, S, c, p)
    split, _ = depth.propagate(P, S, rho_star, E_star, direction, p)
    assert np.array_equal(split, _naive_patchmatch(P, S, c, direction, p))


def test_hierarchical_with_window_covering_chain_and_scale1_reduces():
    """scale 1 and a window as long as the chain: the coarse pass already is the
    full sequential propagation and the later passes cannot change it."""
    win = synth.make_window("planes160", 3, noisy=True)
    P0 = model.problem_from_window(win)
    P = model.Problem(16, 10, P0.N, P0.K, np.ascontiguousarray(P0.flow[:, :10, :16]))
    S = model.State(rho=np.full((10, 16), 0.05, np.float32), q=np.ones((P.N, 10, 16), np.float32),
                    qhat=np.zeros((10, 16), np.float32), G=_truth_state(win, P0).G)
    p = _params(win, n_hyp=6, hierarchical=1, hier_scale=1, hier_window=1000)
    c = depth.hypotheses(P, S.rho, 0, p)
    rho_star, E_star, _ = depth.argmin_candidates(P, S, c, p)
    for d in range(4):
        full, _ = depth.propagate(P, S, rho_star, E_star, d, p)
        hier, _ = depth.hierarchical(P, S, rho_star, E_star, d, p)
        assert np.array_equal(full, hier)


@pytest.mark.parametrize("direction", [0, 1])
def test_propagation_never_raises_a_pixels_energy(direction):
    """Every pass takes a value only when it lowers the pixel's energy, so
    after the full and the hierarchical propagation (coarse cells of 4,
    windows of 5) no pixel's energy is above its own candidate's."""
    win = synth.make_window("planes160", 5, noisy=True)
    P0 = model.problem_from_window(win)
    P = model.Problem(24, 16, P0.N, P0.K, np.ascontiguousarray(P0.flow[:, :16, :24]))
    S = model.State(rho=np.full((16, 24), 0.05, np.float32), q=np.ones((P.N, 16, 24), np.float32),
                    qhat=np.zeros((16, 24), np.float32), G=_truth_state(win, P0).G)
    p = _params(win, n_hyp=4, hierarchical=1, hier_scale=4, hier_window=5)
    c = depth.hypotheses(P, S.rho, 0, p)
    rho_star, E_star, _ = depth.argmin_candidates(P, S, c, p)
    iu, iv = model.pixel_grid(P)
    for fn in (depth.propagate, depth.hierarchical):
        new, E_new = fn(P, S, rho_star, E_star, direction, p)
        E = model.energy(P, S, iu, iv, new, p)
        assert np.array_equal(E, E_new)
        assert np.all(E <= E_star)
        assert np.any(E < E_star)        # the pass did propagate something


def test_initial_inverse_depth_is_uniform_in_range_or_the_prior():
    from scipy import stats
    win = synth.make_window("planes160", 0, noisy=False)
    P = model.problem_from_window(win)
    p = _params(win, rho_min=0.1, rho_max=0.5)
    rho = em.initial_rho(P, p)
    assert rho.dtype == np.float32
    assert np.all((rho >= np.float32(0.1)) & (rho <= np.float32(0.5)))
    assert stats.kstest((rho.ravel().astype(np.float64) - 0.1) / 0.4, "uniform").statistic < 0.02
    # with a prior: its inverse depth (clamped) where valid, the draw at holes
    win = synth.make_window("boxes640_stereo", 1, noisy=True, size=(128, 96), N=2)
    P = model.problem_from_window(win)
    p = _params(win)
    rho = em.initial_rho(P, p)
    pr = P.prior_rho()
    ok = np.isfinite(pr)
    assert 0 < (~ok).sum() and np.array_equal(rho[ok], np.clip(pr[ok], p.f32("rho_min"), p.f32("rho_max")))


# ---------------------------------------------------------------- E-step
def test_estep_moving_blobs_get_low_rigidness():
    win = synth.make_window("boxes640_stereo", 7, noisy=True, size=(160, 120), N=3)
    P = model.problem_from_window(win, prior="none")
    S = model.State(rho=(1.0 / win.depth0).astype(np.float32), q=np.ones((P.N, P.H, P.W), np.float32),
                    qhat=np.zeros((P.H, P.W), np.float32), G=win.G.copy())
    p = _params(win, fisk_alpha0=0.5)
    q, _, C = hmm.rigidness_estep(P, S, S.rho, 0, p)
    # blobs are drawn on frame t-1's grid; for t = 1 that is the reference grid
    blob = win.moving[0]
    assert blob.sum() > 100
    assert np.mean(q[0][blob] < 0.5) >= 0.9
    assert np.mean(q[0][~blob] > 0.5) >= 0.9
    assert np.allclose(C, q.astype(np.float64).mean(0), atol=1e-6)


# ---------------------------------------------------------------- priors
def test_stereo_prior_optimum_is_the_prior():
    win = synth.make_window("boxes640_stereo", 1, noisy=False, size=(128, 96), N=2)
    P = model.problem_from_window(win)
    assert P.prior_kind == "stereo"
    S = model.State(rho=(1.0 / win.depth0).astype(np.float32), q=np.zeros((P.N, P.H, P.W), np.float32),
                    qhat=np.ones((P.H, P.W), np.float32), G=win.G.copy())
    p = _params(win, n_hyp=8)
    iu, iv = model.pixel_grid(P)
    rhat = P.prior_rho()
    E0 = model.energy(P, S, iu, iv, rhat, p)
    for f in [0.98, 1.02]:
        assert np.all(model.energy(P, S, iu, iv, rhat * np.float32(f), p) > E0)
    # the prior's value is d / (fx b) and its energy is l(0)
    assert np.allclose(rhat, win.stereo_disp / np.float32(P.K[0] * 0.25), rtol=1e-7)
    l0 = fisk.inlier_energy(0.0, p.fisk_alpha0, 2.0, p.outlier_density)
    assert np.allclose(E0, l0, rtol=1e-5)


def test_prior_rigidness_at_a_perfect_prior():
    """q_hat is the isolated posterior p1 / (p1 + P0) at the new depth: at the
    prior's own value (residual 0) and beta = 2, p1(0) = 1 / (pi alpha^2)."""
    win = synth.make_window("boxes640_stereo", 1, noisy=False, size=(128, 96), N=2)
    P = model.problem_from_window(win)
    S = model.State(rho=(1.0 / win.depth0).astype(np.float32), q=np.ones((P.N, P.H, P.W), np.float32),
                    qhat=np.ones((P.H, P.W), np.float32), G=win.G.copy())
    p = _params(win)
    rhat = P.prior_rho()
    _, qhat, C = hmm.rigidness_estep(P, S, rhat.astype(np.float64), 0, p)
    a = p.fisk_alpha0
    want = 1.0 / (1.0 + p.outlier_density * math.pi * a * a)
    valid = np.isfinite(rhat)
    assert valid.mean() > 0.5
    assert np.allclose(qhat[valid], want, rtol=1e-6)
    assert np.all(qhat[~valid] == 0.0)


def test_rgbd_prior_closed_forms():
    win = synth.make_window("rgbd_batch", 2, noisy=False, size=(64, 48), N=3)
    P = model.problem_from_window(win)
    assert P.prior_kind == "rgbd"
    p = _params(win, prior_c_sigma=0.01, prior_w_uniform=2.0)
    iu, iv = model.pixel_grid(P)
    rhat = P.prior_rho().astype(np.float64)
    ell, e1, e0, valid = model.prior_terms(P, iu, iv, rhat, p)
    assert valid.all()
    k = math.sqrt(2 * math.pi) * 0.01 / 2.0
    assert np.allclose(ell, math.log1p(k), rtol=1e-12)
    # Eq. 3 densities: Gaussian with sigma = c rho_hat, uniform 1 / (w rho_hat)
    assert np.allclose(e1, 1 / (math.sqrt(2 * math.pi) * 0.01 * rhat), rtol=1e-12)
    assert np.allclose(e0, 1 / (2.0 * rhat), rtol=1e-12)
    # one sigma away: Gaussian density falls by exp(-1/2)
    ell1, e11, _, _ = model.prior_terms(P, iu, iv, rhat * 1.01, p)
    assert np.allclose(e11 / e1, math.exp(-0.5), rtol=1e-9)
    assert np.allclose(ell1, np.log1p(k * math.exp(0.5)), rtol=1e-9)


# ---------------------------------------------------------------- pose step
def test_meanshift_cases():
    p = model.Params()
    T = geometry.se3_exp(np.array([0.1, -0.2, 0.05, 1.0, 0.2, -0.3]))
    x, n = pose.meanshift([T] * 5, T, p)
    assert np.abs(x - T).max() < 1e-14 and n == 1
    # symmetric pair around a centre: the mode of two close Gaussians is the midpoint
    d = np.array([0.002, 0, 0, 0, 0, 0])
    A = geometry.compose(T, geometry.se3_exp(d))
    B = geometry.compose(T, geometry.se3_exp(-d))
    x, _ = pose.meanshift([A, B], A, p)
    assert np.abs(geometry.se3_log(geometry.compose(geometry.inverse(T), x))).max() < 1e-10
    # a far outlier does not move the mode of a tight cluster
    far = geometry.compose(T, geometry.se3_exp(np.array([0.5, 0, 0, 0, 0, 0])))
    x, _ = pose.meanshift([T, T, T, far], far, p)
    assert np.abs(geometry.se3_log(geometry.compose(geometry.inverse(far), x))).max() < 1e-12


def test_meanshift_runs_to_the_mode_where_it_converges_slowly():
    """Two samples at +-a on one rotation axis around T with a just below the
    kernel's sigma: the density has one mode, the midpoint T, and the
    iteration approaches it at the linear rate (a / sigma)^2 = 0.98 -- after
    100 steps still 1e-3 rad away.  The pose is the mode, so the oracle must
    reach T to float64 precision."""
    p = model.Params()
    T = geometry.se3_exp(np.array([0.05, 0.1, -0.2, 0.5, -1.0, 2.0]))
    a = 0.99 * p.pose_sigma_rot
    A = geometry.compose(T, geometry.se3_exp(np.array([a, 0, 0, 0, 0, 0])))
    B = geometry.compose(T, geometry.se3_exp(np.array([-a, 0, 0, 0, 0, 0])))
    x, n = pose.meanshift([A, B], A, p)
    d = geometry.se3_log(geometry.compose(geometry.inverse(T), x))
    assert np.abs(d).max() < 1e-10
    assert n > 500           # a step below 1e-12 takes several hundred


def test_meanshift_mode_on_one_rotation_axis_solves_the_scalar_equation():
    """Samples T, T and T exp(a e_x) (a rotation about one body axis): every
    iterate stays on that axis, the tangent coordinates are (a_g - m) e_x
    exactly, and the mode is the root of sum_g w_g (a_g - m) = 0 with
    w_g = exp(-(a_g - m)^2 / (2 sigma_rot^2)) nearest the start m = 0."""
    from scipy import optimize
    p = model.Params()
    T = geometry.se3_exp(np.array([0.2, -0.1, 0.3, 2.0, -1.5, 1.0]))   # |tau| ~ 2.7
    a = 1.5 * p.pose_sigma_rot
    samples = [T, T, geometry.compose(T, geometry.se3_exp(np.array([a, 0, 0, 0, 0, 0])))]
    x, _ = pose.meanshift(samples, T, p)
    d = geometry.se3_log(geometry.compose(geometry.inverse(T), x))
    assert np.abs(d[1:]).max() < 1e-12
    ag = np.array([0.0, 0.0, a])
    f = lambda m: np.sum(np.exp(-0.5 * ((ag - m) / p.pose_sigma_rot) ** 2) * (ag - m))
    m = optimize.brentq(f, 0.0, a / 2, xtol=1e-15)
    assert abs(d[0] - m) < 1e-10 and 0 < m < a / 3


def test_pose_step_recovers_first_pose_from_true_depth():
    win = synth.make_window("planes160", 4, noisy=False)
    P = model.problem_from_window(win)
    S = _truth_state(win, P)
    G_true = S.G.copy()
    S.G[1] = geometry.IDENTITY
    p = _params(win)
    out = pose.pose_mstep_frame(P, S, 1, 0, p)
    assert out["n_rigid"] == P.W * P.H and len(out["samples"]) == p.n_pose_samples
    d = geometry.se3_log(geometry.compose(geometry.inverse(G_true[1]), S.G[1]))
    # limited only by the float32 storage of depth and flow (3-point samples
    # amplify their ~1e-7 relative rounding)
    assert np.abs(d[:3]).max() < 1e-6
    assert np.abs(d[3:]).max() < 1e-5
    # rigid-set ordering and the sample draws are deterministic
    rs = pose.rigid_set(P, S, 1, p)
    assert np.all(np.diff(rs["j"]) > 0)


def test_sample_triplets_are_distinct_indices():
    """A P3P sample is three different rigid pixels: for a set of 3 every
    drawn triplet is a permutation of {0, 1, 2} (or the sample is void after
    the retries); larger sets give distinct in-range indices."""
    p = model.Params()
    for n in (3, 4, 50):
        void = 0
        for g in range(200):
            tri = pose.draw_triplet(n, g, 1, 0, p)
            if tri is None:
                void += 1
                continue
            assert len(set(tri)) == 3 and all(0 <= i < n for i in tri)
        # a draw is distinct with probability n (n-1) (n-2) / n^3; 8 tries
        p_void = (1 - n * (n - 1) * (n - 2) / n ** 3) ** 8
        assert abs(void - 200 * p_void) <= 4 * math.sqrt(200 * p_void * (1 - p_void)) + 1
    assert pose.draw_triplet(3, 7, 2, 1, p) == pose.draw_triplet(3, 7, 2, 1, p)


def test_pose_step_skips_degenerate_frame():
    win = synth.make_window("planes160", 4, noisy=False)
    P = model.problem_from_window(win)
    S = _truth_state(win, P, q=0.0)
    G0 = S.G.copy()
    out = pose.pose_mstep_frame(P, S, 2, 0, _params(win))
    assert out["degenerate"] and out["n_rigid"] == 0
    assert np.array_equal(S.G, G0)


# ---------------------------------------------------------------- whole EM
def test_whole_em_noise_free_recovers_scene_up_to_scale():
    win = synth.make_window("planes160", 0, noisy=False)
    P = model.problem_from_window(win)
    p = _params(win)
    S, _ = em.run(P, p, 6)
    Gt = win.G.copy()
    Gt[:, :, 3] /= win.params["scale"]
    # monocular scale: align with s* = |tau_1 true| / |tau_1 estimated|
    s_star = np.linalg.norm(Gt[1][:, 3]) / np.linalg.norm(S.G[1][:, 3])
    rho_true = win.params["scale"] / win.depth0
    rel = np.abs(S.rho / s_star - rho_true) / rho_true
    assert np.median(rel) < 2e-3
    for t in range(1, P.N + 1):
        R_err = geometry.so3_log(S.G[t][:, :3].T @ Gt[t][:, :3])
        assert np.linalg.norm(R_err) < 5e-4
        assert np.linalg.norm(S.G[t][:, 3] * s_star - Gt[t][:, 3]) < 2e-2 * np.linalg.norm(Gt[t][:, 3])

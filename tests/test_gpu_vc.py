"""Visibility-coverage score on the GPU (vd_vc_scores, vd_vc_pose) against
the oracle (oracle/vc.py).  Every count is an integer decided by the same
float32 operations on both sides, so counts, ratios and VC must be equal."""
import numpy as np
import pytest

from gpu_common import noisy_state, params_for, push_state, window
from oracle import model as omodel
from oracle import vc as ovc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2104_06800_gb300 import build, voldor
    build.build()
    voldor.load()
    return voldor


def _check(res, rho, K, poses, W, H):
    assert res["n_pixels"] == W * H and res["n_frames"] == len(poses)
    for k, T in enumerate(poses):
        nd, nv, nc = ovc.counts(rho, K, T, W, H)
        got = (res["n_depth"], res["n_visible"][k], res["n_covered"][k])
        assert got == (nd, nv, nc), (k, got, (nd, nv, nc))
        v, c, s = ovc.scores(rho, K, T, W, H)
        assert (res["visibility"][k], res["coverage"][k], res["vc"][k]) == (v, c, s), k


def _holes(rho, rng):
    rho = rho.copy()
    m = rng.uniform(size=rho.shape)
    rho[m < 0.03] = np.nan
    rho[(m >= 0.03) & (m < 0.04)] = -0.5
    rho[(m >= 0.04) & (m < 0.05)] = 0.0
    rho[(m >= 0.05) & (m < 0.06)] = np.inf
    return rho


@pytest.mark.parametrize("name,seed,size", [("driving1216", 2001, (608, 184)),
                                            ("boxes640_stereo", 7, (333, 141)),
                                            ("planes160", 0, None)])
def test_window_scores_match_oracle(V, name, seed, size):
    w = window(name, seed, **({"size": size} if size else {}))
    rng = np.random.default_rng(seed)
    P = omodel.problem_from_window(w)
    S = noisy_state(w, P, rng, rel=0.05)
    S.rho = _holes(S.rho, rng)
    ctx = V.vd_create(w.W, w.H, w.N, w.intrinsics, V.vd_params_default(**params_for(w)))
    try:
        push_state(V, ctx, S)
        res = V.vd_vc_scores(ctx)
        _check(res, S.rho, w.intrinsics, [S.G[t] for t in range(1, w.N + 1)], w.W, w.H)
        assert 0 < res["n_depth"] < w.W * w.H
        assert V.vd_vc_stride(res["vc"], 0.8) == ovc.stride(res["vc"], 0.8)
    finally:
        V.vd_destroy(ctx)


def test_arbitrary_poses_match_oracle(V):
    """Keyframe-test poses: identity, small and large motions, rotations
    beyond the field of view, the camera past the scene."""
    w = window("driving1216", 2002, size=(304, 92))
    rng = np.random.default_rng(5)
    P = omodel.problem_from_window(w)
    S = noisy_state(w, P, rng, rel=0.02)
    from oracle import geometry as ogeo
    poses = [np.hstack([np.eye(3), np.zeros((3, 1))])]
    for scale_r, scale_t in [(0.01, 0.2), (0.1, 1.0), (0.5, 0.5), (1.5, 3.0), (0.0, 50.0)]:
        for _ in range(3):
            xi = np.concatenate([rng.normal(size=3) * scale_r, rng.normal(size=3) * scale_t])
            poses.append(ogeo.se3_exp(xi))
    poses.append(np.hstack([np.eye(3), [[0.0], [0.0], [-1e3]]]))   # everything behind
    ctx = V.vd_create(w.W, w.H, w.N, w.intrinsics, V.vd_params_default(**params_for(w)))
    try:
        push_state(V, ctx, S)
        seen_partial = False
        for T in poses:
            res = V.vd_vc_pose(ctx, T)
            _check(res, S.rho, w.intrinsics, [T], w.W, w.H)
            seen_partial |= 0 < res["n_visible"][0] < res["n_depth"]
        assert seen_partial
        assert V.vd_vc_pose(ctx, poses[-1])["vc"] == [0.0]
        # identity: all but border pixels that float32 rounding pushes a hair out
        assert V.vd_vc_pose(ctx, poses[0])["visibility"][0] > 0.97
        with pytest.raises(V.VoldorError):
            V.vd_vc_pose(ctx, np.full((3, 4), np.nan))
    finally:
        V.vd_destroy(ctx)


def test_full_size_after_the_em(V):
    """1216 x 368, N = 6 after the bootstrap and 8 EM iterations: the
    counts of the GPU's own depth and poses, the stride they imply."""
    w = window("driving1216", 2003)
    ctx = V.vd_create(w.W, w.H, w.N, w.intrinsics, V.vd_params_default(**params_for(w)))
    try:
        for t in range(1, w.N + 1):
            V.vd_push_flow(ctx, t, w.flow[t - 1])
        V.vd_bootstrap(ctx)
        V.vd_run_em(ctx, 8)
        rho = np.empty((w.H, w.W), np.float32)
        V.vd_get_inv_depth(ctx, rho)
        G = V.vd_get_poses(ctx, w.N)
        res = V.vd_vc_scores(ctx)
        _check(res, rho, w.intrinsics, [G[t] for t in range(1, w.N + 1)], w.W, w.H)
        vc = res["vc"]
        assert all(a >= b - 0.05 for a, b in zip(vc, vc[1:]))   # forward motion: VC falls
        for tau in (0.5, 0.7, 0.9):
            assert V.vd_vc_stride(vc, tau) == ovc.stride(vc, tau)
    finally:
        V.vd_destroy(ctx)


def test_tiny_window_one_flow(V):
    """A 3 x 2 window with one flow: a single partial warp."""
    rng = np.random.default_rng(11)
    K = (2.0, 2.0, 1.0, 0.5)
    ctx = V.vd_create(3, 2, 1, K, V.vd_params_default())
    try:
        rho = rng.uniform(0.2, 1.0, (2, 3)).astype(np.float32)
        rho[0, 1] = np.nan
        from oracle import geometry as ogeo
        G = np.stack([np.hstack([np.eye(3), np.zeros((3, 1))]),
                      ogeo.se3_exp(np.array([0.0, 0.02, 0.0, 0.3, 0.0, 0.1]))])
        V.vd_set_poses(ctx, G.reshape(-1, 12))
        V.vd_set_state(ctx, rho)
        res = V.vd_vc_scores(ctx)
        _check(res, rho, K, [G[1]], 3, 2)
    finally:
        V.vd_destroy(ctx)

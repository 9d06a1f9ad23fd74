"""Pose covariance on the GPU (vd_pose_covariance) against the oracle
(oracle/posecov.py), on the samples and modes of real pose M-steps read
back from the GPU (vd_get_frame_samples, vd_get_poses).  Both sides are
float64 with different summation orders: the inlier sets, counts and
rounds must agree, the mean and covariance to rounding."""
import numpy as np
import pytest

from gpu_common import make_ctx, params_for, window
from oracle import geometry, posecov

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2104_06800_gb300 import build, voldor
    build.build()
    voldor.load()
    return voldor


def _compare(V, ctx, w, params, eps):
    """GPU fit of every frame against the oracle's fit of the same samples."""
    res = V.vd_pose_covariance(ctx, w.N, eps)
    G = V.vd_get_poses(ctx, w.N)
    S = params.n_pose_samples
    for t in range(1, w.N + 1):
        poses, energies = V.vd_get_frame_samples(ctx, t, S)
        samples = [poses[g] for g in range(S) if np.isfinite(energies[g])]
        mu, Sig, n_in, rounds, deg = posecov.fit(samples, G[t], eps)
        r = res[t - 1]
        assert r["n_samples"] == len(samples), t
        assert (r["n_inliers"], r["rounds"], r["degenerate"]) == (n_in, rounds, deg), t
        d = geometry.se3_log(geometry.compose(geometry.inverse(mu), r["mean"]))
        tscale = 1 + np.abs(mu[:, 3]).max()
        assert np.all(np.abs(d[:3]) < 1e-9) and np.all(np.abs(d[3:]) < 1e-9 * tscale), (t, d)
        err = np.linalg.norm(r["cov"] - Sig) / np.linalg.norm(Sig)
        assert err < 1e-7, (t, err)
        assert np.allclose(r["cov"], r["cov"].T, rtol=0, atol=1e-18 + 1e-12 * np.abs(Sig).max())
        assert np.linalg.eigvalsh(r["cov"]).min() >= eps * (1 - 1e-6)
    return res


@pytest.mark.parametrize("name,seed,size,iters", [("planes160", 0, None, 3),
                                                  ("driving1216", 2001, (608, 184), 4),
                                                  ("boxes640_stereo", 7, (320, 240), 2)])
def test_covariance_matches_oracle(V, name, seed, size, iters):
    w = window(name, seed, **({"size": size} if size else {}))
    ctx, _, _ = make_ctx(V, w)
    params = V.vd_params_default(**params_for(w))   # the context's parameters
    try:
        with pytest.raises(V.VoldorError):          # no pose M-step yet
            V.vd_pose_covariance(ctx, w.N)
        V.vd_bootstrap(ctx)
        for it in range(iters):
            V.vd_run_em(ctx, 1)
            res = _compare(V, ctx, w, params, 1e-12)
        assert any(r["n_inliers"] >= 7 and not r["degenerate"] for r in res)
        _compare(V, ctx, w, params, 1e-8)           # a floor that binds
        # new poses: the samples no longer belong to the state
        V.vd_set_poses(ctx, V.vd_get_poses(ctx, w.N).reshape(-1, 12))
        with pytest.raises(V.VoldorError):
            V.vd_pose_covariance(ctx, w.N)
    finally:
        V.vd_destroy(ctx)


def test_many_samples_per_lane(V):
    """200 samples per frame: every lane owns up to 7 samples."""
    w = window("planes160", 0)
    ctx, _, _ = make_ctx(V, w, n_pose_samples=200)
    params = V.vd_params_default(**params_for(w, n_pose_samples=200))
    try:
        V.vd_bootstrap(ctx)
        V.vd_run_em(ctx, 2)
        res = _compare(V, ctx, w, params, 1e-12)
        assert all(r["n_samples"] > 64 for r in res)
    finally:
        V.vd_destroy(ctx)

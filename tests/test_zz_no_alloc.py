"""vd_score_poses_noalloc: dense pose scoring for callers that may not
allocate device memory at run time (device memory fully reserved by another
allocator, or a real-time loop where cudaMalloc's implicit synchronisation and
possible failure are not allowed).  Its scratch is a fixed array inside the
library, so it must give the same energies as vd_score_poses, which allocates
its scratch per call -- on two calls in a row, since the second call reuses
the array the first one left behind.

This file is named to be collected last, so that a failure here stops a
first-failure run only after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_06800_gb300 import build, voldor
    build.build()
    voldor.load()
    return voldor


def _problem(rng, n, m, dev):
    import torch
    from oracle import geometry
    X = rng.uniform(-3, 3, size=(n, 3))
    X[:, 2] = rng.uniform(2, 20, size=n)
    K = (300.0, 310.0, 160.0, 120.0)
    xobs = np.stack([K[0] * X[:, 0] / X[:, 2] + K[2], K[1] * X[:, 1] / X[:, 2] + K[3]], 1)
    xobs += rng.normal(size=xobs.shape)
    pts = np.concatenate([X, rng.uniform(0, 1, size=(n, 1))], 1).astype(np.float32)
    obs = np.concatenate([xobs, rng.uniform(0.4, 1.2, size=(n, 1)), np.zeros((n, 1))],
                         1).astype(np.float32)
    poses = np.stack([geometry.se3_exp(rng.normal(size=6) * 0.05) for _ in range(m)])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return t(pts), t(obs), t(poses.reshape(m, 12)), torch.tensor(K, dtype=torch.float64,
                                                                 device=dev)


def test_noalloc_matches_allocating_entry_point_twice(V):
    import torch
    dev = torch.device("cuda")
    rng = np.random.default_rng(7)
    # two calls in a row with different sizes: the second reuses the array
    for n, m in ((6000, 200), (2500, 37)):
        pts, obs, poses, K = _problem(rng, n, m, dev)
        ref = torch.zeros(m, dtype=torch.float64, device=dev)
        got = torch.full((m,), -1.0, dtype=torch.float64, device=dev)
        V.vd_score_poses(pts, obs, poses, K, 2.0, 1e-3, ref)
        V.vd_score_poses_noalloc(pts, obs, poses, K, 2.0, 1e-3, got)
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        # same tolerance as the scoring parity test against the oracle
        assert np.allclose(g, r, rtol=1e-4, atol=0)


def test_noalloc_matches_the_oracle_at_its_limits(V):
    """Against the float64 oracle's pose score (Eq. 7 scoring), at the
    largest pose count the fixed array holds and with no points at all."""
    import torch
    from oracle import model as omodel
    from oracle import pose as opose
    dev = torch.device("cuda")
    rng = np.random.default_rng(11)
    n, m = 3000, V.VD_NOALLOC_MAX_POSES
    pts, obs, poses, K = _problem(rng, n, m, dev)
    got = torch.full((m,), -1.0, dtype=torch.float64, device=dev)
    V.vd_score_poses_noalloc(pts, obs, poses, K, 2.0, 1e-3, got)
    P = omodel.Problem(10, 10, 1, tuple(K.cpu().numpy()), np.zeros((1, 10, 10, 2), np.float32))
    p = omodel.Params(fisk_beta=2.0, outlier_density=1e-3)
    pn, on = pts.cpu().numpy().astype(np.float64), obs.cpu().numpy().astype(np.float64)
    rs = dict(X=pn[:, :3], w=pn[:, 3], xobs=on[:, :2], alpha=on[:, 2])
    want = np.array([opose.score(P, G, rs, p) for G in poses.cpu().numpy().reshape(m, 3, 4)])
    assert np.allclose(got.cpu().numpy(), want, rtol=1e-4, atol=0)
    # no points: every energy is zero (and the array's last contents are not read)
    zero = torch.full((5,), -1.0, dtype=torch.float64, device=dev)
    V.vd_score_poses_noalloc(pts[:0], obs[:0], poses[:5], K, 2.0, 1e-3, zero)
    assert np.array_equal(zero.cpu().numpy(), np.zeros(5))


def test_noalloc_rejects_too_many_poses(V):
    import torch
    dev = torch.device("cuda")
    pts, obs, poses, K = _problem(np.random.default_rng(1), 100, V.VD_NOALLOC_MAX_POSES + 1, dev)
    e = torch.zeros(poses.shape[0], dtype=torch.float64, device=dev)
    with pytest.raises(V.VoldorError) as err:
        V.vd_score_poses_noalloc(pts, obs, poses, K, 2.0, 1e-3, e)
    assert err.value.status == V.VD_ERR_ARG
    assert "VD_NOALLOC_MAX_POSES" in str(err.value)

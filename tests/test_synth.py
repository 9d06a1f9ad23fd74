"""The seeded input generator (synth/): shapes, value distributions and
structure of the synthetic windows that stand in for the paper's sequences,
checked against independent definitions (scipy's Fisk law, the pinhole
projection written out here, the stated hole and blob fractions)."""
import math

import numpy as np
import pytest
from scipy import stats

import synth


def test_configurations_have_the_stated_shapes():
    w = synth.make_window("planes160", 0)
    assert (w.W, w.H, w.N) == (160, 120, 3) and w.flow.shape == (3, 120, 160, 2)
    assert w.flow.dtype == np.float32 and w.flow.flags["C_CONTIGUOUS"]
    assert w.G.shape == (4, 3, 4) and np.array_equal(w.G[0], np.eye(3, 4))
    assert w.params["n_hyp"] == 64 and w.params["n_iters"] == 3
    w = synth.make_window("boxes640_stereo", 1, size=(160, 120), N=4)
    assert (w.W, w.H, w.N) == (160, 120, 4) and w.stereo_disp.shape == (120, 160)
    assert w.stereo_baseline == 0.25 and w.depth_prior is None
    w = synth.make_window("driving1216", 2000)
    assert (w.W, w.H, w.N) == (1216, 368, 6) and w.intrinsics == (720.0, 720.0, 608.0, 184.0)
    assert w.params["n_hyp"] == 128 and w.params["n_iters"] == 8
    assert w.params["fisk_alpha0"] == 1.0 and w.params["fisk_beta"] == 2.0
    # forward motion: tens of px in the middle, a few hundred at the border
    # for the first frame pairs (later pairs pass near boxes: larger flows)
    mag = np.hypot(w.flow[..., 0], w.flow[..., 1])
    assert 20 < np.median(mag[0]) < 60 and 150 < np.percentile(mag[0], 99.9) < 400
    # depth between the nearest box face and the 80 m backstop
    assert w.depth0.min() > 0.5 and w.depth0.max() <= 80.0 + 1e-9


def test_rgbd_batch_draws_sizes_and_flow_counts():
    seen = set()
    for s in range(5000, 5012):
        rng = np.random.default_rng(s)
        size = [(320, 240), (640, 480), (1216, 368)][rng.integers(0, 3)]
        n = int(rng.integers(3, 9))
        seen.add(size)
        assert 3 <= n <= 8
    assert len(seen) == 3
    w = synth.make_window("rgbd_batch", 5001, size=(160, 120), N=3)
    assert w.depth_prior.shape == (120, 160) and w.stereo_disp is None
    assert w.params["n_iters"] == 5


def test_same_seed_same_window_and_seeds_differ():
    a = synth.make_window("boxes640_stereo", 3, size=(96, 64), N=3)
    b = synth.make_window("boxes640_stereo", 3, size=(96, 64), N=3)
    c = synth.make_window("boxes640_stereo", 4, size=(96, 64), N=3)
    assert np.array_equal(a.flow, b.flow) and np.array_equal(a.G, b.G)
    assert np.array_equal(a.stereo_disp, b.stereo_disp, equal_nan=True)
    assert not np.array_equal(a.flow, c.flow)


@pytest.mark.parametrize("alpha,beta", [(0.5, 2.0), (1.0, 2.0), (0.7, 1.5)])
def test_flow_noise_is_fisk_with_uniform_direction(alpha, beta):
    rng = np.random.default_rng(11)
    n = synth.fisk_noise(rng, (200000,), alpha, beta)
    mag = np.hypot(n[:, 0], n[:, 1])
    # scipy's log-logistic law: c = beta (shape), scale = alpha
    assert stats.kstest(mag, stats.fisk(c=beta, scale=alpha).cdf).statistic < 0.005
    ang = np.arctan2(n[:, 1], n[:, 0])
    assert stats.kstest((ang + math.pi) / (2 * math.pi), "uniform").statistic < 0.005


def test_noise_free_flow_is_the_rigid_reprojection():
    w = synth.make_window("planes160", 2, noisy=False)
    fx, fy, cx, cy = w.intrinsics
    v, u = np.mgrid[0:w.H, 0:w.W].astype(np.float64)
    X0 = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], -1) * w.depth0[..., None]
    X1 = X0 @ w.G[1][:, :3].T + w.G[1][:, 3]
    x1 = fx * X1[..., 0] / X1[..., 2] + cx
    y1 = fy * X1[..., 1] / X1[..., 2] + cy
    assert np.abs(w.flow[0, ..., 0] - (x1 - u)).max() < 1e-3
    assert np.abs(w.flow[0, ..., 1] - (y1 - v)).max() < 1e-3
    assert not w.moving.any()


def test_noisy_flow_residuals_follow_the_noise_model():
    w0 = synth.make_window("planes160", 3, noisy=False)
    w1 = synth.make_window("planes160", 3, noisy=True)
    d = (w1.flow - w0.flow).reshape(-1, 2).astype(np.float64)
    mag = np.hypot(d[:, 0], d[:, 1])
    a, b = w1.params["fisk_alpha0"], w1.params["fisk_beta"]
    # float32 storage of the flow adds ~1e-5 px
    assert stats.kstest(mag, stats.fisk(c=b, scale=a).cdf).statistic < 0.01


@pytest.mark.parametrize("name,size,frac", [("boxes640_stereo", (320, 240), 0.10),
                                            ("driving1216", None, 0.05)])
def test_moving_blobs_cover_the_stated_fraction_with_constant_flow(name, size, frac):
    w0 = synth.make_window(name, 7, noisy=False, size=size)
    w = synth.make_window(name, 7, noisy=True, size=size)
    assert not w0.moving.any()
    for t in range(w.N):
        m = w.moving[t]
        assert frac <= m.mean() < frac + 0.04
        # a blob's flow is one constant vector of 5-30 px per axis plus noise
        med = np.median(w.flow[t][m], axis=0)
        assert np.all((np.abs(med) >= 4) & (np.abs(med) <= 31))


def test_stereo_prior_noise_and_holes():
    w0 = synth.make_window("boxes640_stereo", 5, noisy=False, size=(320, 240))
    w = synth.make_window("boxes640_stereo", 5, noisy=True, size=(320, 240))
    fx = w.fx
    assert np.allclose(w0.stereo_disp, fx * 0.25 / w0.depth0, rtol=1e-6)
    holes = np.isnan(w.stereo_disp)
    assert 0.04 < holes.mean() < 0.08
    r = (w.stereo_disp - fx * 0.25 / w.depth0)[~holes]
    assert abs(np.std(r) - 0.5) < 0.02 and abs(np.mean(r)) < 0.02


def test_rgbd_prior_noise_and_holes():
    w = synth.make_window("rgbd_batch", 9, noisy=True, size=(320, 240), N=3)
    holes = np.isnan(w.depth_prior)
    assert 0.08 < holes.mean() < 0.14
    rel = (w.depth_prior / w.depth0 - 1.0)[~holes]
    assert abs(np.std(rel) - 0.01) < 0.0005 and abs(np.mean(rel)) < 0.0005


def test_keyframe_pair_depths_agree_under_the_pose():
    Z0, Zt, T, K = synth.keyframe_pair("driving1216", 3, t=2, size=(304, 92))
    fx, fy, cx, cy = K
    H, W = Zt.shape
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    Xt = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], -1) * Zt[..., None]
    X0 = Xt @ T[:, :3].T + T[:, 3]
    x = fx * X0[..., 0] / X0[..., 2] + cx
    y = fy * X0[..., 1] / X0[..., 2] + cy
    ok = (X0[..., 2] > 0.5) & (x >= 0) & (x <= W - 1) & (y >= 0) & (y <= H - 1)
    xi, yi = np.round(x[ok]).astype(int), np.round(y[ok]).astype(int)
    rel = np.abs(Z0[yi, xi] - X0[..., 2][ok]) / X0[..., 2][ok]
    assert ok.mean() > 0.5
    # nearest-pixel lookup on smooth surfaces: most agree closely (occlusion
    # and depth edges make the rest)
    assert np.median(rel) < 0.01


@pytest.mark.parametrize("seed", [2000, 2001])
def test_kerb_variant_keeps_the_lane_clear(seed):
    # the car boxes at the kerbs and beyond the camera's travel: no frame
    # pair passes close to one, so the rigid flows stay at a street
    # sequence's magnitudes (the road's bottom corners move most, ~200 px
    # at 1.5 m per frame)
    w = synth.make_window("driving1216_kerb", seed)
    assert (w.W, w.H, w.N) == (1216, 368, 6)
    mag = np.hypot(w.flow[..., 0], w.flow[..., 1])
    for t in range(w.N):
        m = mag[t][~w.moving[t]]
        assert np.percentile(m, 99) < 250 and np.percentile(m, 99.9) < 300, t
        assert (m > 400).mean() < 1e-4

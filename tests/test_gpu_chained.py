"""Whole EM runs replayed stage by stage against the float64 oracle
(paper Sec. III-A, Eq. 1-7: bootstrap, then per iteration the depth M-step,
the rigidness E-step and the pose M-step of every frame).

Every stage starts both sides from the library's own state and is held to the
method's bounds: 1e-4 relative inverse depth (tie band for choices that
float32 and float64 rank differently), 1e-4 absolute rigidness, 1e-4 rad and
1e-4 relative translation per pose.  The chained GPU run is then shown to be
bit-identical to the uninterrupted vd_bootstrap + vd_run_em (see chained.py).
"""
import numpy as np
import pytest

import synth
from oracle import geometry as ogeo
from oracle import model as omodel

from chained import crop_problem, replay
from gpu_common import params_for

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


def _factory(V, W, H, N, K, flow, params, stereo=None, depth_prior=None):
    def make():
        ctx = V.vd_create(W, H, N, K, params)
        for t in range(1, N + 1):
            V.vd_push_flow(ctx, t, flow[t - 1])
        if stereo is not None:
            V.vd_push_stereo_prior(ctx, *stereo)
        if depth_prior is not None:
            V.vd_push_depth_prior(ctx, depth_prior)
        return ctx
    return make


def test_chained_driving_kerb_crop_full_schedule(V):
    """The driving workload's schedule (N = 6, K = 128, S = 64, 8 iterations,
    directions i mod 4, monocular bootstrap) on the centred 608 x 184 crop of
    the kerb-side driving scene, every stage at the method's bounds."""
    win = synth.make_window("driving1216_kerb", 2000)
    cw, ch = 608, 184
    flow, K, _ = crop_problem(win, cw, ch)
    kw = params_for(win, n_hyp=128, n_pose_samples=64)
    P = omodel.Problem(cw, ch, win.N, K, flow)
    p = omodel.Params(**kw)
    rep = replay(V, _factory(V, cw, ch, win.N, K, flow, V.vd_params_default(**kw)), P, p,
                 win.params["n_iters"], f"driving1216_kerb seed 2000 {cw}x{ch}")
    print(rep.summary())
    assert win.params["n_iters"] == 8 and win.N == 6


def test_chained_planes_noise_free_recovers_the_scene(V):
    """Monocular, noise-free (the small workload's scene, 4 iterations): every
    stage at the bounds, and the result recovers the scene up to the
    monocular scale (depth and rotations exact to the sampling's precision)."""
    win = window = synth.make_window("planes160", 0, noisy=False)
    kw = params_for(win)
    P = omodel.problem_from_window(win)
    p = omodel.Params(**kw)
    rep = replay(V, _factory(V, win.W, win.H, win.N, win.intrinsics, win.flow,
                             V.vd_params_default(**kw)), P, p, 4, "planes160 noise-free")
    print(rep.summary())
    rho, G = rep.final.rho, rep.final.G
    rho_true = 1.0 / window.depth0
    s = float(np.median(rho_true / rho))
    assert np.median(np.abs(rho * s - rho_true) / rho_true) < 5e-3
    for t in range(1, win.N + 1):
        dR = G[t][:, :3].T @ win.G[t][:, :3]
        assert np.linalg.norm(ogeo.so3_log(dR)) < 1e-3


def test_chained_stereo_prior(V):
    """Stereo prior (the metric scale is fixed): bootstrap from the prior,
    3 iterations, every stage at the bounds."""
    win = synth.make_window("boxes640_stereo", 3, size=(160, 120), N=3)
    kw = params_for(win, n_hyp=32)
    P = omodel.problem_from_window(win)
    assert P.prior_kind == "stereo"
    p = omodel.Params(**kw)
    rep = replay(V, _factory(V, win.W, win.H, win.N, win.intrinsics, win.flow,
                             V.vd_params_default(**kw),
                             stereo=(win.stereo_disp, win.stereo_baseline)),
                 P, p, 3, "boxes640_stereo 160x120")
    print(rep.summary())

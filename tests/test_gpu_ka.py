"""Keyframe alignment on the GPU (vd_ka_align) against the oracle
(oracle/ka.py) on depth maps rendered from a scene of planes.  Both sides
are float64 with different summation orders: the energy, the normal matrix
(through the covariance) and the association counts are compared at a
fixed pose, then whole alignments."""
import numpy as np
import pytest

from ka_scene import K, W, H, pose_err, render, start, T_true
from oracle import geometry, ka

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2104_06800_gb300 import build, voldor
    build.build()
    voldor.load()
    return voldor


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _noisy(theta, rng, holes=0.03, noise=0.0005):
    th = theta * (1 + noise * rng.standard_normal(theta.shape))
    th[rng.uniform(size=th.shape) < holes] = np.nan
    return th.astype(np.float32)


def test_evaluation_at_a_fixed_pose_matches_oracle(V):
    """max_iters = 0: the energy, count and covariance of the start itself."""
    rng = np.random.default_rng(0)
    T = T_true()
    th1, th2 = _noisy(render(geometry.IDENTITY), rng), _noisy(render(T), rng)
    conf = rng.uniform(0.3, 1.0, th2.shape).astype(np.float32)
    for fix in (True, False):
        T0 = start(T, rng)
        got = V.vd_ka_align(_dev(th1), _dev(th2), K, T0, s0=1.1, conf2=_dev(conf), c=0.01,
                            fix_scale=fix, max_iters=0)
        ref = ka.align(th1, th2, K, T0, s0=1.1, conf2=conf, c=0.01, fix_scale=fix, max_iters=0)
        assert got["iterations"] == 0 and got["n_valid"] == ref["n_valid"] > 0.5 * W * H
        assert got["energy"] == pytest.approx(ref["energy"], rel=1e-10)
        assert np.allclose(got["cov"], ref["cov"], rtol=1e-8, atol=1e-14 * np.abs(ref["cov"]).max())
        assert np.array_equal(got["T"], T0)


@pytest.mark.parametrize("fix,s_true", [(True, 1.0), (False, 1.7)])
def test_alignment_matches_oracle(V, fix, s_true):
    rng = np.random.default_rng(1 if fix else 2)
    T = T_true()
    th1 = _noisy(render(geometry.IDENTITY) / s_true, rng)
    th2 = _noisy(render(T), rng)
    conf = rng.uniform(0.3, 1.0, th2.shape).astype(np.float32)
    T0 = start(T, rng)
    s0 = s_true * 1.1
    got = V.vd_ka_align(_dev(th1), _dev(th2), K, T0, s0=s0, conf2=_dev(conf), fix_scale=fix)
    ref = ka.align(th1, th2, K, T0, s0=s0, conf2=conf, fix_scale=fix)
    er, et = pose_err(got["T"], ref["T"])
    assert er < 1e-9 and et < 1e-9, (er, et)
    assert abs(got["s"] - ref["s"]) < 1e-9 * ref["s"]
    assert got["iterations"] == ref["iterations"] and got["n_valid"] == ref["n_valid"]
    assert got["energy"] == pytest.approx(ref["energy"], rel=1e-8)
    assert np.allclose(got["cov"], ref["cov"], rtol=1e-6, atol=1e-12 * np.abs(ref["cov"]).max())
    # and both near the truth (the depth noise is 0.2 %)
    er, et = pose_err(got["T"], T)
    assert er < 2e-3 and et < 2e-2 and abs(got["s"] - s_true) < 0.02 * s_true


def test_full_size_alignment_and_argument_checks(V):
    """1216 x 368 keyframes (the driving workload's size)."""
    rng = np.random.default_rng(3)
    Kf = (720.0, 720.0, 608.0, 184.0)
    T = T_true()
    th1 = _noisy(render(geometry.IDENTITY, 1216, 368, Kf), rng)
    th2 = _noisy(render(T, 1216, 368, Kf), rng)
    T0 = start(T, rng)
    got = V.vd_ka_align(_dev(th1), _dev(th2), Kf, T0, fix_scale=True)
    ref = ka.align(th1, th2, Kf, T0, fix_scale=True)
    er, et = pose_err(got["T"], ref["T"])
    assert er < 1e-9 and et < 1e-9 and got["iterations"] == ref["iterations"]
    with pytest.raises(V.VoldorError):
        V.vd_ka_align(_dev(th1), _dev(th2), Kf, T0, c=0.0)
    with pytest.raises(V.VoldorError):
        V.vd_ka_align(_dev(th1), _dev(th2), Kf, np.full((3, 4), np.nan))


def test_no_valid_pixel_is_reported_not_an_error(V):
    th = np.full((H, W), np.nan, np.float32)
    got = V.vd_ka_align(_dev(th), _dev(th), K, T_true(), fix_scale=True)
    ref = ka.align(th, th, K, T_true(), fix_scale=True)
    assert got["n_valid"] == ref["n_valid"] == 0 and got["iterations"] == ref["iterations"] == 0
    assert np.all(np.isnan(got["cov"])) and got["energy"] == 0.0
    assert np.array_equal(got["T"], T_true())

"""Pins of the keyframe-alignment oracle (oracle/ka.py) on depth maps
rendered analytically from a three-plane scene with a known relative pose
and scale, plus finite-difference Jacobians and the kernel's closed form."""
import numpy as np
import pytest

from ka_scene import H, K, W, render
from ka_scene import T_true as _T_true
from ka_scene import pose_err as _pose_err
from ka_scene import start as _start
from oracle import geometry, ka

def test_normals_of_a_plane_face_the_camera():
    th = render(geometry.IDENTITY)
    n, ok = ka.normals(th, K)
    # back wall interior: pixels around the principal point
    assert ok[60, 80] and np.allclose(n[60, 80], [0, 0, -1], atol=1e-12)
    # floor: bottom rows
    assert ok[115, 80] and np.allclose(n[115, 80], [0, -1, 0], atol=1e-12)
    assert not ok[0].any() and not ok[:, 0].any()


def test_zero_residual_at_the_true_pose_on_plane_interiors():
    T = _T_true()
    th1, th2 = render(geometry.IDENTITY), render(T)
    n1, ok1 = ka.normals(th1, K)
    r, C, _ = ka.residuals(th1, n1, ok1, th2, None, K, T, 1.0)
    assert len(r) > 0.6 * W * H
    assert np.median(np.abs(r)) < 1e-12 and np.mean(np.abs(r) < 1e-9) > 0.9


def test_hidden_points_are_not_paired_with_the_occluder():
    # keyframe 1 sees a near patch (depth 3) in front of the back wall (depth
    # ~9); keyframe 2, without the patch, sees the wall there.  Its wall
    # points land on the patch with three times the patch's depth: hidden in
    # keyframe 1, they must not be paired with the occluder
    T = _T_true()
    th1, th2 = render(geometry.IDENTITY), render(T)
    patch = np.zeros(th1.shape, bool)
    patch[40:70, 60:100] = True
    th1 = th1.copy()
    th1[patch] = 3.0
    n1, ok1 = ka.normals(th1, K)
    assert ok1[55, 80]                    # the patch interior has normals
    a = []
    r, _, _ = ka.residuals(th1, n1, ok1, th2, None, K, T, 1.0, assoc_out=a)
    assert not patch.ravel()[a[0][1]].any()
    assert len(r) > 0.5 * W * H and np.median(np.abs(r)) < 1e-12


def test_jacobian_matches_finite_differences():
    rng = np.random.default_rng(0)
    T = _start(_T_true(), rng, 0.01, 0.02)
    s = 1.1
    th1, th2 = render(geometry.IDENTITY), render(_T_true())
    n1, ok1 = ka.normals(th1, K)
    a0 = []
    r0, _, J = ka.residuals(th1, n1, ok1, th2, None, K, T, s, jac=True, assoc_out=a0)
    h = 1e-6
    for k in range(7):
        e = np.zeros(7)
        e[k] = h
        vals = []
        for sg in (1.0, -1.0):
            Tk = geometry.compose(geometry.se3_exp(sg * e[:6]), T)
            sk = s * np.exp(sg * e[6])
            a = []
            rk, _, _ = ka.residuals(th1, n1, ok1, th2, None, K, Tk, sk, assoc_out=a)
            vals.append(dict(zip(zip(*a[0]), rk)))
        same = [i for i, key in enumerate(zip(*a0[0])) if key in vals[0] and key in vals[1]]
        assert len(same) > 0.9 * len(r0)
        keys = list(zip(*a0[0]))
        fd = np.array([(vals[0][keys[i]] - vals[1][keys[i]]) / (2 * h) for i in same])
        assert np.allclose(J[same, k], fd, rtol=1e-5, atol=1e-7), k


def test_cauchy_energy_and_weights():
    r = np.array([0.0, 0.01, -0.03, 0.5])
    c = 0.01
    assert np.allclose(ka.cauchy(r, c), 0.5 * c * c * np.log(1 + (r / c) ** 2))
    assert ka.cauchy(np.array([c]), c)[0] == pytest.approx(0.5 * c * c * np.log(2.0))


def test_alignment_recovers_the_pose():
    rng = np.random.default_rng(1)
    T = _T_true()
    th1, th2 = render(geometry.IDENTITY), render(T)
    res = ka.align(th1, th2, K, _start(T, rng), fix_scale=True)
    er, et = _pose_err(res["T"], T)
    assert er < 1e-6 and et < 1e-6, (er, et, res["iterations"])
    assert res["s"] == 1.0 and np.all(np.linalg.eigvalsh(res["cov"]) > 0)


def test_alignment_recovers_the_scale():
    rng = np.random.default_rng(2)
    T = _T_true()
    s_true = 1.7
    th1 = render(geometry.IDENTITY) / s_true        # keyframe 1 in another depth gauge
    th2 = render(T)
    # from a start a keyframe alignment gets (the pose graph's estimate):
    # scale within 10 %
    res = ka.align(th1, th2, K, _start(T, rng), s0=s_true * 1.1, fix_scale=False)
    er, et = _pose_err(res["T"], T)
    assert er < 1e-6 and et < 1e-6 and abs(res["s"] - s_true) < 1e-6, (er, et, res["s"])


def test_robust_kernel_downweights_corrupted_depth():
    # 10 % of keyframe 2 pushed 8-18 % farther (inside the occlusion gate,
    # confidence 0.2): the Cauchy kernel at c = 0.002 stays far closer to
    # the truth than a practically quadratic one (c = 100) on the same data
    rng = np.random.default_rng(3)
    T = _T_true()
    th1, th2 = render(geometry.IDENTITY), render(T)
    bad = rng.uniform(size=th2.shape) < 0.1
    th2 = th2.copy()
    th2[bad] *= rng.uniform(1.08, 1.18, size=bad.sum())
    conf = np.where(bad, 0.2, 1.0)
    T0 = _start(T, rng)
    robust = ka.align(th1, th2, K, T0, conf2=conf, fix_scale=True, c=0.002)
    quad = ka.align(th1, th2, K, T0, conf2=conf, fix_scale=True, c=100.0)
    er, et = _pose_err(robust["T"], T)
    eq, tq = _pose_err(quad["T"], T)
    assert er < 0.2 * eq and et < 0.2 * tq and er < 1e-2, (er, et, eq, tq)

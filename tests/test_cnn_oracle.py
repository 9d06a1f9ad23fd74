"""Pins of the learned initialiser's float64 oracle (oracle/cnn.py) against
facts that do not come from it: a library correlation, finite differences,
the Adam closed form of a first step, and torch's bfloat16 rounding."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def test_bf16_rounding_matches_torch_and_known_values():
    torch = pytest.importorskip("torch")
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -2.5, 3.14159, 1e-3, 65504.0])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16(x), ref)
    # ties to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert cnn.bf16(1 + 2 ** -8) == 1.0 and cnn.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6
    r = np.random.default_rng(0).normal(size=1000) * 10
    ref = torch.tensor(r, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16(r), ref)


def test_conv_equals_channel_sum_of_library_correlation():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(3, 7, 9))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    z = cnn.conv(a, W, b)
    for co in range(4):
        ref = b[co] + sum(correlate2d(a[ci], W[co, :, :, ci], mode="same") for ci in range(3))
        assert np.allclose(z[co], ref, atol=1e-12)


def _tiny(rng, layers=3):
    shapes = [(4, 5), (5, 5), (5, 3)][:layers]     # two rigidness heads
    return [(rng.normal(size=(co, 3, 3, ci)) * 0.5, rng.normal(size=co) * 0.1) for ci, co in shapes]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = _tiny(rng)
    a0 = rng.normal(size=(4, 6, 5))
    rho_t = rng.uniform(0.1, 1.0, size=(6, 5))
    q_t = rng.uniform(0, 1, size=(2, 6, 5))
    mask = rng.uniform(size=(6, 5)) > 0.2
    args = (rho_t, q_t, mask, 0.05, 2.0, 0.3)

    def L_of(ps):
        z, _, _ = cnn.forward(ps, a0, bf16_storage=False)
        return cnn.loss_and_grad(z, *args)[0]

    z, acts, zs = cnn.forward(params, a0, bf16_storage=False)
    _, dz = cnn.loss_and_grad(z, *args)
    grads = cnn.backward(params, acts, zs, dz, bf16_storage=False)
    # central differences: the loss is O(100) here, so a step of 1e-4 keeps
    # the cancellation error ~1e-10 and the truncation error ~1e-8, and moves
    # no pre-activation across its ReLU kink (the smallest |z| is ~6e-3)
    h = 1e-4
    for l, (W, b) in enumerate(params):
        for idx in [(0, 0, 0, 0), (1, 2, 1, 3), (-1, 1, 2, -1)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in params]
            Wm = [(w.copy(), bb.copy()) for w, bb in params]
            Wp[l][0][idx] += h
            Wm[l][0][idx] -= h
            fd = (L_of(Wp) - L_of(Wm)) / (2 * h)
            assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx)
        for i in range(len(b)):
            Wp = [(w.copy(), bb.copy()) for w, bb in params]
            Wm = [(w.copy(), bb.copy()) for w, bb in params]
            Wp[l][1][i] += h
            Wm[l][1][i] -= h
            fd = (L_of(Wp) - L_of(Wm)) / (2 * h)
            assert abs(fd - grads[l][1][i]) <= 1e-6 * max(1.0, abs(fd)), (l, i)


def test_input_gradient_of_conv_matches_finite_differences():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(3, 5, 4))
    W = rng.normal(size=(2, 3, 3, 3))
    dz = rng.normal(size=(2, 5, 4))
    da, _, _ = cnn.conv_backward(a, W, dz)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 3), (2, 4, 1)]:
        ap, am = a.copy(), a.copy()
        ap[idx] += h
        am[idx] -= h
        fd = ((cnn.conv(ap, W, np.zeros(2)) - cnn.conv(am, W, np.zeros(2))) * dz).sum() / (2 * h)
        assert abs(fd - da[idx]) < 1e-6


def test_adam_first_step_closed_form():
    # from zero moments, m_hat = g and v_hat = g^2: the step is lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th, m, v = cnn.adam_step(np.ones(4), np.zeros(4), np.zeros(4), g, 1, 0.01)
    assert np.allclose(th, 1 - 0.01 * g / (np.abs(g) + cnn.ADAM_EPS), atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps m_hat = g, v_hat = g^2 at every step
    th, m, v = np.ones(4), np.zeros(4), np.zeros(4)
    for t in range(1, 6):
        th, m, v = cnn.adam_step(th, m, v, g, t, 0.01)
    assert np.allclose(th, 1 - 5 * 0.01 * g / (np.abs(g) + cnn.ADAM_EPS), atol=1e-12)


def test_heads_and_loss_closed_forms():
    """z_0 = 0 gives the geometric centre of the range, z_0 = ln 2 twice it,
    and the rigidness is the logistic function of its channel; the depth
    loss is the mean squared log ratio of the head's depth to the target,
    zero (with a zero gradient) where they agree."""
    rmin, rmax = 0.05, 2.0
    rc = np.sqrt(rmin * rmax)
    z = np.zeros((3, 2, 2))
    z[0, 0, 1] = np.log(2.0)
    z[1] = [[0.0, np.log(3.0)], [-np.log(3.0), 0.0]]
    rho, q = cnn.heads(z, rmin, rmax)
    assert np.allclose(rho, [[rc, 2 * rc], [rc, rc]], rtol=1e-15)
    assert np.allclose(q[0], [[0.5, 0.75], [0.25, 0.5]], rtol=1e-15)
    # targets equal to the heads' depth: zero depth loss and gradient
    q_t = np.full((2, 2, 2), 0.5)
    mask = np.ones((2, 2))
    L, dz = cnn.loss_and_grad(z, rho, q_t, mask, rmin, rmax, 0.0)
    assert abs(L) < 1e-28 and np.abs(dz[0]).max() < 1e-14
    # targets a factor e off everywhere: loss 1
    L, _ = cnn.loss_and_grad(z, rho * np.e, q_t, mask, rmin, rmax, 0.0)
    assert L == pytest.approx(1.0, rel=1e-12)


def test_shapes_and_input_planes():
    assert cnn.in_channels(6) == 16 and cnn.in_channels(3) == 16 and cnn.in_channels(8) == 32
    assert cnn.layer_shapes(6) == [(16, 32)] + [(32, 32)] * 4 + [(32, 7)]
    flow = np.zeros((2, 3, 4, 2), np.float32)
    flow[1, 2, 3] = (32.0, -64.0)
    a = cnn.input_planes(flow)
    assert a.shape == (16, 3, 4) and a[2, 2, 3] == 1.0 and a[3, 2, 3] == -2.0 and a[4:].sum() == 0


def test_geometry_planes_closed_forms():
    """Identity rotation: no rotational flow; a pure translation along the
    optical axis moves a pixel radially (away from the principal point for a
    camera moving forward, tau_z < 0 in frame-1 coordinates) by the classic
    x (rho tau_z) / (1 + rho tau_z) law; a pure rotation about the optical
    axis gives the rotated pixel."""
    K = (100.0, 100.0, 20.0, 10.0)
    H, W = 21, 41
    T = np.concatenate([np.eye(3), [[0.0], [0.0], [-1.0]]], axis=1)
    g = cnn.geometry_planes(K, T, H, W)
    v, u = np.mgrid[0:H, 0:W].astype(float)
    assert np.allclose(g[:2], 0.0)
    k = -cnn.GEO_RHO / (1 - cnn.GEO_RHO)      # point moved from z=1/rho to z=1/rho - 1
    assert np.allclose(g[2], -(u - 20) * k) and np.allclose(g[3], -(v - 10) * k)
    th = 0.1
    Rz = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    g = cnn.geometry_planes(K, np.concatenate([Rz, np.zeros((3, 1))], 1), H, W)
    xr = np.cos(th) * (u - 20) - np.sin(th) * (v - 10) + 20
    yr = np.sin(th) * (u - 20) + np.cos(th) * (v - 10) + 10
    assert np.allclose(g[0], xr - u) and np.allclose(g[1], yr - v) and np.allclose(g[2:], 0.0)

"""Learned initialiser on the GPU (tcgen05 convolutions, CUDA-core weight
gradients, Adam) against the float64 oracle in oracle/cnn.py, stage by
stage: every layer is fed the GPU's own input, so a bf16 rounding that comes
out differently in one layer does not propagate into the next comparison."""
import numpy as np
import pytest

from oracle import cnn

pytestmark = pytest.mark.gpu

RHO_MIN, RHO_MAX, W_Q = 0.05, 2.0, 0.3


@pytest.fixture(scope="module")
def V():
    from paper_2104_06800_gb300 import build, voldor
    build.build()
    voldor.load()
    return voldor


def _unpack(theta, lay):
    out = []
    for l in range(6):
        ci, co = lay["c_in"][l], lay["c_out"][l]
        w0, b0 = lay["w_offset"][l], lay["b_offset"][l]
        out.append((theta[w0:w0 + co * 9 * ci].reshape(co, 3, 3, ci).astype(np.float64),
                    theta[b0:b0 + co].astype(np.float64)))
    return out


def _chw(a):
    return np.ascontiguousarray(a.transpose(2, 0, 1)).astype(np.float64)


def _setup(V, N=6, H=61, W=100, seed=1):
    """A window of H*W pixels (a ragged last 128-pixel tile) with random flow
    and targets; the network's own He initialisation plus random biases."""
    import torch
    rng = np.random.default_rng(seed)
    net = V.vd_cnn_create(N, seed=seed)
    lay = V.vd_cnn_layout(net)
    theta = V.vd_cnn_get_params(net)
    for l in range(6):   # non-zero biases so that every term is exercised
        b0, co = lay["b_offset"][l], lay["c_out"][l]
        theta[b0:b0 + co] = rng.normal(size=co).astype(np.float32) * 0.05
    V.vd_cnn_set_params(net, theta)
    flow = (rng.normal(size=(N, H, W, 2)) * 20).astype(np.float32)
    rho_t = rng.uniform(0.1, 1.5, size=(H, W)).astype(np.float32)
    q_t = (rng.uniform(size=(N, H, W)) > 0.3).astype(np.float32)
    mask = (rng.uniform(size=(H, W)) > 0.1).astype(np.uint8)
    dev = torch.device("cuda")
    T = lambda x: torch.from_numpy(x).to(dev)
    return net, lay, theta, flow, rho_t, q_t, mask, T


def _geom(seed=0):
    """Intrinsics and a pose of flow 1 (small rotation, unit translation)."""
    from oracle import geometry as ogeo
    rng = np.random.default_rng(100 + seed)
    tau = rng.normal(size=3)
    T1 = ogeo.se3_exp(np.concatenate([rng.normal(size=3) * 0.02, tau / np.linalg.norm(tau)]))
    T1[:, 3] /= np.linalg.norm(T1[:, 3])
    return (80.0, 82.0, 50.0, 30.0), T1


def _acts(V, net, lay, W, H):
    a = [_chw(V.vd_cnn_get_activation(net, l, W, H, lay["c_in"][l])) for l in range(6)]
    z = _chw(V.vd_cnn_get_activation(net, 6, W, H, 16))
    assert np.all(z[lay["c_out"][5]:] == 0)      # padding channels of the last layer
    return a, z[:lay["c_out"][5]]


# (N, H, W): one 128-pixel tile, ragged in x and in the 4-row blocks, with
# 16 input planes; three tiles (the halo columns of each tile come from its
# neighbours), ragged rows, and 32 input planes (2N + 4 > 16)
SHAPES = [(6, 61, 100), (8, 37, 300)]


@pytest.mark.parametrize("N,H,W", SHAPES)
def test_forward_layers_match_oracle(V, N, H, W):
    import torch
    net, lay, theta, flow, *_ , T = _setup(V, N, H, W)
    try:
        rho = torch.zeros((H, W), device="cuda")
        q = torch.zeros((N, H, W), device="cuda")
        geom = _geom()
        V.vd_cnn_forward(net, T(flow), RHO_MIN, RHO_MAX, rho, q, geom=geom)
        params = _unpack(theta, lay)
        a, z = _acts(V, net, lay, W, H)
        # input planes: the flows exactly; the geometry planes (float32 here,
        # float64 in the oracle) to one bf16 step next to a rounding boundary
        ref0 = cnn.input_planes(flow, *geom)
        assert np.array_equal(a[0][:2 * N], ref0[:2 * N])
        d0 = np.abs(a[0] - ref0)
        assert np.mean(d0 == 0) > 0.99 and np.all(d0 <= 2.0 ** -7 * np.abs(ref0) + 1e-6)
        assert np.abs(ref0[2 * N:2 * N + 4]).max() > 0.1     # the geometry is there
        for l in range(6):
            Wl, bl = params[l]
            zl = cnn.conv(a[l], cnn.bf16(Wl), bl)
            if l < 5:
                ref = cnn.bf16(np.maximum(zl, 0.0))
                got = a[l + 1]
                diff = np.abs(got - ref)
                # the float32 sum and the float64 one round to the same bf16
                # except next to a rounding boundary: one bf16 step there
                assert np.mean(diff == 0) > 0.99, (l, np.mean(diff == 0))
                scale = np.abs(ref).max()
                assert np.all(diff <= 2.0 ** -7 * np.abs(ref) + 1e-5 * scale), l
            else:
                scale = np.abs(zl).max()
                assert z.shape == zl.shape == (1 + N, H, W)
                assert np.allclose(z, zl, rtol=1e-4, atol=1e-5 * scale)
        rho_ref, q_ref = cnn.heads(z, RHO_MIN, RHO_MAX)
        assert np.allclose(rho.cpu().numpy(), rho_ref, rtol=1e-5, atol=1e-6)
        assert np.allclose(q.cpu().numpy(), q_ref, rtol=1e-5, atol=1e-6)
    finally:
        V.vd_cnn_destroy(net)


@pytest.mark.parametrize("N,H,W", SHAPES)
def test_loss_and_gradients_match_oracle(V, N, H, W):
    net, lay, theta, flow, rho_t, q_t, mask, T = _setup(V, N, H, W, seed=2)
    try:
        loss = V.vd_cnn_train_step(net, T(flow), T(rho_t), T(q_t), T(mask), RHO_MIN, RHO_MAX,
                                   W_Q, 0.0, update=False, geom=_geom(2))
        g = V.vd_cnn_get_grads(net)
        params = _unpack(theta, lay)
        a, z = _acts(V, net, lay, W, H)
        L, dz = cnn.loss_and_grad(z, rho_t.astype(np.float64), q_t.astype(np.float64), mask,
                                  RHO_MIN, RHO_MAX, W_Q)
        assert abs(loss - L) <= 1e-5 * abs(L)
        # ReLU masks from the GPU's activations (z > 0 exactly where relu(z) > 0)
        zs = [a[l + 1] for l in range(5)] + [z]
        grads = cnn.backward(params, a, zs, dz)
        gg = _unpack(g, lay)
        for l in range(6):
            for got, ref in zip(gg[l], grads[l]):
                err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
                assert err < 2e-3, (l, err)
    finally:
        V.vd_cnn_destroy(net)


def test_adam_step_matches_oracle(V):
    N, H, W = 6, 40, 64
    net, lay, theta, flow, rho_t, q_t, mask, T = _setup(V, N, H, W, seed=3)
    try:
        lr = 1e-3
        V.vd_cnn_train_step(net, T(flow), T(rho_t), T(q_t), T(mask), RHO_MIN, RHO_MAX, W_Q, lr,
                            update=True)
        g = V.vd_cnn_get_grads(net).astype(np.float64)
        th1 = V.vd_cnn_get_params(net).astype(np.float64)
        ref, _, _ = cnn.adam_step(theta.astype(np.float64), np.zeros_like(g), np.zeros_like(g), g,
                                  1, lr)
        assert np.allclose(th1, ref, rtol=1e-6, atol=1e-6 * lr)
    finally:
        V.vd_cnn_destroy(net)


def test_training_lowers_the_loss(V):
    N, H, W = 6, 48, 96
    net, lay, theta, flow, rho_t, q_t, mask, T = _setup(V, N, H, W, seed=4)
    try:
        args = (T(flow), T(rho_t), T(q_t), T(mask), RHO_MIN, RHO_MAX, W_Q)
        first = V.vd_cnn_train_step(net, *args, 3e-3, update=True)
        for _ in range(60):
            last = V.vd_cnn_train_step(net, *args, 3e-3, update=True)
        assert last < 0.7 * first, (first, last)
    finally:
        V.vd_cnn_destroy(net)


def test_learned_bootstrap_runs_the_em(V):
    from gpu_common import params_for, window
    w = window("driving1216", 2002, size=(304, 92), N=6)
    net = V.vd_cnn_create(w.N, seed=5)
    ctx = V.vd_create(w.W, w.H, w.N, w.intrinsics, V.vd_params_default(**params_for(w)))
    try:
        for t in range(1, w.N + 1):
            V.vd_push_flow(ctx, t, w.flow[t - 1])
        G0 = V.vd_get_poses(ctx, w.N)
        T1 = V.vd_eight_point(ctx)
        assert np.array_equal(V.vd_get_poses(ctx, w.N), G0)      # state unchanged
        assert abs(np.linalg.norm(T1[:, 3]) - 1.0) < 1e-9
        assert np.allclose(T1[:, :3] @ T1[:, :3].T, np.eye(3), atol=1e-9)
        V.vd_bootstrap_learned(ctx, net)
        rho = np.empty((w.H, w.W), np.float32)
        q = np.empty((w.N, w.H, w.W), np.float32)
        V.vd_get_inv_depth(ctx, rho)
        V.vd_get_rigidness(ctx, q)
        pr = w.params
        assert np.all(rho >= np.float32(pr["rho_min"])) and np.all(rho <= np.float32(pr["rho_max"]))
        assert np.all((q >= 0) & (q <= 1))
        V.vd_run_em(ctx, 2)
        G = V.vd_get_poses(ctx, w.N)
        assert np.all(np.isfinite(G))
        bad = V.vd_cnn_create(3)
        with pytest.raises(V.VoldorError):
            V.vd_bootstrap_learned(ctx, bad)     # built for another N
        V.vd_cnn_destroy(bad)
    finally:
        V.vd_destroy(ctx)
        V.vd_cnn_destroy(net)


def test_a_wait_that_runs_out_reports_timeout_and_the_device_stays_usable(V):
    """The failure path of the tensor-core waits, made to run out on purpose
    by a barrier nothing completes: the kernel gives up after the poll
    budget, the host reads VD_ERR_TIMEOUT, and the device keeps working."""
    import torch
    for polls in (1, 256, 4096):
        with pytest.raises(V.VoldorError) as e:
            V.vd_check_bounded_wait(polls)
        assert e.value.status == V.VD_ERR_TIMEOUT
    with pytest.raises(V.VoldorError) as e:
        V.vd_check_bounded_wait(0)
    assert e.value.status == V.VD_ERR_ARG
    x = torch.arange(1024, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 1023 * 1024 / 2

"""Learned initialiser of the EM state (test infrastructure; no counterpart in
the paper, which starts every window from its bootstrap): a small
convolutional network mapping the N flow fields of a window to an initial
inverse depth and rigidness.  Plain float64 definition of its forward pass,
backward pass, loss and Adam step, for the GPU kernels to be checked against.

Storage precision follows the GPU: weights, the activations between layers
and the gradients dL/dz_l are bfloat16 (round to nearest, ties to even);
products and sums are float64 here (float32 accumulation of exact
bf16 x bf16 products on the GPU).
Pass ``bf16=False`` for the unrounded function (the finite-difference pins).

Architecture (all convolutions 3x3, stride 1, zero padding 1):
  input   a0[c][y][x], all divided by FLOW_SCALE: c < 2N is component c % 2
          of flow c // 2; c = 2N, 2N+1: the flow that the rotation of T_1
          alone gives pixel (x, y); c = 2N+2, 2N+3: the extra flow of a point
          at inverse depth GEO_RHO under the whole T_1 (the pose of flow 1,
          unit translation); the rest zero, and the geometry planes too
          without a pose (C0 = 16 if 2N + 4 <= 16, else 32)
  layer l z_l = conv(a_l, W_l) + b_l, W_l[co][ky][kx][ci];
          a_{l+1} = relu(z_l) for every layer but the last
  output  rho = clip(rho_c exp(z[0]), rho_min, rho_max), rho_c = sqrt(rho_min rho_max),
          q_t = sigmoid(z[t]) for flows t = 1..N (one rigidness map per flow)
Loss over pixels with mask m (e = z[0] + log rho_c - log rho*, the log error):
  L = sum m e^2 / sum m  +  w_q sum_t sum m BCE(q_t, q*_t) / (N sum m)
Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
      theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
import numpy as np

FLOW_SCALE = 32.0
GEO_RHO = 0.1
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def in_channels(n_flows):
    """Input planes: 2N flow planes and 4 geometry planes, padded to 16 or 32."""
    return 16 if 2 * n_flows + 4 <= 16 else 32


def layer_shapes(n_flows, width=32, layers=6):
    """[(C_in, C_out)] of every layer (the last has 1 + N outputs)."""
    c = [in_channels(n_flows)] + [width] * (layers - 1) + [1 + n_flows]
    return [(c[i], c[i + 1]) for i in range(layers)]


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) and widen to float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def geometry_planes(K, T1, H, W):
    """The four geometry planes [4][H][W] (in px, before the scaling)."""
    fx, fy, cx, cy = K
    T1 = np.asarray(T1, np.float64).reshape(3, 4)
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    r = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)])
    h = np.einsum("ij,jhw->ihw", T1[:, :3], r)
    d = h + GEO_RHO * T1[:, 3][:, None, None]
    ok = (h[2] > 1e-6) & (d[2] > 1e-6)
    with np.errstate(divide="ignore", invalid="ignore"):
        x0, y0 = fx * h[0] / h[2] + cx, fy * h[1] / h[2] + cy
        x1, y1 = fx * d[0] / d[2] + cx, fy * d[1] / d[2] + cy
    g = np.stack([x0 - u, y0 - v, x1 - x0, y1 - y0])
    return np.where(ok, g, 0.0)


def input_planes(flow, K=None, T1=None):
    """flow [N][H][W][2] (and the window's intrinsics K and pose T_1 of flow
    1, or none) -> a0 [C0][H][W] (float64, bf16-rounded)."""
    flow = np.asarray(flow, np.float64)
    N, H, W, _ = flow.shape
    a = np.zeros((in_channels(N), H, W))
    for t in range(N):
        a[2 * t] = flow[t, :, :, 0] / FLOW_SCALE
        a[2 * t + 1] = flow[t, :, :, 1] / FLOW_SCALE
    if T1 is not None:
        a[2 * N:2 * N + 4] = geometry_planes(K, T1, H, W) / FLOW_SCALE
    return bf16(a)


def conv(a, W, b):
    """z[co][y][x] = b[co] + sum_{ky,kx,ci} W[co][ky][kx][ci] a[ci][y+ky-1][x+kx-1]."""
    C, H, Wd = a.shape
    ap = np.pad(a, ((0, 0), (1, 1), (1, 1)))
    z = np.broadcast_to(np.asarray(b, np.float64)[:, None, None], (W.shape[0], H, Wd)).copy()
    for ky in range(3):
        for kx in range(3):
            z += np.einsum("oc,chw->ohw", W[:, ky, kx, :], ap[:, ky:ky + H, kx:kx + Wd])
    return z


def conv_backward(a, W, dz):
    """Gradients of conv(a, W, b) given dL/dz: (da, dW, db)."""
    C, H, Wd = a.shape
    ap = np.pad(a, ((0, 0), (1, 1), (1, 1)))
    dzp = np.pad(dz, ((0, 0), (1, 1), (1, 1)))
    dW = np.zeros_like(W, dtype=np.float64)
    da = np.zeros_like(a, dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            dW[:, ky, kx, :] = np.einsum("ohw,chw->oc", dz, ap[:, ky:ky + H, kx:kx + Wd])
            # z[y][x] uses a[y+ky-1][x+kx-1], so a[y][x] feeds z[y-ky+1][x-kx+1]
            da += np.einsum("oc,ohw->chw", W[:, ky, kx, :],
                            dzp[:, 2 - ky:2 - ky + H, 2 - kx:2 - kx + Wd])
    return da, dW, dz.sum(axis=(1, 2))


def forward(params, a0, bf16_storage=True):
    """params: [(W_l, b_l)].  Returns (z of the last layer, [a_l], [z_l])."""
    rnd = bf16 if bf16_storage else (lambda v: np.asarray(v, np.float64))
    acts, zs = [rnd(a0)], []
    for l, (W, b) in enumerate(params):
        z = conv(acts[-1], rnd(W), b)
        zs.append(z)
        if l + 1 < len(params):
            acts.append(rnd(np.maximum(z, 0.0)))
    return zs[-1], acts, zs


def heads(z, rho_min, rho_max):
    """(rho [H][W], q [N][H][W]) from the last layer's z [1 + N][H][W]."""
    rho_c = np.sqrt(rho_min * rho_max)
    rho = np.clip(rho_c * np.exp(z[0]), rho_min, rho_max)
    return rho, 1.0 / (1.0 + np.exp(-z[1:]))


def loss_and_grad(z, rho_t, q_t, mask, rho_min, rho_max, w_q):
    """Loss L and dL/dz of the last layer; q_t: [N][H][W] targets."""
    _, q = heads(z, rho_min, rho_max)
    q_t = np.asarray(q_t, np.float64).reshape(q.shape)
    m = np.asarray(mask, np.float64)
    nm = max(m.sum(), 1.0)
    nq = q.shape[0]
    e = z[0] + 0.5 * np.log(rho_min * rho_max) - np.log(rho_t)
    eps = 1e-12
    bce = -(q_t * np.log(np.maximum(q, eps)) + (1 - q_t) * np.log(np.maximum(1 - q, eps)))
    L = float((m * e * e).sum() / nm + w_q * (m * bce).sum() / (nq * nm))
    dz = np.zeros_like(z)
    dz[0] = m * 2.0 * e / nm
    dz[1:] = w_q * m * (q - q_t) / (nq * nm)
    return L, dz


def backward(params, acts, zs, dz_last, bf16_storage=True):
    """[(dW_l, db_l)] given dL/dz of the last layer.  With bf16 storage the
    weights are used as rounded and every dL/dz_l is stored as bf16 (as the
    activations are), before it enters the weight and input gradients."""
    rnd = bf16 if bf16_storage else (lambda v: np.asarray(v, np.float64))
    grads = [None] * len(params)
    dz = rnd(dz_last)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        da, dW, db = conv_backward(acts[l], rnd(W), dz)
        grads[l] = (dW, db)
        if l > 0:
            dz = rnd(da * (zs[l - 1] > 0.0))
    return grads


def adam_step(theta, m, v, g, t, lr):
    """One Adam step (t = 1 for the first); returns new (theta, m, v)."""
    m = ADAM_B1 * m + (1 - ADAM_B1) * g
    v = ADAM_B2 * v + (1 - ADAM_B2) * g * g
    mh = m / (1 - ADAM_B1 ** t)
    vh = v / (1 - ADAM_B2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v

"""Seeded synthetic flow windows for the dense-indirect EM (inputs only).

This module produces the inputs that both the CUDA path and the CPU oracle
consume: a window of N dense optical-flow fields X_1..X_N (X_t is defined on
frame t-1's pixel grid and points to frame t), the true reference-frame depth,
true camera poses, moving-object masks and optional stereo / RGB-D depth
priors.  It holds none of the estimation arithmetic of the method: it only ray
casts analytic scenes (planes and axis-aligned boxes), projects the hit points
and adds noise.

The paper's workloads (TartanAir, KITTI, TUM sequences with MaskFlowNet flow,
Sec. IV) are not available; these scenes stand in for them with the same
image sizes, motion types and flow magnitudes.

Conventions (shared with the library and the oracle):
  * pixel (u, v): u = column in [0, W), v = row in [0, H); arrays are [H, W].
  * pinhole K = (fx, fy, cx, cy); ray r(u, v) = ((u-cx)/fx, (v-cy)/fy, 1).
  * absolute pose G_t = (R_t, tau_t) maps frame-0 coordinates to frame t:
    X_t = R_t X_0 + tau_t, with G_0 = identity.
  * flow[t-1] (0-based storage) is X_t: frame t-1 grid -> displacement to t.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Window", "make_window", "CONFIGS", "fisk_noise"]


@dataclasses.dataclass
class Window:
    name: str
    W: int
    H: int
    N: int
    fx: float
    fy: float
    cx: float
    cy: float
    G: np.ndarray            # [N+1, 3, 4] float64 true absolute poses (frame 0 -> t)
    depth0: np.ndarray       # [H, W] float64 true depth Z of the reference frame
    flow: np.ndarray         # [N, H, W, 2] float32 (flow[t-1] = X_t)
    moving: np.ndarray       # [N, H, W] bool, pixel of frame t-1 carries non-rigid flow
    stereo_disp: np.ndarray | None = None   # [H, W] float32 disparity (px), NaN = hole
    stereo_baseline: float = 0.0
    depth_prior: np.ndarray | None = None   # [H, W] float32 depth (m), NaN = hole
    params: dict = dataclasses.field(default_factory=dict)

    @property
    def intrinsics(self):
        return (self.fx, self.fy, self.cx, self.cy)


# --------------------------------------------------------------------------
# small rigid-motion helpers (input generation only)
# --------------------------------------------------------------------------
def _rot(axis, angle):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    k = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * k + (1 - math.cos(angle)) * (k @ k)


def _compose(Ta, Tb):
    """(Ta o Tb): apply Tb first, then Ta.  Poses are [3,4] = [R | tau]."""
    R = Ta[:, :3] @ Tb[:, :3]
    tau = Ta[:, :3] @ Tb[:, 3] + Ta[:, 3]
    return np.concatenate([R, tau[:, None]], axis=1)


def fisk_noise(rng, shape, alpha, beta):
    """Isotropic 2-D noise whose magnitude is Fisk(alpha, beta) distributed.

    magnitude = alpha * (u / (1 - u))^(1/beta) is the inverse CDF of the Fisk
    (log-logistic) law; the direction is uniform on the circle."""
    u = rng.uniform(1e-12, 1 - 1e-12, size=shape)
    mag = alpha * (u / (1.0 - u)) ** (1.0 / beta)
    ang = rng.uniform(0.0, 2 * math.pi, size=shape)
    return np.stack([mag * np.cos(ang), mag * np.sin(ang)], axis=-1)


# --------------------------------------------------------------------------
# ray casting of analytic primitives
# --------------------------------------------------------------------------
class _Scene:
    def __init__(self):
        self.planes = []   # (n[3], d): points with n.X = d
        self.boxes = []    # (lo[3], hi[3]) axis aligned in frame-0 coordinates

    def cast(self, G, W, H, fx, fy, cx, cy):
        """Ray cast the pixel grid of a camera with absolute pose G.

        Returns world points P [H, W, 3] and the camera depth Z [H, W]."""
        R, tau = G[:, :3], G[:, 3]
        u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
        rc = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=-1)  # z = 1
        D = rc @ R            # world direction (R^T rc), per pixel
        C = -R.T @ tau        # camera centre in world
        lam = np.full((H, W), np.inf)
        for n, d in self.planes:
            n = np.asarray(n, np.float64)
            den = D @ n
            with np.errstate(divide="ignore", invalid="ignore"):
                l = (d - n @ C) / den
            l = np.where((l > 1e-6) & np.isfinite(l), l, np.inf)
            lam = np.minimum(lam, l)
        with np.errstate(divide="ignore"):
            inv = [1.0 / D[..., k] for k in range(3)]
        for lo, hi in self.boxes:
            lo = np.asarray(lo, np.float64)
            hi = np.asarray(hi, np.float64)
            # slab test; fmax / fmin skip the NaN of a ray parallel to a slab
            # face (0 * inf), as a NaN-ignoring max / min over the axes would
            tmin = tmax = None
            with np.errstate(invalid="ignore"):
                for k in range(3):
                    t1 = (lo[k] - C[k]) * inv[k]
                    t2 = (hi[k] - C[k]) * inv[k]
                    a, b = np.minimum(t1, t2), np.maximum(t1, t2)
                    tmin = a if tmin is None else np.fmax(tmin, a)
                    tmax = b if tmax is None else np.fmin(tmax, b)
            hit = (tmax >= tmin) & (tmin > 1e-6)
            lam = np.minimum(lam, np.where(hit, tmin, np.inf))
        lam = np.where(np.isfinite(lam), lam, 1e3)
        P = C + D * lam[..., None]
        return P, lam


def _project(G, P, fx, fy, cx, cy):
    X = P @ G[:, :3].T + G[:, 3]
    z = np.maximum(X[..., 2], 1e-9)
    return np.stack([fx * X[..., 0] / z + cx, fy * X[..., 1] / z + cy], axis=-1), X[..., 2]


def _blob_mask(rng, H, W, frac, rmin, rmax):
    """Union of random ellipses covering about `frac` of the image."""
    m = np.zeros((H, W), bool)
    if frac <= 0:
        return m
    v, u = np.mgrid[0:H, 0:W]
    target = frac * H * W
    for _ in range(1000):
        if m.sum() >= target:
            break
        cu, cv = rng.uniform(0, W), rng.uniform(0, H)
        a, b = rng.uniform(rmin, rmax), rng.uniform(rmin, rmax)
        th = rng.uniform(0, math.pi)
        du, dv = u - cu, v - cv
        x = du * math.cos(th) + dv * math.sin(th)
        y = -du * math.sin(th) + dv * math.cos(th)
        m |= (x / a) ** 2 + (y / b) ** 2 <= 1.0
    return m


Z_NEAR = 0.5   # m


def _flows(rng, scene, G, W, H, N, K, noise_alpha, noise_beta, moving_frac, noisy, blob_r):
    fx, fy, cx, cy = K
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    flow = np.zeros((N, H, W, 2), np.float64)
    moving = np.zeros((N, H, W), bool)
    for t in range(1, N + 1):
        P, _ = scene.cast(G[t - 1], W, H, fx, fy, cx, cy)
        x, zt = _project(G[t], P, fx, fy, cx, cy)
        f = np.stack([x[..., 0] - u, x[..., 1] - v], axis=-1)
        # a scene point less than Z_NEAR in front of camera t (the camera has
        # passed it) has no flow: an estimator returns a bounded guess there,
        # which the model must treat as an outlier; take zero motion
        f[zt < Z_NEAR] = 0.0
        m = _blob_mask(rng, H, W, moving_frac, *blob_r)
        if m.any():
            # independently moving blobs: one constant random flow per blob image
            mv = rng.uniform(5, 30, size=2) * rng.choice([-1, 1], size=2)
            f[m] = mv
        if noisy:
            f = f + fisk_noise(rng, (H, W), noise_alpha, noise_beta)
        flow[t - 1] = f
        moving[t - 1] = m
    return flow.astype(np.float32), moving


def _holes(rng, H, W, frac):
    """Half random pixels, half blobs."""
    m = rng.uniform(size=(H, W)) < frac * 0.5
    m |= _blob_mask(rng, H, W, frac * 0.5, 3, max(4, min(H, W) // 12))
    return m


# --------------------------------------------------------------------------
# the configurations
# --------------------------------------------------------------------------
def _cfg_planes(rng, noisy):
    W, H, N = 160, 120, 3
    K = (120.0, 120.0, 80.0, 60.0)
    sc = _Scene()
    # two tilted planes forming a ridge, plus a backstop at 10 m
    da, db = rng.uniform(3.0, 6.0, size=2)
    ta, tb = np.deg2rad(rng.uniform(15, 35, size=2))
    na = _rot([0, 1, 0], ta) @ np.array([0, 0, 1.0])
    nb = _rot([0, 1, 0], -tb) @ np.array([0, 0, 1.0])
    na = _rot([1, 0, 0], np.deg2rad(rng.uniform(-10, 10))) @ na
    sc.planes.append((na, da * na[2]))
    sc.planes.append((nb, db * nb[2]))
    sc.planes.append((np.array([0, 0, 1.0]), 10.0))
    G = [np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)]
    for _ in range(N):
        ax = rng.normal(size=3)
        R = _rot(ax, np.deg2rad(rng.uniform(1.0, 5.0)))
        d = rng.normal(size=3)
        d = d / np.linalg.norm(d) * rng.uniform(0.1, 0.2)
        T = np.concatenate([R, d[:, None]], axis=1)
        G.append(_compose(T, G[-1]))
    G = np.stack(G)
    flow, moving = _flows(rng, sc, G, W, H, N, K, 0.5, 2.0, 0.0, noisy, (4, 12))
    return W, H, N, K, sc, G, flow, moving, dict(fisk_alpha0=0.5, fisk_beta=2.0, n_hyp=64,
                                                  n_iters=3, dmin=2.0, dmax=10.0,
                                                  tmin=0.1, tmax=0.2)


def _cfg_boxes(rng, noisy, W=640, H=480, N=5, moving=0.10, dmax=40.0):
    f = 525.0 * W / 640.0
    K = (f, f, W / 2.0, H / 2.0)
    sc = _Scene()
    cam_h = 1.5
    sc.planes.append((np.array([0, -1.0, 0]), -cam_h))   # ground: y = cam_h (y points down)
    sc.planes.append((np.array([0, 0, 1.0]), dmax))      # far wall
    for _ in range(20):
        z = rng.uniform(3.0, dmax * 0.9)
        x = rng.uniform(-12, 12)
        sx, sy, sz = rng.uniform(0.5, 3.0, size=3)
        lo = np.array([x - sx / 2, cam_h - sy, z - sz / 2])
        hi = np.array([x + sx / 2, cam_h, z + sz / 2])
        sc.boxes.append((lo, hi))
    G = [np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)]
    yaw_rate = rng.uniform(-1.5, 1.5)
    for _ in range(N):
        R = _rot([0, 1, 0], np.deg2rad(yaw_rate + rng.normal(0, 0.3))) @ \
            _rot([1, 0, 0], np.deg2rad(rng.normal(0, 0.3)))
        d = np.array([rng.normal(0, 0.03), rng.normal(0, 0.01), -rng.uniform(0.2, 0.4)])
        T = np.concatenate([R, d[:, None]], axis=1)
        G.append(_compose(T, G[-1]))
    G = np.stack(G)
    flow, mv = _flows(rng, sc, G, W, H, N, K, 0.5, 2.0, moving, noisy, (6, max(10, W // 16)))
    return W, H, N, K, sc, G, flow, mv, dict(fisk_alpha0=0.5, fisk_beta=2.0, n_hyp=64,
                                              n_iters=5, dmin=1.0, dmax=dmax,
                                              tmin=0.2, tmax=0.45)


def _cfg_driving(rng, noisy, W=1216, H=368, N=6, kerb=False):
    """kerb: the car boxes stand at the kerbs (|x| >= 2.5 m) and at least
    12 m ahead, beyond the camera's travel over the window (at most 9 m), so
    that the camera passes none of them; otherwise anywhere across the street
    from 6 m on, so that the camera passes close to some of them."""
    K = (720.0, 720.0, W / 2.0, H / 2.0)
    sc = _Scene()
    cam_h = 1.65
    sc.planes.append((np.array([0, -1.0, 0]), -cam_h))     # road
    sc.planes.append((np.array([0, 0, 1.0]), 80.0))        # far backstop
    xl, xr = rng.uniform(6, 12), rng.uniform(6, 12)
    sc.planes.append((np.array([1.0, 0, 0]), -xl))         # left facade x = -xl
    sc.planes.append((np.array([-1.0, 0, 0]), -xr))        # right facade x = +xr
    for _ in range(12):
        z = rng.uniform(12.0 if kerb else 6.0, 60.0)
        if kerb:
            x = -rng.uniform(2.5, xl - 1) if rng.uniform() < 0.5 else rng.uniform(2.5, xr - 1)
        else:
            x = rng.uniform(-xl + 1, xr - 1)
        lo = np.array([x - 0.9, cam_h - 1.5, z - 2.0])
        hi = np.array([x + 0.9, cam_h, z + 2.0])
        sc.boxes.append((lo, hi))
    G = [np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)]
    for _ in range(N):
        R = _rot([0, 1, 0], np.deg2rad(rng.uniform(-2, 2)))
        d = np.array([rng.normal(0, 0.02), rng.normal(0, 0.01), -rng.uniform(1.0, 1.5)])
        T = np.concatenate([R, d[:, None]], axis=1)
        G.append(_compose(T, G[-1]))
    G = np.stack(G)
    flow, mv = _flows(rng, sc, G, W, H, N, K, 1.0, 2.0, 0.05 if noisy else 0.0, noisy, (8, 40))
    return W, H, N, K, sc, G, flow, mv, dict(fisk_alpha0=1.0, fisk_beta=2.0, n_hyp=128,
                                              n_iters=8, dmin=2.0, dmax=80.0,
                                              tmin=1.0, tmax=1.55)


CONFIGS = {
    # name: (builder, description)
    "planes160": "160x120 N=3, two random planes 2-10 m, small random motion, Fisk noise 0.5 px",
    "boxes640_stereo": "640x480 N=5, ground + 20 boxes 1-40 m, 10% moving blobs, stereo prior",
    "driving1216": "1216x368 N=6, road + facades + boxes 2-80 m, forward 1-1.5 m/frame, 5% moving",
    "driving1216_kerb": "driving1216 with the car boxes at the kerbs, 12-60 m ahead (none passed)",
    "rgbd_batch": "320x240 / 640x480 / 1216x368, N 3..8, RGB-D prior 1% noise 10% holes",
}


def _config(name, rng, noisy, N, size):
    """Scene, poses, flows and parameters of one window of config `name`."""
    if name == "planes160":
        return _cfg_planes(rng, noisy)
    if name == "boxes640_stereo":
        W, H = size or (640, 480)
        return _cfg_boxes(rng, noisy, W, H, N or 5, 0.10 if noisy else 0.0)
    if name in ("driving1216", "driving1216_kerb"):
        W, H = size or (1216, 368)
        return _cfg_driving(rng, noisy, W, H, N or 6, kerb=name.endswith("_kerb"))
    if name == "rgbd_batch":
        if size is None:
            size = [(320, 240), (640, 480), (1216, 368)][rng.integers(0, 3)]
        Nw = N or int(rng.integers(3, 9))
        W, H = size
        out = _cfg_boxes(rng, noisy, W, H, Nw, 0.05 if noisy else 0.0)
        out[8]["n_iters"] = 5
        return out
    raise ValueError(f"unknown window config {name!r}")


def keyframe_pair(name: str = "driving1216", seed: int = 0, t: int = 3,
                  size: tuple[int, int] | None = None):
    """Two keyframes of one window's scene: the true depth Z of the reference
    frame and of frame t (float32 [H, W]), the pose that maps frame-t
    coordinates to reference coordinates (G_0 G_t^-1, 3x4) and the
    intrinsics (fx, fy, cx, cy)."""
    rng = np.random.default_rng(seed)
    W, H, _, K, sc, G, _, _, _ = _config(name, rng, False, None, size)
    fx, fy, cx, cy = K
    _, Z0 = sc.cast(G[0], W, H, fx, fy, cx, cy)
    _, Zt = sc.cast(G[t], W, H, fx, fy, cx, cy)
    Rt, taut = G[t][:, :3], G[t][:, 3]
    inv = np.hstack([Rt.T, (-Rt.T @ taut)[:, None]])
    T = _compose(G[0], inv)
    return Z0.astype(np.float32), Zt.astype(np.float32), T, (fx, fy, cx, cy)


def make_window(name: str, seed: int = 0, noisy: bool = True, N: int | None = None,
                size: tuple[int, int] | None = None) -> Window:
    """Build one seeded synthetic window.

    name  : one of CONFIGS.
    seed  : numpy Generator seed (every random choice of the scene derives from it).
    noisy : add Fisk flow noise (and moving blobs where the config has them).
    N, size : optional overrides of the flow count and (W, H) (rgbd_batch and tests)."""
    rng = np.random.default_rng(seed)
    stereo = depth_prior = None
    baseline = 0.25 if name == "boxes640_stereo" else 0.0
    W, H, Nn, K, sc, G, flow, mv, prm = _config(name, rng, noisy, N, size)
    fx, fy, cx, cy = K
    _, Z0 = sc.cast(G[0], W, H, fx, fy, cx, cy)
    if name == "boxes640_stereo":
        d = fx * baseline / Z0
        if noisy:
            d = d + rng.normal(0.0, 0.5, size=d.shape)
            d[_holes(rng, H, W, 0.05)] = np.nan
        stereo = d.astype(np.float32)
    if name == "rgbd_batch":
        z = Z0.copy()
        if noisy:
            z = z * (1.0 + 0.01 * rng.normal(size=z.shape))
            z[_holes(rng, H, W, 0.10)] = np.nan
        depth_prior = z.astype(np.float32)
    # inverse-depth search range: metric when a prior fixes the scale, else in
    # units of |tau_1| (the monocular bootstrap normalises the first
    # translation), from the workload's bounds on depth and per-frame motion
    # (tmin..tmax, the generator's), never from this window's true motion
    metric = stereo is not None or depth_prior is not None
    lo, hi = (1.0, 1.0) if metric else (prm["tmin"], prm["tmax"])
    prm = dict(prm)
    prm["rho_min"] = float(np.float32(0.5 * lo / prm["dmax"]))
    prm["rho_max"] = float(np.float32(2.0 * hi / prm["dmin"]))
    # the true |tau_1| (the monocular gauge of the scene's depth): tests only
    prm["scale"] = 1.0 if metric else float(np.linalg.norm(G[1][:, 3]))
    return Window(name=name, W=W, H=H, N=Nn, fx=fx, fy=fy, cx=cx, cy=cy, G=G, depth0=Z0,
                  flow=np.ascontiguousarray(flow), moving=mv, stereo_disp=stereo,
                  stereo_baseline=baseline, depth_prior=depth_prior, params=prm)

"""ctypes binding of libvoldor_em.so (the C ABI in include/voldor_em.h).

Argument marshalling only: every function below converts Python arguments to
the C types and calls the entry point of the same name; all computation runs
in the library's CUDA kernels.  Buffers may be numpy arrays (host memory,
VD_MEM_HOST) or CUDA torch tensors (device memory, VD_MEM_DEVICE).

The library must have been built (``paper_2104_06800_gb300.build.build()``);
there is no fallback: a missing library raises at load time.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvoldor_em.so")

VD_OK, VD_WARN_DEGENERATE = 0, 1
VD_ERR_ARG, VD_ERR_CUDA, VD_ERR_OOM, VD_ERR_STATE, VD_ERR_TIMEOUT, VD_ERR_NUMERIC = -1, -2, -3, -4, -5, -6
VD_MEM_HOST, VD_MEM_DEVICE = 0, 1
VD_POSE_ABSOLUTE, VD_POSE_RELATIVE = 0, 1


class vd_window_desc(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("n_flows", C.c_int),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double)]


class vd_params(C.Structure):
    _fields_ = [("fisk_alpha0", C.c_float), ("fisk_alpha1", C.c_float), ("fisk_beta", C.c_float),
                ("outlier_density", C.c_float), ("gamma_stay", C.c_float),
                ("rho_min", C.c_float), ("rho_max", C.c_float),
                ("n_hyp", C.c_int), ("n_pose_samples", C.c_int),
                ("pose_sigma_rot", C.c_double), ("pose_sigma_trans_rel", C.c_double),
                ("pose_sigma_trans_abs", C.c_double),
                ("sample_share", C.c_int), ("hierarchical", C.c_int), ("hier_scale", C.c_int),
                ("hier_window", C.c_int), ("prior_c_sigma", C.c_float),
                ("prior_w_uniform", C.c_float), ("seed", C.c_ulonglong)]


class vd_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("bootstrapped", C.c_int), ("degenerate_frames", C.c_int),
                ("mean_energy", C.c_double), ("rigid_fraction", C.c_double)]


VD_N_STAGES = 8
STAGE_NAMES = ("depth_sample", "depth_propagate", "rigidness_estep", "pose_rigid_set",
               "pose_p3p", "pose_score", "pose_select_meanshift", "bootstrap_other")


class vd_profile(C.Structure):
    _fields_ = [("ms", C.c_double * VD_N_STAGES), ("calls", C.c_longlong * VD_N_STAGES),
                ("launches", C.c_longlong * VD_N_STAGES), ("total_launches", C.c_longlong),
                ("score_evals", C.c_longlong)]


class vd_tune(C.Structure):
    _fields_ = [("k1_warps", C.c_int), ("score_threads", C.c_int),
                ("score_blocks_per_sm", C.c_int), ("k1_ms", C.c_float * 3),
                ("score_ms", (C.c_float * 4) * 2)]


class vd_cnn_geometry(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("T1", C.c_double * 12)]


class vd_batch_stats(C.Structure):
    _fields_ = [("windows", C.c_int), ("captures", C.c_longlong), ("replays", C.c_longlong),
                ("graph_nodes", C.c_longlong), ("kernels_per_run", C.c_longlong)]


VD_BATCH_BOOTSTRAP = 1
VD_BATCH_AUTOTUNE = 2
VD_VC_MAX_FRAMES = 8


class vd_ka(C.Structure):
    _fields_ = [("pose", C.c_double * 12), ("s", C.c_double), ("cauchy_c", C.c_double),
                ("fix_scale", C.c_int), ("max_iters", C.c_int), ("cov", C.c_double * 36),
                ("energy", C.c_double), ("iterations", C.c_int), ("n_valid", C.c_longlong)]


class vd_pose_cov(C.Structure):
    _fields_ = [("mean", C.c_double * 12), ("cov", C.c_double * 36), ("n_samples", C.c_int),
                ("n_inliers", C.c_int), ("rounds", C.c_int), ("degenerate", C.c_int)]


class vd_vc(C.Structure):
    _fields_ = [("n_frames", C.c_int), ("n_pixels", C.c_longlong), ("n_depth", C.c_longlong),
                ("n_visible", C.c_longlong * VD_VC_MAX_FRAMES),
                ("n_covered", C.c_longlong * VD_VC_MAX_FRAMES),
                ("visibility", C.c_double * VD_VC_MAX_FRAMES),
                ("coverage", C.c_double * VD_VC_MAX_FRAMES),
                ("vc", C.c_double * VD_VC_MAX_FRAMES)]


class VoldorError(RuntimeError):
    def __init__(self, fn, status, lib):
        msg = lib.vd_status_str(status).decode()
        last = lib.vd_last_error().decode()
        super().__init__(f"{fn} -> {status} ({msg}){': ' + last if last else ''}")
        self.status = status


_P = C.c_void_p
_SIGS = {
    "vd_params_default": [C.POINTER(vd_params)],
    "vd_create": [C.POINTER(vd_window_desc), C.POINTER(vd_params), _P, C.POINTER(_P)],
    "vd_destroy": [_P],
    "vd_set_stream": [_P, _P],
    "vd_set_params": [_P, C.POINTER(vd_params)],
    "vd_push_flow": [_P, C.c_int, _P, C.c_long, C.c_int],
    "vd_push_stereo_prior": [_P, _P, C.c_double, C.c_int],
    "vd_push_depth_prior": [_P, _P, _P, _P, C.c_int],
    "vd_clear_prior": [_P],
    "vd_set_poses": [_P, _P, C.c_int],
    "vd_get_poses": [_P, _P, C.c_int],
    "vd_set_state": [_P, _P, _P, _P, C.c_int],
    "vd_bootstrap": [_P],
    "vd_run_em": [_P, C.c_int, C.POINTER(vd_stats)],
    "vd_depth_mstep": [_P, C.c_int, C.c_int],
    "vd_rigidness_estep": [_P, C.c_int],
    "vd_pose_mstep": [_P, C.c_int, C.c_int],
    "vd_get_inv_depth": [_P, _P, C.c_int],
    "vd_get_rigidness": [_P, _P, C.c_int],
    "vd_get_prior_rigidness": [_P, _P, C.c_int],
    "vd_get_confidence": [_P, _P, C.c_int],
    "vd_get_depth_candidates": [_P, _P, _P, C.c_int],
    "vd_eval_energy": [_P, _P, _P, C.c_int],
    "vd_get_pose_samples": [_P, _P, _P, _P],
    "vd_score_poses": [_P, _P, C.c_int, _P, C.c_int, _P, C.c_float, C.c_float, _P, _P],
    "vd_score_poses_noalloc": [_P, _P, C.c_int, _P, C.c_int, _P, C.c_float, C.c_float, _P, _P],
    "vd_profile_enable": [_P, C.c_int],
    "vd_get_profile": [_P, C.POINTER(vd_profile)],
    "vd_autotune": [_P, C.POINTER(vd_tune)],
    "vd_set_tune": [_P, C.POINTER(vd_tune)],
    "vd_get_tune": [_P, C.POINTER(vd_tune)],
    "vd_batch_create": [C.c_int, C.POINTER(vd_window_desc), C.POINTER(vd_params), C.c_int, _P,
                        C.POINTER(_P)],
    "vd_batch_destroy": [_P],
    "vd_batch_window": [_P, C.c_int, C.POINTER(_P)],
    "vd_batch_run": [_P, C.c_int, C.c_int, _P],
    "vd_batch_get_stats": [_P, C.POINTER(vd_batch_stats)],
    "vd_check_bounded_wait": [C.c_int, _P],
    "vd_probe_pipe": [C.c_int, C.c_int, C.c_int, _P, _P],
    "vd_check_report": [_P],
    "vd_cnn_create": [C.c_int, C.c_ulonglong, C.POINTER(_P)],
    "vd_cnn_destroy": [_P],
    "vd_cnn_layout": [_P, C.POINTER(C.c_int), _P, _P, _P, _P],
    "vd_cnn_get_params": [_P, _P],
    "vd_cnn_set_params": [_P, _P],
    "vd_cnn_get_grads": [_P, _P],
    "vd_cnn_forward": [_P, _P, C.c_int, C.c_int, C.POINTER(vd_cnn_geometry), C.c_float,
                       C.c_float, _P, _P, _P],
    "vd_cnn_get_activation": [_P, C.c_int, _P, C.c_int, C.c_int],
    "vd_cnn_train_step": [_P, _P, C.c_int, C.c_int, C.POINTER(vd_cnn_geometry), _P, _P, _P,
                          C.c_float, C.c_float, C.c_float, C.c_float, C.c_int,
                          C.POINTER(C.c_double), _P],
    "vd_eight_point": [_P, _P],
    "vd_vc_scores": [_P, C.POINTER(vd_vc)],
    "vd_pose_covariance": [_P, C.c_double, _P],
    "vd_ka_align": [_P, _P, _P, C.c_int, C.c_int, _P, C.POINTER(vd_ka), _P],
    "vd_get_frame_samples": [_P, C.c_int, _P, _P],
    "vd_vc_pose": [_P, _P, C.POINTER(vd_vc)],
    "vd_vc_stride": [_P, C.c_int, C.c_double],
    "vd_vc_is_keyframe": [C.c_double, C.c_double],
    "vd_bootstrap_learned": [_P, _P],
    "vd_export_state": [_P, _P, C.POINTER(C.c_size_t)],
    "vd_import_state": [_P, _P, C.c_size_t],
}

_lib = None


def load(path: str | None = None):
    """Load the shared library (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"{p} not found: build it with paper_2104_06800_gb300.build.build()")
    lib = C.CDLL(p)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.vd_status_str.argtypes = [C.c_int]
    lib.vd_status_str.restype = C.c_char_p
    lib.vd_last_error.argtypes = []
    lib.vd_last_error.restype = C.c_char_p
    if path is None:
        _lib = lib
    return lib


def _check(name, st, allow_warn=True):
    if st == VD_OK or (allow_warn and st == VD_WARN_DEGENERATE):
        return st
    raise VoldorError(name, st, load())


def _call(name, *args, allow_warn=True):
    return _check(name, getattr(load(), name)(*args), allow_warn)


# ------------------------------------------------------------------ buffers
def _is_tensor(x):
    return type(x).__module__.startswith("torch")


def _buf(x, dtype=np.float32):
    """(pointer, mem kind, keep-alive) of a numpy array or CUDA tensor."""
    if x is None:
        return None, VD_MEM_HOST, None
    if _is_tensor(x):
        if not x.is_cuda:
            x = x.numpy()
        else:
            if not x.is_contiguous():
                raise ValueError("device tensors must be contiguous")
            return C.c_void_p(x.data_ptr()), VD_MEM_DEVICE, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), VD_MEM_HOST, a


def current_stream():
    """The torch current CUDA stream handle (0 when torch has no CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


# ------------------------------------------------------------------ entry points
def vd_params_default(**overrides):
    p = vd_params()
    _call("vd_params_default", C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def vd_create(W, H, N, K, params=None, stream=None):
    d = vd_window_desc(int(W), int(H), int(N), *[float(v) for v in K])
    h = C.c_void_p()
    _call("vd_create", C.byref(d), C.byref(params) if params is not None else None,
          stream if stream is not None else current_stream(), C.byref(h))
    return h


def vd_destroy(ctx):
    _call("vd_destroy", ctx)


def vd_set_stream(ctx, stream):
    _call("vd_set_stream", ctx, stream)


def vd_set_params(ctx, params):
    _call("vd_set_params", ctx, C.byref(params))


def vd_push_flow(ctx, t, uv, row_pitch_floats=None):
    ptr, mem, keep = _buf(uv)
    W = uv.shape[-2]
    _call("vd_push_flow", ctx, int(t), ptr, int(row_pitch_floats or 2 * W), mem)


def vd_push_stereo_prior(ctx, disparity, baseline):
    ptr, mem, keep = _buf(disparity)
    _call("vd_push_stereo_prior", ctx, ptr, float(baseline), mem)


def vd_push_depth_prior(ctx, depth, confidence=None, T_hat=None):
    ptr, mem, keep = _buf(depth)
    cptr, cmem, ckeep = _buf(confidence)
    if confidence is not None and cmem != mem:
        raise ValueError("depth and confidence must live in the same memory")
    tptr = None
    if T_hat is not None:
        T_hat = np.ascontiguousarray(T_hat, np.float64).reshape(12)
        tptr = T_hat.ctypes.data_as(C.c_void_p)
    _call("vd_push_depth_prior", ctx, ptr, cptr, tptr, mem)


def vd_clear_prior(ctx):
    _call("vd_clear_prior", ctx)


def vd_set_poses(ctx, poses, kind=VD_POSE_ABSOLUTE):
    a = np.ascontiguousarray(poses, np.float64)
    _call("vd_set_poses", ctx, a.ctypes.data_as(C.c_void_p), int(kind))


def vd_get_poses(ctx, N, kind=VD_POSE_ABSOLUTE):
    n = N + 1 if kind == VD_POSE_ABSOLUTE else N
    out = np.zeros((n, 3, 4), np.float64)
    _call("vd_get_poses", ctx, out.ctypes.data_as(C.c_void_p), int(kind))
    return out


def vd_set_state(ctx, rho, q=None, q_hat=None):
    p1, m1, k1 = _buf(rho)
    p2, m2, k2 = _buf(q)
    p3, m3, k3 = _buf(q_hat)
    for x, m in ((q, m2), (q_hat, m3)):
        if x is not None and m != m1:
            raise ValueError("state buffers must live in the same memory")
    _call("vd_set_state", ctx, p1, p2, p3, m1)


def vd_bootstrap(ctx):
    return _call("vd_bootstrap", ctx)


def vd_run_em(ctx, n_iters, stats=True):
    s = vd_stats()
    st = _call("vd_run_em", ctx, int(n_iters), C.byref(s) if stats else None)
    return st, s


def vd_depth_mstep(ctx, iter, direction):
    _call("vd_depth_mstep", ctx, int(iter), int(direction))


def vd_rigidness_estep(ctx, direction):
    _call("vd_rigidness_estep", ctx, int(direction))


def vd_pose_mstep(ctx, iter, t):
    return _call("vd_pose_mstep", ctx, int(iter), int(t))


def _get(name, ctx, out):
    ptr, mem, keep = _buf(out)
    if mem == VD_MEM_HOST and keep is not out:
        raise ValueError("host outputs must be contiguous float32 numpy arrays")
    _call(name, ctx, ptr, mem)
    return out


def vd_get_inv_depth(ctx, out):
    return _get("vd_get_inv_depth", ctx, out)


def vd_get_rigidness(ctx, out):
    return _get("vd_get_rigidness", ctx, out)


def vd_get_prior_rigidness(ctx, out):
    return _get("vd_get_prior_rigidness", ctx, out)


def vd_get_confidence(ctx, out):
    return _get("vd_get_confidence", ctx, out)


def vd_get_depth_candidates(ctx, rho_star, e_star):
    p1, m1, k1 = _buf(rho_star)
    p2, m2, k2 = _buf(e_star)
    _call("vd_get_depth_candidates", ctx, p1, p2, m1)
    return rho_star, e_star


def vd_eval_energy(ctx, rho, out):
    p1, m1, k1 = _buf(rho)
    p2, m2, k2 = _buf(out)
    if m1 != m2:
        raise ValueError("rho and out must live in the same memory")
    _call("vd_eval_energy", ctx, p1, p2, m1)
    return out


def vd_get_pose_samples(ctx, S):
    poses = np.zeros((S, 3, 4), np.float64)
    en = np.zeros(S, np.float64)
    n = C.c_int(0)
    _call("vd_get_pose_samples", ctx, poses.ctypes.data_as(C.c_void_p),
          en.ctypes.data_as(C.c_void_p), C.byref(n))
    return poses, en, int(n.value)


def vd_score_poses(points, obs, poses, intrinsics, beta, p0, energies, stream=None):
    """All arguments except beta, p0 and stream are CUDA tensors."""
    n = points.shape[0]
    m = poses.shape[0]
    _call("vd_score_poses", C.c_void_p(points.data_ptr()), C.c_void_p(obs.data_ptr()), int(n),
          C.c_void_p(poses.data_ptr()), int(m), C.c_void_p(intrinsics.data_ptr()), float(beta),
          float(p0), C.c_void_p(energies.data_ptr()), stream if stream is not None else current_stream())
    return energies


def vd_profile_enable(ctx, enable=True):
    _call("vd_profile_enable", ctx, 1 if enable else 0)


def vd_get_profile(ctx):
    p = vd_profile()
    _call("vd_get_profile", ctx, C.byref(p))
    return {name: dict(ms=p.ms[i], calls=p.calls[i], launches=p.launches[i])
            for i, name in enumerate(STAGE_NAMES)} | {"total_launches": p.total_launches,
                                                      "score_evals": p.score_evals}


VD_NOALLOC_MAX_POSES = 256


def vd_score_poses_noalloc(points, obs, poses, intrinsics, beta, p0, energies, stream=None):
    """vd_score_poses without any device allocation (scratch in a fixed
    library array; at most VD_NOALLOC_MAX_POSES poses; overlapping calls race).
    All arguments except beta, p0 and stream are CUDA tensors."""
    n = points.shape[0]
    m = poses.shape[0]
    _call("vd_score_poses_noalloc", C.c_void_p(points.data_ptr()), C.c_void_p(obs.data_ptr()),
          int(n), C.c_void_p(poses.data_ptr()), int(m), C.c_void_p(intrinsics.data_ptr()),
          float(beta), float(p0), C.c_void_p(energies.data_ptr()),
          stream if stream is not None else current_stream())
    return energies


def _tune_dict(t):
    return dict(k1_warps=t.k1_warps, score_threads=t.score_threads,
                score_blocks_per_sm=t.score_blocks_per_sm, k1_ms=list(t.k1_ms),
                score_ms=[list(r) for r in t.score_ms])


def vd_autotune(ctx):
    t = vd_tune()
    _call("vd_autotune", ctx, C.byref(t))
    return _tune_dict(t)


def vd_set_tune(ctx, k1_warps, score_blocks_per_sm, score_threads=256):
    t = vd_tune()
    t.k1_warps, t.score_blocks_per_sm = int(k1_warps), int(score_blocks_per_sm)
    t.score_threads = int(score_threads)
    _call("vd_set_tune", ctx, C.byref(t))


def vd_get_tune(ctx):
    t = vd_tune()
    _call("vd_get_tune", ctx, C.byref(t))
    return _tune_dict(t)


def vd_batch_create(windows, params=None, stream=None):
    """windows: list of (W, H, N, (fx, fy, cx, cy)); params: None, one
    vd_params for all, or a list with one per window."""
    n = len(windows)
    descs = (vd_window_desc * n)(*[vd_window_desc(int(W), int(H), int(N), *[float(v) for v in K])
                                   for (W, H, N, K) in windows])
    if params is None:
        pp, stride = None, 0
    elif isinstance(params, vd_params):
        pp, stride = C.byref(params), 0
    else:
        arr = (vd_params * n)(*params)
        pp, stride = arr, 1
    h = C.c_void_p()
    _call("vd_batch_create", n, descs, pp, stride,
          stream if stream is not None else current_stream(), C.byref(h))
    return h


def vd_batch_destroy(batch):
    _call("vd_batch_destroy", batch)


def vd_batch_window(batch, i):
    h = C.c_void_p()
    _call("vd_batch_window", batch, int(i), C.byref(h))
    return h


def vd_batch_run(batch, n_iters, flags=VD_BATCH_BOOTSTRAP, n_windows=None):
    """Returns the per-window degenerate-frame counts when n_windows is given."""
    deg = (C.c_int * n_windows)() if n_windows else None
    _call("vd_batch_run", batch, int(n_iters), int(flags), deg)
    return list(deg) if deg is not None else None


def vd_batch_get_stats(batch):
    st = vd_batch_stats()
    _call("vd_batch_get_stats", batch, C.byref(st))
    return dict(windows=st.windows, captures=st.captures, replays=st.replays,
                graph_nodes=st.graph_nodes, kernels_per_run=st.kernels_per_run)


# ------------------------------------------------------------------ pose covariance
def vd_pose_covariance(ctx, N, eps=1e-12):
    """Per frame t = 1..N: dict(mean 3x4, cov 6x6, n_samples, n_inliers,
    rounds, degenerate)."""
    arr = (vd_pose_cov * N)()
    _call("vd_pose_covariance", ctx, float(eps), C.cast(arr, C.c_void_p))
    return [dict(mean=np.array(r.mean[:]).reshape(3, 4), cov=np.array(r.cov[:]).reshape(6, 6),
                 n_samples=r.n_samples, n_inliers=r.n_inliers, rounds=r.rounds,
                 degenerate=bool(r.degenerate)) for r in arr]


def vd_get_frame_samples(ctx, t, S):
    """(poses S x 3 x 4, energies S) of frame t's last pose M-step."""
    poses = np.zeros((S, 3, 4), np.float64)
    energies = np.zeros(S, np.float64)
    _call("vd_get_frame_samples", ctx, int(t), poses.ctypes.data_as(C.c_void_p),
          energies.ctypes.data_as(C.c_void_p))
    return poses, energies


# ------------------------------------------------------------------ keyframe alignment
def vd_ka_align(depth1, depth2, K, T0, s0=1.0, conf2=None, c=0.01, fix_scale=False,
                max_iters=50, stream=None):
    """depth1, depth2 (and conf2): CUDA float32 tensors [H][W] of depth; K =
    (fx, fy, cx, cy); T0: 3x4 keyframe-2 -> keyframe-1.  Returns dict(T, s,
    cov 6x6, energy, iterations, n_valid)."""
    H, W = depth1.shape
    io = vd_ka()
    for i, v in enumerate(np.asarray(T0, np.float64).reshape(12)):
        io.pose[i] = float(v)
    io.s, io.cauchy_c = float(s0), float(c)
    io.fix_scale, io.max_iters = int(bool(fix_scale)), int(max_iters)
    k = np.ascontiguousarray(K, np.float64)
    _call("vd_ka_align", _dev(depth1), _dev(depth2), _dev(conf2) if conf2 is not None else None,
          int(W), int(H), k.ctypes.data_as(C.c_void_p), C.byref(io),
          stream if stream is not None else current_stream())
    return dict(T=np.array(io.pose[:]).reshape(3, 4), s=io.s, cov=np.array(io.cov[:]).reshape(6, 6),
                energy=io.energy, iterations=io.iterations, n_valid=io.n_valid)


# ------------------------------------------------------------------ VC score
def _vc_dict(s):
    n = s.n_frames
    return dict(n_frames=n, n_pixels=s.n_pixels, n_depth=s.n_depth,
                n_visible=list(s.n_visible[:n]), n_covered=list(s.n_covered[:n]),
                visibility=list(s.visibility[:n]), coverage=list(s.coverage[:n]),
                vc=list(s.vc[:n]))


def vd_vc_scores(ctx):
    """Visibility, coverage and VC of the reference depth in frames 1..N."""
    s = vd_vc()
    _call("vd_vc_scores", ctx, C.byref(s))
    return _vc_dict(s)


def vd_vc_pose(ctx, T):
    """The same in one frame of pose T (3x4, reference -> frame)."""
    t = np.ascontiguousarray(np.asarray(T, np.float64).reshape(12))
    s = vd_vc()
    _call("vd_vc_pose", ctx, t.ctypes.data_as(C.c_void_p), C.byref(s))
    return _vc_dict(s)


def vd_vc_stride(vc, tau_stride):
    a = np.ascontiguousarray(vc, np.float64)
    return int(load().vd_vc_stride(a.ctypes.data_as(C.c_void_p), int(a.size), float(tau_stride)))


def vd_vc_is_keyframe(vc, tau_keyframe):
    return bool(load().vd_vc_is_keyframe(float(vc), float(tau_keyframe)))


# ------------------------------------------------------------------ learned initialiser
VD_CNN_LAYERS = 6


def _dev(x):
    """Pointer of a CUDA tensor (the learned-initialiser calls take device memory)."""
    if not (_is_tensor(x) and x.is_cuda and x.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    return C.c_void_p(x.data_ptr())


def vd_cnn_create(n_flows, seed=0):
    h = C.c_void_p()
    _call("vd_cnn_create", int(n_flows), int(seed), C.byref(h))
    return h


def vd_check_bounded_wait(polls, stream=None):
    """Raises VoldorError with status VD_ERR_TIMEOUT: the bounded wait gave up."""
    _call("vd_check_bounded_wait", int(polls), stream)


VD_PROBE_FP32, VD_PROBE_MUFU = 0, 1


def vd_probe_pipe(kind, blocks, iters, stream=None):
    """Launch a pipe throughput probe (no synchronisation); returns the number
    of thread-level operations launched."""
    ops = C.c_double(0.0)
    _call("vd_probe_pipe", int(kind), int(blocks), int(iters), C.byref(ops),
          stream if stream is not None else current_stream())
    return ops.value


def vd_check_report():
    """Index-check record of the checked build (see voldor_em.h): dict with
    site, index, bound, count and checked (whether this library checks)."""
    out = (C.c_longlong * 5)()
    _call("vd_check_report", C.cast(out, C.c_void_p))
    return dict(site=out[0], index=out[1], bound=out[2], count=out[3], checked=bool(out[4]))


def vd_cnn_destroy(net):
    _call("vd_cnn_destroy", net)


def vd_cnn_layout(net):
    n = C.c_int(0)
    cin = (C.c_int * VD_CNN_LAYERS)()
    cout = (C.c_int * VD_CNN_LAYERS)()
    wo = (C.c_long * VD_CNN_LAYERS)()
    bo = (C.c_long * VD_CNN_LAYERS)()
    _call("vd_cnn_layout", net, C.byref(n), cin, cout, wo, bo)
    return dict(n_params=n.value, c_in=list(cin), c_out=list(cout), w_offset=list(wo),
                b_offset=list(bo))


def vd_cnn_get_params(net):
    out = np.zeros(vd_cnn_layout(net)["n_params"], np.float32)
    _call("vd_cnn_get_params", net, out.ctypes.data_as(C.c_void_p))
    return out


def vd_cnn_set_params(net, params):
    p = np.ascontiguousarray(params, np.float32)
    _call("vd_cnn_set_params", net, p.ctypes.data_as(C.c_void_p))


def vd_cnn_get_grads(net):
    out = np.zeros(vd_cnn_layout(net)["n_params"], np.float32)
    _call("vd_cnn_get_grads", net, out.ctypes.data_as(C.c_void_p))
    return out


def _geom(geom):
    """(K, T1) -> vd_cnn_geometry pointer (None: no geometry planes)."""
    if geom is None:
        return None
    K, T1 = geom
    g = vd_cnn_geometry(*[float(v) for v in K])
    for i, v in enumerate(np.asarray(T1, np.float64).reshape(12)):
        g.T1[i] = float(v)
    return C.byref(g)


def vd_cnn_forward(net, flow, rho_min, rho_max, rho_out=None, q_out=None, geom=None,
                   stream=None):
    """flow: CUDA float32 tensor [N][H][W][2]; geom: (K, T1) or None; outputs
    CUDA float32, rho [H][W] and q [N][H][W]."""
    H, W = flow.shape[1], flow.shape[2]
    _call("vd_cnn_forward", net, _dev(flow), int(W), int(H), _geom(geom), float(rho_min),
          float(rho_max),
          _dev(rho_out) if rho_out is not None else None,
          _dev(q_out) if q_out is not None else None,
          stream if stream is not None else current_stream())


def vd_cnn_get_activation(net, layer, W, H, channels):
    out = np.zeros((H, W, channels), np.float32)
    _call("vd_cnn_get_activation", net, int(layer), out.ctypes.data_as(C.c_void_p), int(W), int(H))
    return out


def vd_cnn_train_step(net, flow, rho_t, q_t, mask, rho_min, rho_max, w_q, lr, update=True,
                      geom=None, stream=None):
    """All arrays CUDA tensors ([N][H][W][2] flow, [H][W] rho target, [N][H][W]
    rigidness targets, [H][W] uint8 mask).  Returns the loss of the forward
    pass before the update."""
    H, W = flow.shape[1], flow.shape[2]
    loss = C.c_double(0.0)
    _call("vd_cnn_train_step", net, _dev(flow), int(W), int(H), _geom(geom), _dev(rho_t),
          _dev(q_t), _dev(mask), float(rho_min), float(rho_max), float(w_q), float(lr),
          1 if update else 0,
          C.byref(loss), stream if stream is not None else current_stream())
    return loss.value


def vd_eight_point(ctx):
    """The monocular bootstrap's pose of flow 1 (3x4), state unchanged."""
    T = np.zeros(12, np.float64)
    _call("vd_eight_point", ctx, T.ctypes.data_as(C.c_void_p))
    return T.reshape(3, 4)


def vd_bootstrap_learned(ctx, net):
    _call("vd_bootstrap_learned", ctx, net)


def vd_export_state(ctx):
    n = C.c_size_t(0)
    _call("vd_export_state", ctx, None, C.byref(n))
    blob = (C.c_char * n.value)()
    _call("vd_export_state", ctx, C.cast(blob, C.c_void_p), C.byref(n))
    return bytes(blob)


def vd_import_state(ctx, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _call("vd_import_state", ctx, C.cast(buf, C.c_void_p), len(blob))

"""The library's float64 device geometry, compiled for the host, against the
oracle and against closed forms (no GPU needed)."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import geometry, p3p

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hc():
    from paper_2104_06800_gb300.build import nvcc_path
    out = os.path.join(tempfile.mkdtemp(), "libvd_hostcheck.so")
    src = os.path.join(ROOT, "tests", "native", "vd_hostcheck.cu")
    # -ffp-contract=off: the host compiler must not fuse the error-free
    # transformations' products and sums (the device code spells out its
    # fused multiply-adds)
    cmd = [nvcc_path(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
           "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "paper_2104_06800_gb300", "csrc"), src, "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = C.CDLL(out)
    P = C.POINTER(C.c_double)
    lib.hc_p3p.argtypes = [P, P, P]
    lib.hc_p3p_df.argtypes = [P, P, P]
    lib.hc_real_roots.argtypes = [P, C.c_int, P]
    lib.hc_quartic_fast.argtypes = [P, P]
    for n in ("hc_se3_exp", "hc_se3_log"):
        getattr(lib, n).argtypes = [P, P]
    for n in ("hc_jacobi9", "hc_jacobi3"):
        getattr(lib, n).argtypes = [P, P, P]
    F = C.POINTER(C.c_float)
    lib.hc_em_project.argtypes = [F, F, C.c_int, C.c_int, C.c_float, P]
    lib.hc_em_inside.argtypes = [C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, C.c_int]
    lib.hc_em_tap.argtypes = [C.c_float, C.c_float, C.c_int, F]
    return lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def test_real_roots_of_products_and_random_polynomials(hc):
    rng = np.random.default_rng(0)
    out = np.zeros(4)
    for _ in range(300):
        r = np.sort(rng.uniform(-5, 5, size=4))
        c = np.polynomial.polynomial.polyfromroots(r) * rng.uniform(0.1, 10)
        n = hc.hc_real_roots(_p(c), 4, _p(out))
        assert n == 4 and np.allclose(out[:n], r, atol=1e-9)
    for _ in range(300):
        c = rng.normal(size=5)
        n = hc.hc_real_roots(_p(c), 4, _p(out))
        ref = np.roots(c[::-1])
        real = np.sort(ref[np.abs(ref.imag) < 1e-9].real)
        assert n == len(real) and np.allclose(out[:n], real, atol=1e-8)
    # degenerate leading coefficients fall back to lower degrees
    c = np.array([-6.0, 11.0, -6.0, 1.0, 0.0])
    assert hc.hc_real_roots(_p(c), 4, _p(out)) == 3 and np.allclose(out[:3], [1, 2, 3])
    c = np.array([2.0, 0.0, 1.0, 0.0, 0.0])      # no real root
    assert hc.hc_real_roots(_p(c), 4, _p(out)) == 0


def test_fast_quartic_roots_match_the_full_search(hc):
    """The P3P kernel's quartic roots (float32 split points, float64 Newton
    on the quartic's roots only) equal the product's roots to float64
    precision, and the full float64 search's on random quartics."""
    rng = np.random.default_rng(5)
    out, full = np.zeros(4), np.zeros(4)
    for _ in range(300):
        r = np.sort(rng.uniform(-5, 5, size=4))
        if np.min(np.diff(r)) < 1e-3:
            continue
        c = np.polynomial.polynomial.polyfromroots(r) * rng.uniform(0.1, 10)
        n = hc.hc_quartic_fast(_p(c), _p(out))
        assert n == 4 and np.allclose(out[:n], r, rtol=0, atol=1e-9)
    worst = 0.0
    for _ in range(500):
        c = rng.normal(size=5) * np.exp(rng.uniform(-3, 3, size=5))
        n = hc.hc_quartic_fast(_p(c), _p(out))
        nf = hc.hc_real_roots(_p(c), 4, _p(full))
        assert n == nf
        worst = max(worst, float(np.max(np.abs(out[:n] - full[:n]) / (1 + np.abs(full[:n])),
                                        initial=0.0)))
    assert worst < 1e-12


def _reproj(G, X, f):
    Y = X @ G[:, :3].T + G[:, 3]
    return np.abs(Y / np.linalg.norm(Y, axis=1, keepdims=True)
                  - f / np.linalg.norm(f, axis=1, keepdims=True)).max()


def test_p3p_matches_oracle_and_is_exact(hc):
    rng = np.random.default_rng(11)
    errs = []
    illcond = 0
    poses = np.zeros(48)
    for _ in range(300):
        R = geometry.so3_exp(rng.normal(size=3) * 0.5)
        X = rng.normal(size=(3, 3))
        tau = rng.normal(size=3)
        tau[2] += 5 - (X @ R.T + tau)[:, 2].min()
        Xc = X @ R.T + tau
        f = np.ascontiguousarray(Xc / Xc[:, 2:3])      # bearings as (x, y, 1)
        n = hc.hc_p3p(_p(f), _p(np.ascontiguousarray(X)), _p(poses))
        got = [poses[12 * k:12 * k + 12].reshape(3, 4) for k in range(n)]
        ref = p3p.solve(f, X)
        assert 1 <= n <= 4
        G = np.concatenate([R, tau[:, None]], 1)
        errs.append(min(np.abs(g - G).max() for g in got))
        # the same solution set as the oracle (up to order); on an
        # ill-conditioned quartic (clustered roots) the two roundings may
        # differ, then both must still reproject the three bearings
        if len(ref) == n:
            for r in ref:
                g = min(got, key=lambda g: np.abs(g - r).max())
                if np.abs(g - r).max() >= 1e-6:
                    illcond += 1
                    assert _reproj(g, X, f) < 1e-6 and _reproj(r, X, f) < 1e-6
        else:
            illcond += 1
    errs = np.array(errs)
    assert illcond <= 3
    assert np.percentile(errs, 90) < 1e-9 and errs.max() < 1e-5


def test_se3_maps_match_oracle(hc):
    rng = np.random.default_rng(5)
    T = np.zeros(12)
    xi2 = np.zeros(6)
    for _ in range(200):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        xi = np.concatenate([ax * rng.choice([1e-9, 1e-4, 0.3, 3.0]), rng.normal(size=3)])
        hc.hc_se3_exp(_p(xi), _p(T))
        assert np.allclose(T.reshape(3, 4), geometry.se3_exp(xi), atol=1e-13)
        hc.hc_se3_log(_p(T), _p(xi2))
        assert np.allclose(xi2, xi, atol=1e-9)


def test_jacobi_eigen_matches_numpy(hc):
    rng = np.random.default_rng(2)
    for n, fn in ((9, hc.hc_jacobi9), (3, hc.hc_jacobi3)):
        for _ in range(50):
            B = rng.normal(size=(n, n))
            A = B @ B.T
            w = np.zeros(n)
            V = np.zeros(n * n)
            a = np.ascontiguousarray(A.copy().ravel())
            fn(_p(a), _p(w), _p(V))
            V = V.reshape(n, n)
            assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), rtol=1e-10, atol=1e-10)
            assert np.allclose(A @ V, V * w, atol=1e-9)


def test_double_float_p3p_matches_the_oracle(hc):
    """The pose kernel's double-float P3P (vd_p3p_df.cuh, compiled for the
    host) returns the oracle's solutions of exact instances: the same count,
    every pose a solution of the minimal problem, the true pose among them to
    1e-7 on 98 % of the instances (ill-conditioned ones lose digits in any
    precision: the float64 solver's error there is up to ~4e-8, double-float
    carries ~5 bits fewer) and to 1e-5 on all."""
    rng = np.random.default_rng(12)
    poses = np.zeros(48)
    errs = []
    for _ in range(300):
        R = geometry.so3_exp(rng.normal(size=3) * 0.5)
        X = rng.normal(size=(3, 3)) * rng.uniform(0.5, 20)
        tau = rng.normal(size=3)
        tau[2] += 5 - (X @ R.T + tau)[:, 2].min()
        Xc = X @ R.T + tau
        f = np.ascontiguousarray(Xc / Xc[:, 2:3])
        n = hc.hc_p3p_df(_p(f), _p(np.ascontiguousarray(X)), _p(poses))
        got = [poses[12 * k:12 * k + 12].reshape(3, 4) for k in range(n)]
        assert n == len(p3p.solve(f, X))
        for G in got:
            assert _reproj(G, X, f) < 1e-6
        G0 = np.concatenate([R, tau[:, None]], 1)
        errs.append(min(np.abs(G - G0).max() for G in got))
    errs = np.array(errs)
    assert np.mean(errs < 1e-7) >= 0.98 and errs.max() < 1e-5
    assert np.median(errs) < 1e-11


# ------------------------------------------------ rigidness emission positions
def _df_pairs(a):
    """float64 values -> interleaved float32 (hi, lo) pairs."""
    a = np.asarray(a, np.float64).ravel()
    hi = a.astype(np.float32)
    lo = (a - hi.astype(np.float64)).astype(np.float32)
    return np.ascontiguousarray(np.stack([hi, lo], -1).ravel())


def _kdf(K):
    fx, fy, cx, cy = K
    return _df_pairs([fx, fy, cx, cy, 1.0 / fx, 1.0 / fy])


def _rows(K, G):
    """K [R | tau] as 12 float64 entries: the 3 x 3 part by rows, then the
    last column (the library's layout of a frame's pose rows)."""
    fx, fy, cx, cy = K
    KM = np.array([[fx, 0, cx], [0, fy, cy], [0, 0, 1.0]])
    A = KM @ G
    return np.concatenate([A[:, :3].ravel(), A[:, 3]])


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def test_emission_positions_match_the_float64_projection(hc):
    """Double-float projection and dehomogenisation against the oracle's
    float64 ones, within the bound that the replay harness allows them
    (`chained._df_proj_err`), and the camera-plane decision wherever z is
    not within 1e-10 of the plane."""
    import chained
    rng = np.random.default_rng(7)
    W, H = 1216, 368
    K = (720.0, 720.0, 607.5, 183.5)
    kdf = _kdf(K)
    out = np.zeros(2)
    worst = 0.0
    n_behind = 0
    for _ in range(40):
        xi = np.concatenate([rng.normal(0, 0.05, 3), rng.normal(0, 0.5, 3)])
        G = geometry.se3_exp(xi)[:3]
        M = _df_pairs(_rows(K, G))
        us = rng.integers(0, W, 50)
        vs = rng.integers(0, H, 50)
        cs = rng.uniform(0.0, 2.0, 50).astype(np.float32)
        r = geometry.rays(W, H, K)[vs, us]
        h = geometry.project_h(K, G, r, cs.astype(np.float64))
        x, y, front = geometry.dehom(h)
        ex, ey = chained._df_proj_err(h, geometry.project_h(K, np.abs(G), np.abs(r),
                                                            cs.astype(np.float64)))
        for i in range(50):
            f = hc.hc_em_project(_fp(M), _fp(kdf), int(us[i]), int(vs[i]), float(cs[i]), _p(out))
            if abs(h[i, 2] - geometry.Z_EPS) > 1e-10:
                assert bool(f) == bool(front[i])
            if f and front[i]:
                for e, ref, b in ((out[0], x[i], ex[i]), (out[1], y[i], ey[i])):
                    assert abs(e - ref) <= b, (e, ref, b)
                    worst = max(worst, abs(e - ref) / b)
            n_behind += int(not f)
    assert n_behind > 0          # the camera-plane branch was exercised
    assert worst < 0.5, worst


def test_emission_border_and_tap_decisions_are_exact(hc):
    """Border tests and bilinear taps decide on the exact value hi + lo."""
    W, H = 1216, 368
    tiny = np.float32(1e-5)
    ins = lambda xh, xl, yh, yl: hc.hc_em_inside(xh, xl, yh, yl, W, H)
    assert ins(W - 1, 0.0, 0.0, 0.0) == 1 and ins(0.0, 0.0, H - 1, 0.0) == 1
    assert ins(W - 1, tiny, 5.0, 0.0) == 0 and ins(W - 1, -tiny, 5.0, 0.0) == 1
    assert ins(0.0, -tiny, 5.0, 0.0) == 0 and ins(0.0, tiny, 5.0, 0.0) == 1
    assert ins(5.0, 0.0, H - 1, tiny) == 0 and ins(5.0, 0.0, 0.0, -tiny) == 0
    w = np.zeros(1, np.float32)
    # an integer hi with a negative lo is below the integer
    assert hc.hc_em_tap(40.0, -tiny, W, _fp(w)) == 39 and abs(w[0] - (1 - tiny)) < 1e-7
    assert hc.hc_em_tap(40.0, tiny, W, _fp(w)) == 40 and abs(w[0] - tiny) < 1e-7
    assert hc.hc_em_tap(0.0, 0.0, W, _fp(w)) == 0 and w[0] == 0.0
    # the last column is reached from the tap before it with weight 1
    assert hc.hc_em_tap(W - 1, 0.0, W, _fp(w)) == W - 2 and w[0] == 1.0
    assert hc.hc_em_tap(W - 1, -tiny, W, _fp(w)) == W - 2 and abs(w[0] - (1 - tiny)) < 1e-7
    rng = np.random.default_rng(3)
    for _ in range(2000):
        x = rng.uniform(0, W - 1)
        hi = np.float32(x)
        lo = np.float32(x - np.float64(hi))
        x0 = hc.hc_em_tap(hi, lo, W, _fp(w))
        e = np.float64(hi) + np.float64(lo)
        ref0 = min(int(np.floor(e)), W - 2)
        assert x0 == ref0 and abs(w[0] - (e - ref0)) < 1e-6

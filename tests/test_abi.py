"""The shared library builds, loads, and exports every symbol of the header.

No compute calls here (no GPU on this host)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(vd_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2104_06800_gb300 import build, voldor
    build.build()
    return voldor.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2104_06800_gb300 import voldor
    for n in _declared():
        assert n in voldor._SIGS or n in ("vd_status_str", "vd_last_error"), n
        assert hasattr(voldor, n) or n in ("vd_status_str", "vd_last_error"), n


def test_host_only_calls(lib):
    from paper_2104_06800_gb300 import voldor as V
    p = V.vd_params_default()
    assert p.n_hyp == 64 and abs(p.fisk_alpha0 - 0.5) < 1e-7 and p.sample_share == 1
    assert lib.vd_status_str(V.VD_ERR_STATE) == b"call out of order"
    assert lib.vd_params_default(None) == V.VD_ERR_ARG
    # argument validation happens before any CUDA call
    h = V.C.c_void_p()
    bad = V.vd_window_desc(1, 10, 3, 100.0, 100.0, 0.0, 0.0)
    assert lib.vd_create(V.C.byref(bad), None, None, V.C.byref(h)) == V.VD_ERR_ARG
    bad = V.vd_window_desc(10, 10, 9, 100.0, 100.0, 0.0, 0.0)
    assert lib.vd_create(V.C.byref(bad), None, None, V.C.byref(h)) == V.VD_ERR_ARG
    good = V.vd_window_desc(10, 10, 3, 100.0, 100.0, 0.0, 0.0)
    pp = V.vd_params_default(rho_min=1.0, rho_max=0.5)
    assert lib.vd_create(V.C.byref(good), V.C.byref(pp), None, V.C.byref(h)) == V.VD_ERR_ARG
    assert lib.vd_run_em(None, 1, None) == V.VD_ERR_ARG


def test_struct_layouts_match_the_header():
    """ctypes structures mirror the C declarations field by field."""
    from paper_2104_06800_gb300 import voldor as V
    src = open(os.path.join(ROOT, "include", "voldor_em.h")).read()
    body = src[src.index("typedef struct {\n  float fisk_alpha0"):]
    body = body[:body.index("} vd_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b([a-z_0-9]+)\s*[,;]", body.replace("typedef struct {", ""))
    assert [f for f, _ in V.vd_params._fields_] == fields


def _struct_fields(src, closing):
    body = src[:src.index(closing)]
    body = body[body.rindex("typedef struct {"):]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S).replace("typedef struct {", "")
    return re.findall(r"\b([a-z_0-9]+)\s*(?:\[[A-Z0-9_]+\])*\s*[,;]", body)


def test_tune_and_batch_structs_match_the_header():
    from paper_2104_06800_gb300 import voldor as V
    src = open(os.path.join(ROOT, "include", "voldor_em.h")).read()
    assert [f for f, _ in V.vd_tune._fields_] == _struct_fields(src, "} vd_tune;")
    assert [f for f, _ in V.vd_batch_stats._fields_] == _struct_fields(src, "} vd_batch_stats;")
    assert V.VD_BATCH_BOOTSTRAP == 1 and V.VD_BATCH_AUTOTUNE == 2


def test_vc_struct_and_host_rules(lib):
    """The VC result structure mirrors the header; the stride and keyframe
    rules run on the host and agree with the oracle's."""
    from paper_2104_06800_gb300 import voldor as V
    from oracle import vc as ovc
    src = open(os.path.join(ROOT, "include", "voldor_em.h")).read()
    assert [f for f, _ in V.vd_vc._fields_] == _struct_fields(src, "} vd_vc;")
    assert "#define VD_VC_MAX_FRAMES 8" in src and V.VD_VC_MAX_FRAMES == 8
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = int(rng.integers(1, 9))
        vc = rng.uniform(0.3, 1.0, n)
        tau = float(rng.uniform(0.3, 1.0))
        assert V.vd_vc_stride(vc, tau) == ovc.stride(list(vc), tau)
        assert V.vd_vc_is_keyframe(vc[0], tau) == ovc.is_keyframe(vc[0], tau)
    assert lib.vd_vc_stride(None, 3, 0.5) == 0
    s = V.vd_vc()
    assert lib.vd_vc_scores(None, V.C.byref(s)) == V.VD_ERR_ARG
    assert lib.vd_vc_pose(None, None, V.C.byref(s)) == V.VD_ERR_ARG


def test_pose_cov_struct_and_argument_checks(lib):
    from paper_2104_06800_gb300 import voldor as V
    src = open(os.path.join(ROOT, "include", "voldor_em.h")).read()
    assert [f for f, _ in V.vd_pose_cov._fields_] == _struct_fields(src, "} vd_pose_cov;")
    out = (V.vd_pose_cov * 1)()
    assert lib.vd_pose_covariance(None, 1e-12, out) == V.VD_ERR_ARG
    assert lib.vd_get_frame_samples(None, 1, None, None) == V.VD_ERR_ARG


def test_ka_struct_and_argument_checks(lib):
    from paper_2104_06800_gb300 import voldor as V
    src = open(os.path.join(ROOT, "include", "voldor_em.h")).read()
    assert [f for f, _ in V.vd_ka._fields_] == _struct_fields(src, "} vd_ka;")
    io = V.vd_ka()
    io.s, io.cauchy_c, io.max_iters = 1.0, 0.01, 10
    k = (V.C.c_double * 4)(100.0, 100.0, 5.0, 5.0)
    assert lib.vd_ka_align(None, None, None, 10, 10, k, V.C.byref(io), None) == V.VD_ERR_ARG
    io.cauchy_c = 0.0
    p = V.C.c_void_p(16)   # never dereferenced: the arguments are checked first
    assert lib.vd_ka_align(p, p, None, 10, 10, k, V.C.byref(io), None) == V.VD_ERR_ARG


def test_batch_and_tune_argument_checks(lib):
    """Argument validation of the batch and tuning calls needs no GPU."""
    from paper_2104_06800_gb300 import voldor as V
    h = V.C.c_void_p()
    d = (V.vd_window_desc * 1)(V.vd_window_desc(10, 10, 3, 100.0, 100.0, 5.0, 5.0))
    assert lib.vd_batch_create(0, d, None, 0, None, V.C.byref(h)) == V.VD_ERR_ARG
    assert lib.vd_batch_create(1, None, None, 0, None, V.C.byref(h)) == V.VD_ERR_ARG
    assert lib.vd_batch_create(1, d, None, 2, None, V.C.byref(h)) == V.VD_ERR_ARG
    assert lib.vd_batch_run(None, 1, V.VD_BATCH_BOOTSTRAP, None) == V.VD_ERR_ARG
    assert lib.vd_batch_window(None, 0, V.C.byref(h)) == V.VD_ERR_ARG
    assert lib.vd_batch_destroy(None) == V.VD_ERR_ARG
    t = V.vd_tune()
    assert lib.vd_set_tune(None, V.C.byref(t)) == V.VD_ERR_ARG
    assert lib.vd_autotune(None, None) == V.VD_ERR_ARG


def test_header_is_plain_c(tmp_path):
    """include/voldor_em.h compiles as C99 with warnings as errors (a C ABI)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "voldor_em.h"\n'
                   "int main(void) { vd_params p; vd_vc v; vd_pose_cov c; vd_ka k;\n"
                   "  (void)v; (void)c; (void)k; return vd_params_default(&p) == VD_OK ? 0 : 1; }\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o",
                        str(tmp_path / "use.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_checked_build_compiles_and_exports_every_symbol():
    """The index-checking build (-DVD_CHECKED) of the same sources."""
    import ctypes as C
    from paper_2104_06800_gb300 import build
    path = build.build(checked=True)
    assert path.endswith("libvoldor_em_checked.so")
    lib = C.CDLL(path)
    for n in sorted(_declared()):
        assert hasattr(lib, n), n

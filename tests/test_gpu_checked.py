"""The index-checking build (-DVD_CHECKED, the stand-in for a memory
checker): every index the kernels form from data stays inside its buffer on
the workloads' windows.  The checked library runs in a child process (the
test process holds the regular one): a monocular driving window (bootstrap
and 8 iterations at K = 128), a stereo window, a batch of RGB-D windows of
uneven size and N, the VC score, the pose covariance and the keyframe
alignment; then vd_check_report must show the checked build and no index
out of range."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import synth
from paper_2104_06800_gb300 import build, voldor as V
V._lib = V.load(build.build(checked=True))
from gpu_common import params_for
def ctx_of(w):
    c = V.vd_create(w.W, w.H, w.N, w.intrinsics, V.vd_params_default(**params_for(w)))
    for t in range(1, w.N + 1):
        V.vd_push_flow(c, t, w.flow[t - 1])
    if w.stereo_disp is not None:
        V.vd_push_stereo_prior(c, w.stereo_disp, w.stereo_baseline)
    elif w.depth_prior is not None:
        V.vd_push_depth_prior(c, w.depth_prior)
    return c
out = {}
w = synth.make_window("driving1216_kerb", 2000, size=(608, 184))
c = ctx_of(w)
V.vd_bootstrap(c); V.vd_run_em(c, 8)
V.vd_vc_scores(c); V.vd_pose_covariance(c, w.N, 1e-12)
V.vd_destroy(c)
out["driving"] = V.vd_check_report()
c = ctx_of(synth.make_window("boxes640_stereo", 3, size=(320, 240), N=4))
V.vd_bootstrap(c); V.vd_run_em(c, 3); V.vd_destroy(c)
out["stereo"] = V.vd_check_report()
ws = [synth.make_window("rgbd_batch", 5400 + i, size=sz, N=n)
      for i, (sz, n) in enumerate([((96, 72), 3), ((320, 240), 8)])]
b = V.vd_batch_create([(x.W, x.H, x.N, x.intrinsics) for x in ws],
                      [V.vd_params_default(**params_for(x)) for x in ws])
for i, x in enumerate(ws):
    cc = V.vd_batch_window(b, i)
    for t in range(1, x.N + 1):
        V.vd_push_flow(cc, t, x.flow[t - 1])
    V.vd_push_depth_prior(cc, x.depth_prior)
V.vd_batch_run(b, 3, V.VD_BATCH_BOOTSTRAP)
V.vd_batch_destroy(b)
out["batch"] = V.vd_check_report()
import torch
Z0, Zt, T, K = synth.keyframe_pair("driving1216", 2000, 2, size=(304, 92))
dev = torch.device("cuda")
V.vd_ka_align(torch.from_numpy(Z0).to(dev), torch.from_numpy(Zt).to(dev), K, T, max_iters=5)
out["ka"] = V.vd_check_report()
print(json.dumps(out))
"""


def test_no_index_leaves_its_buffer_in_the_checked_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    print(rep)
    for name, x in rep.items():
        assert x["checked"], name
        assert x["count"] == 0, (name, x)

#!/usr/bin/env python
"""Throughput of the dense-indirect EM (VOLDOR+, Sec. III-A) on one GPU per rank.

One step = a batch of --batch (default 8) whole windows of EM on the
KITTI-like driving workload (1216 x 368, N = 6 flows, K = 128 hypotheses,
8 EM iterations, S = 64 P3P samples per frame): per window the monocular
bootstrap plus 8 iterations of depth M-step, rigidness E-step and pose
M-step, all windows in one CUDA-graph launch (vd_batch_run).  Inputs are
synthetic (synth.make_window("driving1216_kerb", ...): road, facades, car
boxes at the kerbs, 1-1.5 m per frame) and resident in HBM; L2 is flushed
before every timed step.

value  = pixel*frame*iterations per second over all ranks (W*H*N*8 per window)
single_window = the same for one window at a time (vd_bootstrap + vd_run_em),
         with the per-stage breakdown.
e2e    = the batched metric through the C ABI with host buffers: flows pushed
         from pinned host memory, inverse depth and poses read back, every step.
roofline = the depth-sampling kernel (the dominant kernel), FP32-issue bound:
         algorithmic FP32 operations per launch (counted below) over its
         CUDA-event time in the single-window run, against the FFMA
         throughput measured on the same GPU by the library's probe.
configs = the other workloads on one GPU: the small two-plane window, the
         stereo 640 x 480 window, the 64-window RGB-D batch (plain vs batched),
         and plain vs learned-initialised EM at equal accuracy.
cpu_baseline = the float64 oracle on the host: one iteration of the whole
         window over every core (row bands in spawned processes), one
         iteration of a crop on one core, and the small workload in full.

--impl reference times the oracle (the CPU definition of the method) instead:
every step one iteration of the whole window over every host core.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

# the float64 oracle (cpu_baseline, --impl reference) runs on one host core:
# no BLAS thread pool (set before numpy loads its BLAS)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EM pixel\u00b7frame\u00b7iters/s and windows/s at 1216x368 N=6; plain vs learned-init at \u22641% err"
UNIT = "pixel*frame*iter/s"
WORK = dict(name="driving1216_kerb", W=1216, H=368, N=6, iters=8, K=128, S=64, seed=2000)

# Algorithmic FP32 work of one hypothesis evaluation against one flow term
# (Eq. 5 with the beta = 2 closed form), counted operation by operation:
#   candidate projection hx, hy, hz = A + c B            3 FFMA
#   x = hx / hz, y = hy / hz (1 / hz on the MUFU)        2 FMUL
#   residual F - (x - x_prev), both coordinates          4 FADD
#   r^2                                                  1 FMUL + 1 FFMA
#   s = 1 + r^2 / alpha^2, y = c0 s^2                    1 FFMA + 2 FMUL
#   log(1 + y) (log2 on the MUFU)                        1 FADD
#   q_t-weighted sum                                     1 FFMA
#   camera-plane test                                    1 FSETP
# = 17 for X_1, read at the pixel itself.  A gathered flow (t >= 2) adds the
# inside-image test (4 FSETP), the tap position and weights (2 floor,
# 2 FADD) and the bilinear sample (2 x (2 FADD + 2 FFMA) per row pair, then
# 2 FADD + 2 FFMA) = 20: 37.  MUFU: one reciprocal and one log2 per term.
FP32_T1, FP32_TN, MUFU_PER_EVAL = 17, 37, 2
# One root against one rigid pixel in the pose scoring (same closed form):
# projection 9 FFMA, 2 FMUL, residual 2 FADD, r^2 2, s and y 3, log 1 FADD,
# weighted sum 1 FFMA, camera-plane test 1 FSETP = 21 FP32 + 2 MUFU.
FP32_SCORE, MUFU_SCORE = 21, 2
# DRAM bytes (read + write) per launch of k_depth_sample_q on this workload,
# from one ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum, one launch on the kerb-side driving window); re-measure
# when it changes.
K1_TRAFFIC_BYTES = 34.03e6
SM_MAX_MHZ = 2070.0


def measure_peaks(V, stream, sms):
    """FP32 FFMA and MUFU throughput of this GPU, measured with the
    library's probes (independent chains, 8 blocks of 256 threads per SM):
    thread-level operations per second, best of five CUDA-event timings of
    launches of a few ms."""
    import torch
    sptr = V.C.c_void_p(stream.cuda_stream)
    out = {}
    for name, kind, iters in (("fp32_ffma_per_s", V.VD_PROBE_FP32, 4000),
                              ("mufu_per_s", V.VD_PROBE_MUFU, 500)):
        blocks = 8 * sms
        for _ in range(2):
            V.vd_probe_pipe(kind, blocks, iters, sptr)
        best = 0.0
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ops = V.vd_probe_pipe(kind, blocks, iters, sptr)
            e1.record(stream)
            e1.synchronize()
            best = max(best, ops / (e0.elapsed_time(e1) / 1e3))
        out[name] = best
    out["fp32_per_sm_per_clk_at_max"] = round(out["fp32_ffma_per_s"] / (sms * SM_MAX_MHZ * 1e6), 2)
    out["mufu_per_sm_per_clk_at_max"] = round(out["mufu_per_s"] / (sms * SM_MAX_MHZ * 1e6), 2)
    out["sms"] = sms
    out["how"] = ("vd_probe_pipe: 8 blocks x 256 threads per SM, 8 independent chains per "
                  "thread of FFMA (4000 x 128 each) or MUFU log2 (500 x 128 each); best of 5 "
                  "CUDA-event timings")
    return out


def alu_roofline(kernel, evals, fp32_per_eval, mufu_per_eval, launch_ms, peaks, traffic, how):
    """Roofline entry of an FP32-issue-bound kernel: algorithmic FP32
    operations per launch over its CUDA-event time, against the measured
    FFMA throughput (the MUFU time is reported beside it)."""
    fp32 = evals * fp32_per_eval
    achieved = fp32 / (launch_ms / 1e3) / 1e12
    peak = peaks["fp32_ffma_per_s"] / 1e12
    t_fp32 = fp32 / peaks["fp32_ffma_per_s"]
    t_mufu = evals * mufu_per_eval / peaks["mufu_per_s"]
    return {"bound": "alu", "kernel": kernel, "achieved": round(achieved, 3),
            "peak": round(peak, 3), "unit": "TFP32-inst/s", "frac": round(achieved / peak, 4),
            "traffic": traffic, "traffic_unit": "B per launch", "launch_ms": round(launch_ms, 4),
            "evals_per_launch": int(evals), "fp32_per_eval": fp32_per_eval,
            "mufu_per_eval": mufu_per_eval,
            "roofline_ms": {"fp32": round(1e3 * t_fp32, 4), "mufu": round(1e3 * t_mufu, 4)},
            "peak_basis": "measured FFMA throughput of this GPU (vd_probe_pipe, of measured)",
            "measured_in": how}


def workload_config(nb, world):
    """The headline workload (both arms report it)."""
    return {"workload": f"{WORK['name']} x {nb} windows per step: 1216x368, N=6 flows, "
                        "K=128 hypotheses, 8 EM iterations, S=64 P3P samples, "
                        "monocular bootstrap; all windows in one CUDA-graph launch",
            "windows_per_step_per_gpu": nb,
            "l2": "flushed (256 MB write) before every timed step",
            "parallelism": f"replicas x{world}"}


def fp32_per_pixel_hyp(N):
    return FP32_T1 + (N - 1) * FP32_TN


def fp32_per_eval(N):
    """Mean algorithmic FP32 operations per (pixel, flow, hypothesis)."""
    return fp32_per_pixel_hyp(N) / N


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads' measurements (small, stereo, RGB-D batch)")
    ap.add_argument("--batch", type=int, default=8, help="windows per step (one graph launch)")
    ap.add_argument("--workload", default="driving1216_kerb",
                    choices=["driving1216_kerb", "driving1216", "rgbd_batch64", "ka1216"],
                    help="rgbd_batch64: 64 RGB-D windows of uneven size and N, plain vs "
                         "batched; ka1216: keyframe alignment of two 1216x368 depth maps")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch shapes (no vd_autotune; for profiling)")
    ap.add_argument("--phase", default="both", choices=["both", "single", "batch"],
                    help="single: only the one-window run (for profiling); batch: skip it")
    ap.add_argument("--hierarchical", action="store_true",
                    help="hierarchical depth propagation (coarse cells of 4 px, windows of "
                         "32 px) instead of full chains")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        if not shutil.which("nvidia-smi"):
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen(
            ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ distributed
def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        # one process per GPU over NCCL; gloo where there is no GPU (host tests)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x, device):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job(pg, world, units_per_rank, local_ms, device):
    """(slowest rank's time in ms, whole-job rate): every rank processes
    units_per_rank units of its own (weak scaling, no data-path exchange);
    the job ends when the slowest rank does."""
    ms = max_over_ranks(pg, local_ms, device)
    return ms, units_per_rank * world / (ms / 1e3)


def rank_window_seeds(seed, rank, nb):
    """Seeds of the nb windows rank `rank` runs: the first is seed + rank (the
    single-window run's), the others distinct across ranks and windows."""
    return [seed + rank] + [seed + 100 * (rank + 1) + i for i in range(1, nb)]


# ------------------------------------------------------------------ oracle timing
_ORACLE_WINDOW = []


def _oracle_window():
    import synth
    if not _ORACLE_WINDOW:
        _ORACLE_WINDOW.append(synth.make_window(WORK["name"], WORK["seed"]))
    return _ORACLE_WINDOW[0]


def _oracle_band(args):
    """One EM iteration of the float64 oracle on a sub-window (run in a
    worker process): returns (pixel*frames, seconds)."""
    flow, K, rho, G, prm, u0, v0 = args
    from oracle import em as oem
    from oracle import model as omodel
    N, ch, cw = flow.shape[0], flow.shape[1], flow.shape[2]
    fx, fy, cx, cy = K
    P = omodel.Problem(cw, ch, N, (fx, fy, cx - u0, cy - v0), np.ascontiguousarray(flow))
    p = omodel.Params(**prm)
    S = omodel.State(rho=rho, q=np.ones((N, ch, cw), np.float32),
                     qhat=np.zeros((ch, cw), np.float32), G=G)
    t0 = time.perf_counter()
    oem.iteration(P, S, 0, p)
    return cw * ch * N, time.perf_counter() - t0


def _oracle_inputs(u0, v0, cw, ch):
    """The oracle's start on a cw x ch sub-window at (u0, v0): the scene's
    true inverse depth (in |tau_1| units) and poses, rigidness 1 -- not a
    mid-EM state, and no bootstrap (the oracle's per-iteration work does not
    depend on the state: it evaluates every candidate in full)."""
    win = _oracle_window()
    pr = win.params
    prm = dict(fisk_alpha0=pr["fisk_alpha0"], rho_min=pr["rho_min"], rho_max=pr["rho_max"],
               n_hyp=WORK["K"], n_pose_samples=WORK["S"])
    s = pr["scale"]
    G = win.G.copy()
    G[:, :, 3] /= s
    rho = (s / win.depth0[v0:v0 + ch, u0:u0 + cw]).astype(np.float32)
    flow = win.flow[:, v0:v0 + ch, u0:u0 + cw]
    return flow, win.intrinsics, rho, G, prm, u0, v0


def oracle_sample(cw=WORK["W"] // 2, ch=WORK["H"] // 2):
    """Time the float64 oracle on one host core: one EM iteration (depth
    M-step, E-step, pose M-step of every frame) on the centred cw x ch crop
    of the workload's first window (608 x 184 = 1/4 of its pixels by
    default; same N, K, S), from the start of _oracle_inputs."""
    u0, v0 = (WORK["W"] - cw) // 2, (WORK["H"] - ch) // 2
    units, dt = _oracle_band(_oracle_inputs(u0, v0, cw, ch))
    return units / dt, dt, (f"one EM iteration (no bootstrap; start: true depth and poses, "
                            f"rigidness 1) of the float64 oracle on a centred {cw}x{ch} crop of "
                            f"{WORK['name']} seed {WORK['seed']} (N={WORK['N']}, K={WORK['K']}, "
                            f"S={WORK['S']}) on one core, {dt:.1f} s")


def oracle_all_cores():
    """The oracle on every host core: the whole 1216 x 368 window cut into
    one row band per core, each band one EM iteration in its own process
    (spawned: this process has used the GPU), from the start of
    _oracle_inputs.  Bands run the method on their own pixels (a pose step
    scores the band's rigid pixels), so the work is the window's, split.
    Wall time from the pool's first task to its last result."""
    import concurrent.futures
    import multiprocessing
    ncores = os.cpu_count() or 1
    H, W = WORK["H"], WORK["W"]
    edges = np.linspace(0, H, ncores + 1).astype(int)
    tasks = [_oracle_inputs(0, int(edges[i]), W, int(edges[i + 1] - edges[i]))
             for i in range(ncores) if edges[i + 1] > edges[i]]
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=len(tasks), mp_context=ctx) as ex:
        list(ex.map(_oracle_warm, range(len(tasks))))      # imports in every worker
        t0 = time.perf_counter()
        res = list(ex.map(_oracle_band, tasks))
        dt = time.perf_counter() - t0
    units = sum(r[0] for r in res)
    return units / dt, dt, len(tasks), (
        f"one EM iteration (no bootstrap; start: true depth and poses, rigidness 1) of the "
        f"float64 oracle on the whole {W}x{H} window of {WORK['name']} seed {WORK['seed']} "
        f"(N={WORK['N']}, K={WORK['K']}, S={WORK['S']}), {len(tasks)} row bands in {len(tasks)} "
        f"processes, {dt:.1f} s wall")


def _oracle_warm(_):
    from oracle import em  # noqa: F401
    return os.getpid()


def oracle_small_full():
    """The oracle's whole run of the small workload (planes160 seed 0:
    160 x 120, N = 3, K = 64, monocular bootstrap and 3 EM iterations) on one
    core: windows/s and pixel*frame*iter/s."""
    import synth
    from oracle import em as oem
    from oracle import model as omodel
    win = synth.make_window("planes160", 0)
    pr = win.params
    P = omodel.problem_from_window(win)
    p = omodel.Params(fisk_alpha0=pr["fisk_alpha0"], rho_min=pr["rho_min"],
                      rho_max=pr["rho_max"], n_hyp=pr["n_hyp"])
    t0 = time.perf_counter()
    oem.run(P, p, pr["n_iters"])
    dt = time.perf_counter() - t0
    return {"windows_per_s": round(1.0 / dt, 5),
            "value": round(win.W * win.H * win.N * pr["n_iters"] / dt, 1), "unit": UNIT,
            "cores": 1, "seconds": round(dt, 2),
            "sample": "planes160 seed 0 in full: monocular bootstrap + 3 EM iterations, K=64"}


def host_cpu():
    """The host the oracle ran on: its CPU model (or part number) and core count."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                k, _, v = ln.partition(":")
                if k.strip() in ("model name", "Model", "CPU part") and v.strip():
                    model = v.strip()
                    if k.strip() != "CPU part":
                        break
    except OSError:
        pass
    import platform
    return {"model": model or platform.processor() or platform.machine(),
            "machine": platform.machine(), "nproc": os.cpu_count()}


# ------------------------------------------------------------------ our arm
def _timed(stream, flush, fn, steps):
    """CUDA-event time of `steps` calls of fn on `stream`, L2 flushed before each."""
    import torch
    times = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def run_ours(args, rank, world, local, pg):
    import torch
    from paper_2104_06800_gb300 import build as B
    from paper_2104_06800_gb300 import voldor as V
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    V.load()
    stream = torch.cuda.current_stream(dev)
    sptr = V.C.c_void_p(stream.cuda_stream)
    win = synth.make_window(WORK["name"], WORK["seed"] + rank)
    pr = win.params
    params = V.vd_params_default(fisk_alpha0=pr["fisk_alpha0"], rho_min=pr["rho_min"],
                                 rho_max=pr["rho_max"], n_hyp=WORK["K"],
                                 n_pose_samples=WORK["S"], seed=WORK["seed"] + rank,
                                 hierarchical=1 if args.hierarchical else 0)
    W, H, N, iters = win.W, win.H, win.N, WORK["iters"]
    units_per_window = W * H * N * iters
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # ---- one window at a time (latency, stage breakdown, kernel roofline)
    if args.phase == "batch":
        return run_batch(args, rank, world, local, pg, V, synth, win, params, sptr, stream, flush,
                         dev, None, None, None)
    ctx = V.vd_create(W, H, N, win.intrinsics, params, sptr)
    flows_dev = torch.from_numpy(win.flow).to(dev)
    for t in range(1, N + 1):
        V.vd_push_flow(ctx, t, flows_dev[t - 1])
    tune = V.vd_get_tune(ctx) if args.no_tune else V.vd_autotune(ctx)

    def step1():
        V.vd_bootstrap(ctx)
        V.vd_run_em(ctx, iters, stats=False)

    for _ in range(args.warmup):
        step1()
    torch.cuda.synchronize()
    V.vd_profile_enable(ctx, True)
    t1 = _timed(stream, flush, step1, args.steps)
    torch.cuda.synchronize()
    prof = V.vd_get_profile(ctx)
    V.vd_profile_enable(ctx, False)
    single_ms = statistics.median(t1)
    smp = prof["depth_sample"]
    launch_ms = smp["ms"] / max(smp["calls"], 1)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measure_peaks(V, stream, sms)
    roofline = alu_roofline("k_depth_sample_q", W * H * N * WORK["K"], fp32_per_eval(N),
                            MUFU_PER_EVAL, launch_ms, peaks, K1_TRAFFIC_BYTES,
                            "single-window run, kernel timed alone (CUDA events per stage)")
    roofline["peaks_measured"] = peaks
    # the dense pose scoring (K5, Eq. 7): every (rigid pixel, root) pair of
    # the timed steps, counted by the device, over the stage's event time
    sc = prof["pose_score"]
    roofline_score = alu_roofline("k_pose_score", prof["score_evals"] / max(sc["calls"], 1),
                                  FP32_SCORE, MUFU_SCORE, sc["ms"] / max(sc["calls"], 1), peaks,
                                  None, "single-window run, kernel timed alone (CUDA events "
                                  "per stage); evals = rigid pixels x roots of each launch")
    stages = {k: round(v["ms"] / args.steps, 4) for k, v in prof.items() if isinstance(v, dict)}
    # the stride / keyframe score of the window just estimated (VC, Eq. 8):
    # the call's time including its counter read-back, median of 20
    vc_res = V.vd_vc_scores(ctx)
    vc_ms = []
    for _ in range(20):
        t0 = time.perf_counter()
        V.vd_vc_scores(ctx)
        vc_ms.append(1e3 * (time.perf_counter() - t0))
    vc_line = {"ms_per_call": round(statistics.median(vc_ms), 4),
               "visibility": [round(x, 4) for x in vc_res["visibility"]],
               "coverage": [round(x, 4) for x in vc_res["coverage"]],
               "vc": [round(x, 4) for x in vc_res["vc"]],
               "stride_at_tau_0.7": V.vd_vc_stride(vc_res["vc"], 0.7)}
    # the pose covariance of every frame (Sec. III-A): median call time of 10
    pc = V.vd_pose_covariance(ctx, N, 1e-12)
    pc_ms = []
    for _ in range(10):
        t0 = time.perf_counter()
        V.vd_pose_covariance(ctx, N, 1e-12)
        pc_ms.append(1e3 * (time.perf_counter() - t0))
    pc_line = {"ms_per_call": round(statistics.median(pc_ms), 4),
               "n_inliers": [r["n_inliers"] for r in pc],
               "rounds": [r["rounds"] for r in pc],
               "sd_rot_rad": [round(float(np.sqrt(np.diag(r["cov"])[:3].mean())), 6) for r in pc],
               "degenerate": [r["degenerate"] for r in pc]}
    single = {"windows_per_s": round(1e3 / single_ms, 3), "ms_per_window": round(single_ms, 3),
              "value": round(units_per_window / (single_ms / 1e3), 1),
              "gpu_launches_per_window": int(prof["total_launches"] / args.steps),
              "vc_scores": vc_line, "pose_covariance": pc_line,
              "stage_ms_per_window": stages, "tune": tune,
              "roofline_pose_score": roofline_score}
    V.vd_destroy(ctx)
    if args.phase == "single":
        return {"metric": METRIC, "value": single["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(single_ms, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "phase": "single",
                "config": {"workload": f"{WORK['name']}: one window per step",
                           "propagation": "hierarchical (cells 4, windows 32)"
                           if args.hierarchical else "full chains"},
                "single_window": single, "roofline": roofline,
                "gpu_launches": int(prof["total_launches"])}
    return run_batch(args, rank, world, local, pg, V, synth, win, params, sptr, stream, flush, dev,
                     single, roofline, stages)


def run_batch(args, rank, world, local, pg, V, synth, win, params, sptr, stream, flush, dev,
              single, roofline, stages):
    import torch
    W, H, N, iters = win.W, win.H, win.N, WORK["iters"]
    units_per_window = W * H * N * iters
    # ---- a batch of windows in one graph launch (the headline throughput)
    nb = max(1, args.batch)
    seeds = rank_window_seeds(WORK["seed"], rank, nb)
    bw = [win] + make_windows([(WORK["name"], sd, {}) for sd in seeds[1:]])
    b = V.vd_batch_create([(w.W, w.H, w.N, w.intrinsics) for w in bw], params, sptr)
    for i, w in enumerate(bw):
        fl = torch.from_numpy(w.flow).to(dev)
        for t in range(1, N + 1):
            V.vd_push_flow(V.vd_batch_window(b, i), t, fl[t - 1])
    V.vd_batch_run(b, iters, V.VD_BATCH_BOOTSTRAP | (0 if args.no_tune else V.VD_BATCH_AUTOTUNE))

    def stepb():
        V.vd_batch_run(b, iters, V.VD_BATCH_BOOTSTRAP)

    for _ in range(args.warmup):
        stepb()
    torch.cuda.synchronize()
    barrier(pg)
    clocks = Clocks(local)
    clocks.start()
    tb = _timed(stream, flush, stepb, args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(pg)
    bstats = V.vd_batch_get_stats(b)
    bt = V.vd_get_tune(V.vd_batch_window(b, 0))
    bstats["tune"] = {k: bt[k] for k in ("k1_warps", "score_threads", "score_blocks_per_sm")}
    total_ms, value = whole_job(pg, world, units_per_window * nb * args.steps, sum(tb), dev)

    e2e = None
    if not args.no_e2e:
        e2e = run_batch_e2e(args, pg, V, b, bw, params, dev, iters, units_per_window, world)

    V.vd_batch_destroy(b)
    configs = None
    if world == 1 and not args.no_configs:
        # the other workloads, one line: small, stereo, the RGB-D batch
        configs = {
            "planes160": single_config(V, dev, stream, sptr, flush, "planes160", 0, {}, "none"),
            "boxes640_stereo": single_config(V, dev, stream, sptr, flush, "boxes640_stereo", 1000,
                                             {}, "stereo", steps=10, warmup=3),
            "rgbd_batch64": rgbd64_measure(V, dev, stream, sptr, flush, 3, 1, rank, pg),
            "learned_init": learned_measure(V)}
    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_config(nb, world),
                           **({"propagation": "hierarchical (cells 4, windows 32)"}
                              if args.hierarchical else {})),
            "windows_per_s": round(nb * args.steps * world / (total_ms / 1e3), 3),
            "single_window": single, "batch": bstats,
            "roofline": roofline, "stage_ms_per_window": stages,
            "gpu_launches": int(bstats["kernels_per_run"] * args.steps), "clocks": clk,
            "e2e": e2e, "configs": configs}
    return line



def pipelined_steps(n, bufs, stage, run, drain, submit):
    """n steps over two alternating buffers: step k runs bufs[k % 2] on the
    calling thread while submit() (a one-worker pool) drains the previous
    step's buffer and stages the next step's into it.  Every step is staged
    before its run and drained after it, exactly once; a buffer is staged
    again only after its previous step was drained."""
    stage(bufs[0])
    for k in range(n):
        cur, other = bufs[k % 2], bufs[(k + 1) % 2]

        def side_work(k=k, other=other):
            if k > 0:
                drain(other)
            if k + 1 < n:
                stage(other)

        fut = submit(side_work)
        run(cur)
        fut.result()
    drain(bufs[(n - 1) % 2])

def run_batch_e2e(args, pg, V, b, bw, params, dev, iters, units_per_window, world):
    """End-to-end throughput through the C ABI with host buffers: every step
    pushes one batch of flows from pinned host memory, runs the batch and
    reads every window's inverse depth and poses back.  Two batches on
    independent streams alternate, so that a helper thread pushes the next
    batch's flows and reads back the previous batch's results while the
    current batch runs (vd_batch_run blocks the calling thread; ctypes drops
    the interpreter lock around it).  Every copy is inside the timed region."""
    import concurrent.futures
    import torch
    N, W, H = bw[0].N, bw[0].W, bw[0].H
    nb = len(bw)
    side = torch.cuda.Stream(device=dev)
    b2 = V.vd_batch_create([(w.W, w.H, w.N, w.intrinsics) for w in bw], params,
                           V.C.c_void_p(side.cuda_stream))
    try:
        for i in range(nb):
            t = V.vd_get_tune(V.vd_batch_window(b, i))
            V.vd_set_tune(V.vd_batch_window(b2, i), t["k1_warps"], t["score_blocks_per_sm"],
                          t["score_threads"])
        host = [torch.from_numpy(w.flow).pin_memory() for w in bw]
        host_rho = torch.empty((H, W), dtype=torch.float32).pin_memory()
        bufs = (b, b2)

        def stage(x):
            for i in range(nb):
                c = V.vd_batch_window(x, i)
                for t in range(N):
                    V.vd_push_flow(c, t + 1, host[i][t].numpy())

        def drain(x):
            for i in range(nb):
                c = V.vd_batch_window(x, i)
                V.vd_get_inv_depth(c, host_rho.numpy())
                V.vd_get_poses(c, N)

        # one untimed pass through both batches (graph capture of the second)
        for x in bufs:
            stage(x)
            V.vd_batch_run(x, iters, V.VD_BATCH_BOOTSTRAP)
            drain(x)
        n_e2e = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        barrier(pg)
        with concurrent.futures.ThreadPoolExecutor(max_workers=1) as pool:
            t0 = time.perf_counter()
            pipelined_steps(n_e2e, bufs, stage,
                            lambda x: V.vd_batch_run(x, iters, V.VD_BATCH_BOOTSTRAP),
                            drain, pool.submit)
            torch.cuda.synchronize()
            dt = max_over_ranks(pg, time.perf_counter() - t0, dev)
    finally:
        V.vd_batch_destroy(b2)
    return {"value": round(units_per_window * nb * n_e2e * world / dt, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(sum(w.flow.nbytes for w in bw)),
            "d2h_bytes_per_step": int(nb * (W * H * 4 + (N + 1) * 12 * 8)), "steps": n_e2e,
            "path": "vd_push_flow from pinned host memory, vd_batch_run, vd_get_inv_depth + "
                    "vd_get_poses per window; two batches alternate so that one batch's "
                    "copies overlap the other's run"}


def _make_window(spec):
    import synth
    name, seed, kw = spec
    return synth.make_window(name, seed, **kw)


def make_windows(specs):
    """synth windows for [(name, seed, kwargs)], generated in parallel by
    spawned worker processes (this process may already hold a GPU context)."""
    import concurrent.futures
    import multiprocessing
    if len(specs) <= 1:
        return [_make_window(sp) for sp in specs]
    n = min(len(specs), os.cpu_count() or 1)
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=n, mp_context=ctx) as ex:
        return list(ex.map(_make_window, specs))


def rgbd64_measure(V, dev, stream, sptr, flush, steps, warmup, rank, pg):
    """64 windows with an RGB-D prior, sizes drawn from 320x240 / 640x480 /
    1216x368 and N from 3..8 (seeds 5000..5063), 5 EM iterations each: one
    window at a time (vd_bootstrap + vd_run_em per window) versus all of them
    in one graph launch (vd_batch_run).  Both give bit-identical results."""
    import torch
    nw, iters = 64, 5
    wins = make_windows([("rgbd_batch", 5000 + 64 * rank + i, {}) for i in range(nw)])
    prms = [V.vd_params_default(fisk_alpha0=w.params["fisk_alpha0"], rho_min=w.params["rho_min"],
                                rho_max=w.params["rho_max"], n_hyp=w.params["n_hyp"],
                                n_pose_samples=64) for w in wins]
    units = sum(w.W * w.H * w.N * iters for w in wins)

    def push(ctx, w):
        for t in range(1, w.N + 1):
            V.vd_push_flow(ctx, t, w.flow[t - 1])
        V.vd_push_depth_prior(ctx, w.depth_prior)

    # one window at a time, each on its own context
    ctxs = []
    for w, p in zip(wins, prms):
        c = V.vd_create(w.W, w.H, w.N, w.intrinsics, p, sptr)
        push(c, w)
        ctxs.append(c)

    def plain():
        for c in ctxs:
            V.vd_bootstrap(c)
            V.vd_run_em(c, iters, stats=False)

    for _ in range(max(1, warmup)):
        plain()
    torch.cuda.synchronize()
    tp = _timed(stream, flush, plain, steps)
    # the same windows as one batch
    b = V.vd_batch_create([(w.W, w.H, w.N, w.intrinsics) for w in wins], prms, sptr)
    for i, w in enumerate(wins):
        push(V.vd_batch_window(b, i), w)
    V.vd_batch_run(b, iters, V.VD_BATCH_BOOTSTRAP | V.VD_BATCH_AUTOTUNE)
    for _ in range(warmup):
        V.vd_batch_run(b, iters, V.VD_BATCH_BOOTSTRAP)
    torch.cuda.synchronize()
    clocks = Clocks(dev.index or 0)
    clocks.start()
    tb = _timed(stream, flush, lambda: V.vd_batch_run(b, iters, V.VD_BATCH_BOOTSTRAP), steps)
    torch.cuda.synchronize()
    clk = clocks.stop()
    # accuracy against the scenes' true depth (metric: the prior fixes the scale)
    errs, same = [], True
    for i, w in enumerate(wins):
        rb = np.empty((w.H, w.W), np.float32)
        rp = np.empty((w.H, w.W), np.float32)
        V.vd_get_inv_depth(V.vd_batch_window(b, i), rb)
        V.vd_get_inv_depth(ctxs[i], rp)
        same &= bool(np.array_equal(rb, rp))
        d = 1.0 / np.maximum(rb, 1e-9)
        errs.append(float(np.median(np.abs(d - w.depth0) / w.depth0)))
    bstats = V.vd_batch_get_stats(b)
    V.vd_batch_destroy(b)
    for c in ctxs:
        V.vd_destroy(c)
    world = 1 if pg is None else pg.get_world_size()
    tot_b = max_over_ranks(pg, sum(tb), dev)
    tot_p = max_over_ranks(pg, sum(tp), dev)
    sizes = {}
    for w in wins:
        sizes[f"{w.W}x{w.H}"] = sizes.get(f"{w.W}x{w.H}", 0) + 1
    return {"value": round(units * steps * world / (tot_b / 1e3), 1), "unit": UNIT,
            "windows_per_s": round(nw * steps * world / (tot_b / 1e3), 3),
            "ms_per_step": round(tot_b / steps, 3),
            "workload": f"rgbd_batch64: {nw} windows, RGB-D prior (1% noise, 10% holes), "
                        f"{iters} EM iterations, K=64, S=64; sizes {sizes}, "
                        f"N {min(w.N for w in wins)}..{max(w.N for w in wins)}",
            "plain": {"windows_per_s": round(nw * steps * world / (tot_p / 1e3), 3),
                      "value": round(units * steps * world / (tot_p / 1e3), 1),
                      "ms_per_step": round(tot_p / steps, 3)},
            "batched_equals_plain": same,
            "median_depth_rel_err": {"median_over_windows": round(float(np.median(errs)), 5),
                                     "max_over_windows": round(float(np.max(errs)), 5)},
            "batch": bstats, "gpu_launches": int(bstats["kernels_per_run"] * steps),
            "clocks": clk, "steps": steps}


def single_config(V, dev, stream, sptr, flush, name, seed, kw, prior, steps=20, warmup=5):
    """windows/s of one window at a time (vd_bootstrap + vd_run_em) for one of
    the smaller workloads, median of `steps` CUDA-event timings."""
    import torch
    w = make_windows([(name, seed, kw)])[0]
    pr = w.params
    params = V.vd_params_default(fisk_alpha0=pr["fisk_alpha0"], rho_min=pr["rho_min"],
                                 rho_max=pr["rho_max"], n_hyp=pr["n_hyp"], n_pose_samples=64)
    ctx = V.vd_create(w.W, w.H, w.N, w.intrinsics, params, sptr)
    try:
        for t in range(1, w.N + 1):
            V.vd_push_flow(ctx, t, w.flow[t - 1])
        if prior == "stereo":
            V.vd_push_stereo_prior(ctx, w.stereo_disp, w.stereo_baseline)
        iters = pr["n_iters"]

        def step():
            V.vd_bootstrap(ctx)
            V.vd_run_em(ctx, iters, stats=False)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        ms = statistics.median(_timed(stream, flush, step, steps))
        rho = np.empty((w.H, w.W), np.float32)
        V.vd_get_inv_depth(ctx, rho)
    finally:
        V.vd_destroy(ctx)
    d = 1.0 / np.maximum(rho, 1e-9)
    scale = float(np.median(w.depth0 / d)) if prior == "none" else 1.0
    return {"windows_per_s": round(1e3 / ms, 2), "ms_per_window": round(ms, 4),
            "value": round(w.W * w.H * w.N * iters / (ms / 1e3), 1), "unit": UNIT,
            "workload": f"{name} seed {seed}: {w.W}x{w.H}, N={w.N}, K={pr['n_hyp']}, "
                        f"{iters} EM iterations, prior {prior}, one window per call",
            "median_depth_rel_err_vs_truth": round(
                float(np.median(np.abs(d * scale - w.depth0) / w.depth0)), 5)}


def learned_measure(V, n_windows=16):
    """Plain vs learned-initialised EM (the committed network) on held-out
    windows of the learned initialiser's workload (640 x 480, N = 6, scenes
    of the stereo configuration's kind run monocularly, seeds 6000..): the
    iterations and windows/s to reach a median inverse-depth error against
    the converged plain EM (16 iterations) and against the scene's truth
    (paper_2104_06800_gb300.learned_init.evaluate)."""
    from paper_2104_06800_gb300 import learned_init as LI
    wins = make_windows([("boxes640_stereo", LI.EVAL_SEED0 + i, {"N": LI.N_FLOWS})
                         for i in range(n_windows)])
    net = V.vd_cnn_create(LI.N_FLOWS, seed=1)
    try:
        V.vd_cnn_set_params(net, np.load(os.path.join(ROOT, "paper_2104_06800_gb300", "weights",
                                                      "learned_init_boxes640_n6.npy")))
        rep = LI.evaluate(V, net, wins, log=lambda *a, **k: None)
    finally:
        V.vd_cnn_destroy(net)
    out = {"workload": f"boxes640_stereo scenes run monocularly, 640x480, N={LI.N_FLOWS}, "
                       f"{n_windows} held-out windows (seeds {LI.EVAL_SEED0}..), K=64",
           "reference": f"plain EM after {LI.REF_ITERS} iterations; error = median relative "
                        "inverse-depth error over its rigid pixels after the monocular scale "
                        "alignment",
           "max_iters": LI.MAX_ITERS}
    for kind in ("plain", "learned"):
        d = rep[kind]
        out[kind] = {k: {kk: round(vv, 4) for kk, vv in v.items()} for k, v in d.items()
                     if k.startswith("tol_") or k.startswith("truth_tol_")}
        out[kind]["ms_bootstrap"] = round(d["ms_bootstrap"], 4)
        out[kind]["ms_iteration"] = round(d["ms_iteration"], 4)
    return out


def run_rgbd64(args, rank, world, local, pg):
    """--workload rgbd_batch64: the 64-window RGB-D batch as the line's workload."""
    import torch
    from paper_2104_06800_gb300 import build as B
    from paper_2104_06800_gb300 import voldor as V
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    V.load()
    stream = torch.cuda.current_stream(dev)
    sptr = V.C.c_void_p(stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    r = rgbd64_measure(V, dev, stream, sptr, flush, args.steps, args.warmup, rank, pg)
    return {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": r["workload"],
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}"},
            "windows_per_s": r["windows_per_s"], "plain": r["plain"],
            "batched_equals_plain": r["batched_equals_plain"],
            "median_depth_rel_err": r["median_depth_rel_err"], "batch": r["batch"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "e2e": None}


def run_ka(args, rank, world, local, pg):
    """Keyframe alignment (Sec. III-C, Eq. 9-12) of two 1216 x 368 depth maps
    of the driving scene two frames apart (true depth times a smooth error
    field of up to 0.6 %, as the EM's propagated depth has, and 2 % holes;
    confidence 1), scale free, from a start 0.005 rad / 2 % off (the scale
    3 % off): the whole Levenberg-Marquardt run per step (vd_ka_align)."""
    import torch
    from paper_2104_06800_gb300 import build as B
    from paper_2104_06800_gb300 import voldor as V
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    V.load()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    Z0, Zt, T, K = synth.keyframe_pair("driving1216", WORK["seed"] + rank, 2)
    rng = np.random.default_rng(WORK["seed"] + rank)
    noisy = []
    for Z in (Z0, Zt):
        Hh, Ww = Z.shape
        vv, uu = np.mgrid[0:Hh, 0:Ww]
        ph = rng.uniform(0, 2 * np.pi, 4)
        field = 0.002 * (np.sin(uu / 97.0 + ph[0]) + np.sin(vv / 41.0 + ph[1]) +
                         np.sin((uu + vv) / 163.0 + ph[2]) * np.cos(uu / 57.0 + ph[3]))
        z = Z * (1.0 + field)
        z[rng.uniform(size=Z.shape) < 0.02] = np.nan
        noisy.append(torch.from_numpy(z.astype(np.float32)).to(dev))
    # start: a 0.005 rad rotation about a random axis and a 2 % translation offset
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rp = np.eye(3) + np.sin(0.005) * Kx + (1 - np.cos(0.005)) * Kx @ Kx
    off = rng.normal(size=3)
    off *= 0.02 * np.linalg.norm(T[:, 3]) / np.linalg.norm(off)
    T0 = np.hstack([Rp @ T[:, :3], (Rp @ T[:, 3] + off)[:, None]])

    def step(iters=50):
        return V.vd_ka_align(noisy[0], noisy[1], K, T0, s0=1.03, c=0.01, fix_scale=False,
                             max_iters=iters)

    for _ in range(max(1, args.warmup)):
        res = step()
    t_align = _timed(stream, flush, step, args.steps)
    t_eval = _timed(stream, flush, lambda: step(0), args.steps)
    ms = statistics.median(t_align)
    tot = max_over_ranks(pg, sum(t_align), dev)
    Re = res["T"][:, :3].T @ T[:, :3]
    rot_err = float(np.arccos(np.clip(0.5 * (np.trace(Re) - 1.0), -1.0, 1.0)))
    trans_err = float(np.linalg.norm(res["T"][:, 3] - T[:, 3]) / np.linalg.norm(T[:, 3]))
    W, H = Z0.shape[1], Z0.shape[0]
    return {"metric": "keyframe alignments/s", "value": round(args.steps * world / (tot / 1e3), 3),
            "unit": "alignments/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"ka1216: two {W}x{H} keyframes of the driving scene two "
                                   "frames apart, smooth depth error up to 0.6%, 2% holes, "
                                   "Cauchy c=0.01, scale free, start 0.005 rad / 2% / scale "
                                   "3% off",
                       "l2": "flushed (256 MB write) before every timed step"},
            "ms_per_evaluation": round(statistics.median(t_eval), 4),
            "iterations": res["iterations"], "n_valid": res["n_valid"],
            "rot_err_rad": rot_err, "trans_err_rel": trans_err,
            "scale": res["s"], "gpu_launches": int(args.steps * (2 * res["iterations"] + 3)),
            "e2e": None}


def cpu_baselines(small=True):
    """The oracle on the host: every core (the reported baseline), one core,
    and the small workload in full on one core."""
    v1, dt1, desc1 = oracle_sample()
    va, dta, ncores, desca = oracle_all_cores()
    out = {"value": round(va, 1), "unit": UNIT, "cores": ncores, "host": host_cpu(),
           "kind": "oracle", "sample": desca,
           "single_core": {"value": round(v1, 1), "unit": UNIT, "cores": 1, "sample": desc1}}
    if small:
        out["planes160_full"] = oracle_small_full()
    return out


def main():
    args = parse()
    rank, world, local, pg = dist_setup(args.gpus)
    if args.impl == "reference":
        if rank != 0:
            return 0
        # each timed step: one EM iteration of the oracle over the whole
        # window, one row band per host core (a few s of wall time);
        # warm-up steps one iteration on a 304 x 92 crop on one core (they
        # only take the one-time costs: imports, the window, first touches)
        for _ in range(max(args.warmup, 0)):
            oracle_sample(WORK["W"] // 4, WORK["H"] // 4)
        units_s, samples = [], []
        for _ in range(args.steps):
            v, dt, ncores, desc = oracle_all_cores()
            units_s.append(v)
            samples.append(dt)
        value = statistics.median(units_s)
        cfg = dict(workload_config(args.batch, 1))
        cfg["reference_step"] = desc
        line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
                "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1e3 * statistics.median(samples), 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg,
                "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": ncores,
                                 "host": host_cpu(), "kind": "oracle", "sample": desc},
                "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    if args.workload in ("rgbd_batch64", "ka1216"):
        line = (run_rgbd64 if args.workload == "rgbd_batch64" else run_ka)(args, rank, world,
                                                                         local, pg)
        if rank == 0:
            print(json.dumps(line))
        if pg is not None:
            pg.destroy_process_group()
        return 0
    if args.workload.startswith("driving1216"):
        WORK["name"] = args.workload
    line = run_ours(args, rank, world, local, pg)
    if rank == 0:
        if not args.no_cpu and world == 1:   # the host baseline: rank 0 of a 1-GPU run only
            line["cpu_baseline"] = cpu_baselines(small=not args.no_configs)
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

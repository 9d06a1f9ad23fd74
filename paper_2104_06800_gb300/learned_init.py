"""Training and evaluation of the learned initialiser (vd_cnn_*) on synthetic
windows.

Workload: scenes of the stereo configuration's kind (640 x 480, ground plane
and boxes to 40 m, 10 % moving blobs, smooth trajectory) with N = 6 flows, run
monocularly (no prior), so that the initial inverse depth and rigidness come
either from the monocular bootstrap (plain) or from the network (learned,
vd_bootstrap_learned).

Labels are the EM's own converged output: every training window is run with
the plain bootstrap and LABEL_ITERS iterations, and its inverse depth (in
units of |tau_1|, the monocular gauge) and per-flow rigidness are the targets.
The network is trained by the library's own kernels (tcgen05 forward and data
gradient, CUDA-core weight gradient, Adam).

Evaluation on held-out windows: the reference is the plain EM after REF_ITERS
iterations (the converged result); plain and learned-initialised EM then run
one iteration at a time, and after each the median relative inverse-depth
error against the reference, over the reference's rigid pixels and after
the monocular scale alignment, is recorded.  For a tolerance (1 %, 2 %, 5 %)
the iterations a window needs are the first at or below it (MAX_ITERS if
none), and windows/s at that accuracy is the number of windows over the
summed GPU time of the bootstrap and those iterations.  The same error
against the scene's true inverse depth is recorded too: the reference is
the plain EM's own future (same random draws), which favours the plain
start; the true depth favours neither.

    python -m paper_2104_06800_gb300.learned_init --train 2000 --epochs 8 \\
        --eval 100 --out weights.npy --report report.json

`--timing` instead times the network's kernels alone on one window of the
workload's size (random flow, pose and targets): the forward pass and a
training step (forward, loss, backward, no update), as the median of CUDA
event timings on the launching stream.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

N_FLOWS = 6
LABEL_ITERS = 12
REF_ITERS = 16
MAX_ITERS = 12
TOLS = (0.01, 0.02, 0.05)
TRUTH_TOLS = (0.06, 0.08, 0.10)
W_Q = 0.1
TRAIN_SEED0, EVAL_SEED0 = 4000, 6000


def _make(seed):
    import synth
    return synth.make_window("boxes640_stereo", seed, N=N_FLOWS)


def mono_range(win):
    """Inverse-depth search range in units of |tau_1| (the monocular gauge)
    for these windows run without their prior: the workload's, from its
    bounds on depth and on the per-frame motion (the window's own motion is
    not known to a deployed initialiser)."""
    pr = win.params
    return (float(np.float32(0.5 * pr["tmin"] / pr["dmax"])),
            float(np.float32(2.0 * pr["tmax"] / pr["dmin"])))


def params_for(V, win, seed=0):
    rmin, rmax = mono_range(win)
    return V.vd_params_default(fisk_alpha0=win.params["fisk_alpha0"], rho_min=rmin, rho_max=rmax,
                               n_hyp=win.params["n_hyp"], seed=seed)


def context(V, win, stream=None):
    ctx = V.vd_create(win.W, win.H, win.N, win.intrinsics, params_for(V, win), stream)
    for t in range(1, win.N + 1):
        V.vd_push_flow(ctx, t, win.flow[t - 1])
    return ctx


def depth_error(rho, ref, rigid):
    """Median relative inverse-depth error after the monocular scale alignment."""
    m = rigid & (rho > 0) & (ref > 0)
    if not m.any():
        return float("inf")
    s = np.median(ref[m] / rho[m])
    return float(np.median(np.abs(s * rho[m] - ref[m]) / ref[m]))


def label(V, win):
    """(rho [H][W], q [N][H][W]) of the plain EM after LABEL_ITERS iterations,
    and the bootstrap's pose of flow 1 (the network's geometry input)."""
    ctx = context(V, win)
    try:
        T1 = V.vd_eight_point(ctx)
        V.vd_bootstrap(ctx)
        V.vd_run_em(ctx, LABEL_ITERS)
        rho = np.empty((win.H, win.W), np.float32)
        q = np.empty((win.N, win.H, win.W), np.float32)
        V.vd_get_inv_depth(ctx, rho)
        V.vd_get_rigidness(ctx, q)
        return rho, q, T1
    finally:
        V.vd_destroy(ctx)


def train(V, net, data, epochs, lr0, seed=0, log=print):
    """data: list of (flow, rho, q, rho_min, rho_max, geometry) with CUDA
    tensors; geometry = (K, T1)."""
    import torch
    rng = np.random.default_rng(seed)
    H, W = data[0][0].shape[1], data[0][0].shape[2]
    mask = torch.ones((H, W), dtype=torch.uint8, device=data[0][0].device)
    history = []
    total = epochs * len(data)
    step = 0
    for ep in range(epochs):
        losses = []
        for i in rng.permutation(len(data)):
            flow, rho, q, rmin, rmax, geom = data[i]
            lr = lr0 * (0.1 + 0.9 * 0.5 * (1 + np.cos(np.pi * step / total)))   # cosine to lr0/10
            losses.append(V.vd_cnn_train_step(net, flow, rho, q, mask, rmin, rmax, W_Q, lr,
                                              geom=geom))
            step += 1
        history.append(float(np.mean(losses)))
        log(f"epoch {ep}: mean loss {history[-1]:.5f}", flush=True)
    return history


def evaluate(V, net, wins, log=print):
    """Per window, plain and learned: the depth error against the reference
    after the bootstrap and after each iteration, and the GPU time of each;
    summarised per tolerance as iterations needed and windows/s."""
    import torch
    stream = torch.cuda.current_stream()
    sptr = V.C.c_void_p(stream.cuda_stream)
    rows = []
    for win in wins:
        ctx = context(V, win, sptr)
        try:
            V.vd_bootstrap(ctx)
            V.vd_run_em(ctx, REF_ITERS)
            ref = np.empty((win.H, win.W), np.float32)
            qr = np.empty((win.N, win.H, win.W), np.float32)
            V.vd_get_inv_depth(ctx, ref)
            V.vd_get_rigidness(ctx, qr)
            rigid = qr.mean(axis=0) > 0.5
            truth = (np.linalg.norm(win.G[1][:, 3]) / win.depth0).astype(np.float32)
            row = {}
            for kind in ("plain", "learned"):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                rho = np.empty((win.H, win.W), np.float32)
                errs, ms, terrs = [], [], []
                for k in range(MAX_ITERS + 1):
                    e0.record(stream)
                    if k > 0:
                        V.vd_run_em(ctx, 1, stats=False)
                    elif kind == "plain":
                        V.vd_bootstrap(ctx)
                    else:
                        V.vd_bootstrap_learned(ctx, net)
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                    V.vd_get_inv_depth(ctx, rho)
                    errs.append(depth_error(rho, ref, rigid))
                    terrs.append(depth_error(rho, truth, rigid))
                row[kind] = {"err": errs, "ms": ms, "truth_err": terrs}
            rows.append(row)
            log("window: error after bootstrap plain %.3f learned %.3f; after %d iterations "
                "plain %.3f learned %.3f" % (row["plain"]["err"][0], row["learned"]["err"][0],
                                            MAX_ITERS, row["plain"]["err"][-1],
                                            row["learned"]["err"][-1]), flush=True)
        finally:
            V.vd_destroy(ctx)
    out = {"windows": len(rows), "max_iters": MAX_ITERS, "reference_iters": REF_ITERS}
    for kind in ("plain", "learned"):
        d = {"mean_error_by_iteration": [float(np.mean([r[kind]["err"][k] for r in rows]))
                                         for k in range(MAX_ITERS + 1)],
             "median_truth_error_by_iteration": [
                 float(np.median([r[kind]["truth_err"][k] for r in rows]))
                 for k in range(MAX_ITERS + 1)],
             "ms_bootstrap": float(np.mean([r[kind]["ms"][0] for r in rows])),
             "ms_iteration": float(np.mean([np.mean(r[kind]["ms"][1:]) for r in rows]))}
        for key, tols in (("err", TOLS), ("truth_err", TRUTH_TOLS)):
            for tol in tols:
                need, total = [], 0.0
                for r in rows:
                    k = next((i for i, e in enumerate(r[kind][key]) if e <= tol), None)
                    kk = MAX_ITERS if k is None else k
                    need.append(kk)
                    total += sum(r[kind]["ms"][:kk + 1])
                name = f"tol_{tol:g}" if key == "err" else f"truth_tol_{tol:g}"
                d[name] = {"mean_iters": float(np.mean(need)),
                           "reached": float(np.mean([
                               any(e <= tol for e in r[kind][key]) for r in rows])),
                           "windows_per_s": len(rows) / (total / 1e3)}
        out[kind] = d
    out["per_window"] = [{k: {"err": [round(e, 5) for e in r[k]["err"]],
                              "truth_err": [round(e, 5) for e in r[k]["truth_err"]],
                              "ms": [round(m, 3) for m in r[k]["ms"]]} for k in r} for r in rows]
    return out


def timing(V, reps=20, H=480, W=640, seed=0):
    """Median GPU time (ms) of the forward pass and of a training step of the
    network at H x W with N_FLOWS flows, after three untimed calls."""
    import torch
    dev = torch.device("cuda")
    rng = np.random.default_rng(seed)
    T = lambda a: torch.from_numpy(a).to(dev)
    flow = T((rng.normal(size=(N_FLOWS, H, W, 2)) * 20).astype(np.float32))
    rho_t = T(rng.uniform(0.1, 1.5, size=(H, W)).astype(np.float32))
    q_t = T((rng.uniform(size=(N_FLOWS, H, W)) > 0.3).astype(np.float32))
    mask = torch.ones((H, W), dtype=torch.uint8, device=dev)
    rho = torch.zeros((H, W), device=dev)
    geom = ((0.8 * W, 0.8 * W, W / 2, H / 2), np.hstack([np.eye(3), [[0.0], [0.0], [1.0]]]))
    net = V.vd_cnn_create(N_FLOWS, seed=1)
    stream = torch.cuda.current_stream()

    def med(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    try:
        fwd = med(lambda: V.vd_cnn_forward(net, flow, 0.05, 2.0, rho_out=rho, geom=geom))
        step = med(lambda: V.vd_cnn_train_step(net, flow, rho_t, q_t, mask, 0.05, 2.0, W_Q, 0.0,
                                               update=False, geom=geom))
    finally:
        V.vd_cnn_destroy(net)
    return {"size": [W, H], "flows": N_FLOWS, "forward_ms": round(fwd, 4),
            "train_step_ms": round(step, 4), "reps": reps}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train", type=int, default=2000, help="training windows")
    ap.add_argument("--eval", type=int, default=100, help="held-out evaluation windows")
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--weights", default=None, help="evaluate these weights (skip training)")
    ap.add_argument("--out", default=None, help="write the trained parameters (.npy)")
    ap.add_argument("--report", default=None, help="write the evaluation report (.json)")
    ap.add_argument("--timing", action="store_true",
                    help="only time the forward pass and a training step (640 x 480)")
    args = ap.parse_args(argv)
    if args.timing:
        from . import build, voldor as V
        build.build()
        V.load()
        print(json.dumps(timing(V)))
        return 0
    # the host pool (spawned processes, no CUDA) makes the scenes; the labels
    # and the training data live on the GPU, a chunk of windows at a time
    pool = mp.get_context("spawn").Pool(args.workers) if args.workers > 1 else None
    gen = (lambda seeds: pool.map(_make, seeds, chunksize=2)) if pool else \
        (lambda seeds: [_make(s) for s in seeds])
    t0 = time.time()
    eval_w = gen(range(EVAL_SEED0, EVAL_SEED0 + args.eval))
    report = {"eval_generation_s": round(time.time() - t0, 1)}
    import torch
    from . import build, voldor as V
    build.build()
    V.load()
    dev = torch.device("cuda")
    net = V.vd_cnn_create(N_FLOWS, seed=1)
    if args.weights:
        V.vd_cnn_set_params(net, np.load(args.weights))
    else:
        t0 = time.time()
        t_lab = 0.0
        data = []
        seeds = list(range(TRAIN_SEED0, TRAIN_SEED0 + args.train))
        for c in range(0, len(seeds), 128):
            chunk = gen(seeds[c:c + 128])
            t1 = time.time()
            for w in chunk:
                rho, q, T1 = label(V, w)
                rmin, rmax = mono_range(w)
                data.append((torch.from_numpy(w.flow).to(dev), torch.from_numpy(rho).to(dev),
                             torch.from_numpy(q).to(dev), rmin, rmax, (w.intrinsics, T1)))
            t_lab += time.time() - t1
            del chunk
            print(f"training windows: {len(data)}", flush=True)
        report["train_generation_and_label_s"] = round(time.time() - t0, 1)
        report["label_s"] = round(t_lab, 1)
        t0 = time.time()
        report["loss_per_epoch"] = train(V, net, data, args.epochs, args.lr)
        torch.cuda.synchronize()
        report["train_s"] = round(time.time() - t0, 1)
        report.update(train_windows=args.train, epochs=args.epochs)
        del data
        if args.out:
            np.save(args.out, V.vd_cnn_get_params(net))
    report["eval"] = evaluate(V, net, eval_w)
    V.vd_cnn_destroy(net)
    if pool:
        pool.close()
    summary = {k: v for k, v in report.items() if k != "eval"}
    summary["eval"] = {k: v for k, v in report["eval"].items() if k != "per_window"}
    print(json.dumps(summary))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f)
    return 0


if __name__ == "__main__":
    sys.exit(main())

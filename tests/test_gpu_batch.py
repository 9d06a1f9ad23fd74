"""Batched, graph-captured EM and the launch-shape tuner.

A batch runs the bootstrap and the EM iterations of many independent windows
of uneven size, flow count and prior as one CUDA graph.  Each window's
kernels, inputs and order are those of the window run alone, so its results
must be bit-identical to vd_bootstrap + vd_run_em on that window; parity of
the single-window path with the float64 oracle is covered by
test_gpu_parity.py and test_gpu_chained.py, and the windows of a mixed
RGB-D batch are replayed stage by stage against the oracle here.  The
depth-sampling launch shapes the tuner chooses between must not change a
single output bit either."""
import numpy as np
import pytest

import chained
from gpu_common import noisy_state, params_for, push_state, window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2104_06800_gb300 import build, voldor
    build.build()
    voldor.load()
    return voldor


def _windows():
    """RGB-D windows of the batched workload's kind (uneven size and N), plus
    a monocular and a stereo window."""
    ws = [window("rgbd_batch", 5000 + i, size=sz, N=n)
          for i, (sz, n) in enumerate([((320, 240), 3), ((640, 480), 5), ((320, 240), 8)])]
    ws.append(window("planes160", 0))
    ws.append(window("boxes640_stereo", 7, size=(320, 240)))
    return ws


def _push(V, ctx, w):
    for t in range(1, w.N + 1):
        V.vd_push_flow(ctx, t, w.flow[t - 1])
    if w.stereo_disp is not None:
        V.vd_push_stereo_prior(ctx, w.stereo_disp, w.stereo_baseline)
    elif w.depth_prior is not None:
        V.vd_push_depth_prior(ctx, w.depth_prior)


def _results(V, ctx, w):
    rho = np.empty((w.H, w.W), np.float32)
    q = np.empty((w.N, w.H, w.W), np.float32)
    V.vd_get_inv_depth(ctx, rho)
    V.vd_get_rigidness(ctx, q)
    return rho, q, V.vd_get_poses(ctx, w.N)


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def _alone(V, w, tune=None):
    ctx = V.vd_create(w.W, w.H, w.N, w.intrinsics, V.vd_params_default(**params_for(w)))
    if tune is not None:
        V.vd_set_tune(ctx, tune["k1_warps"], tune["score_blocks_per_sm"], tune["score_threads"])
    _push(V, ctx, w)
    return ctx


def test_batch_equals_each_window_alone_and_replays(V):
    wins = _windows()
    iters = 3
    alone = []
    for w in wins:
        ctx = _alone(V, w)
        V.vd_bootstrap(ctx)
        V.vd_run_em(ctx, iters)
        alone.append(ctx)
    b = V.vd_batch_create([(w.W, w.H, w.N, w.intrinsics) for w in wins],
                          [V.vd_params_default(**params_for(w)) for w in wins])
    try:
        for i, w in enumerate(wins):
            _push(V, V.vd_batch_window(b, i), w)
        for rep in range(2):        # capture, then replay of the captured graph
            deg = V.vd_batch_run(b, iters, V.VD_BATCH_BOOTSTRAP, len(wins))
            assert len(deg) == len(wins)
            for i, w in enumerate(wins):
                assert _same(_results(V, V.vd_batch_window(b, i), w), _results(V, alone[i], w)), \
                    (rep, i)
        st = V.vd_batch_get_stats(b)
        assert st["windows"] == len(wins) and st["captures"] == 1 and st["replays"] == 1
        assert st["kernels_per_run"] > 0 and st["graph_nodes"] >= st["kernels_per_run"]
        # one more iteration without the bootstrap: a new capture, still equal
        V.vd_batch_run(b, 1, 0)
        for i, w in enumerate(wins):
            V.vd_run_em(alone[i], 1)
            assert _same(_results(V, V.vd_batch_window(b, i), w), _results(V, alone[i], w)), i
        assert V.vd_batch_get_stats(b)["captures"] == 2
        # the batch owns its windows' streams and lifetimes
        with pytest.raises(V.VoldorError):
            V.vd_destroy(V.vd_batch_window(b, 0))
        with pytest.raises(V.VoldorError):
            V.vd_set_stream(V.vd_batch_window(b, 0), None)
    finally:
        V.vd_batch_destroy(b)
        for ctx in alone:
            V.vd_destroy(ctx)


def test_batch_autotune_shares_choices_and_matches_alone(V):
    wins = [window("rgbd_batch", 5100 + i, size=(320, 240), N=4) for i in range(2)]
    wins.append(window("planes160", 0))
    b = V.vd_batch_create([(w.W, w.H, w.N, w.intrinsics) for w in wins],
                          [V.vd_params_default(**params_for(w)) for w in wins])
    try:
        for i, w in enumerate(wins):
            _push(V, V.vd_batch_window(b, i), w)
        V.vd_batch_run(b, 2, V.VD_BATCH_BOOTSTRAP | V.VD_BATCH_AUTOTUNE)
        tunes = [V.vd_get_tune(V.vd_batch_window(b, i)) for i in range(len(wins))]
        for t in tunes:
            assert t["k1_warps"] in (1, 2, 4) and 1 <= t["score_blocks_per_sm"] <= 4
            assert t["score_threads"] in (256, 512)
        same = ("k1_warps", "score_blocks_per_sm", "score_threads")
        assert all(tunes[0][k] == tunes[1][k] for k in same)   # same launch configuration
        assert all(v > 0 for v in tunes[0]["k1_ms"] + tunes[0]["score_ms"][0] + tunes[0]["score_ms"][1])
        for i, w in enumerate(wins):
            ctx = _alone(V, w, tunes[i])
            V.vd_bootstrap(ctx)
            V.vd_run_em(ctx, 2)
            assert _same(_results(V, V.vd_batch_window(b, i), w), _results(V, ctx, w)), i
            V.vd_destroy(ctx)
        with pytest.raises(V.VoldorError):     # tuning needs the bootstrap flag
            V.vd_batch_run(b, 1, V.VD_BATCH_AUTOTUNE)
    finally:
        V.vd_batch_destroy(b)


def test_depth_sampling_launch_shapes_are_bit_identical(V):
    """The staged depth-sampling kernel at 1, 2 and 4 warps per block: the
    same argmin and energy on every pixel (the shapes only change which lane
    evaluates which candidate)."""
    w = window("driving1216", 2001, size=(608, 184))
    rng = np.random.default_rng(3)
    ctx = _alone(V, w)
    try:
        from oracle import model as omodel
        P = omodel.problem_from_window(w)
        S = noisy_state(w, P, rng, rel=0.05)
        out = []
        for warps in (1, 2, 4):
            V.vd_set_tune(ctx, warps, 2)
            push_state(V, ctx, S)
            V.vd_depth_mstep(ctx, 2, 1)
            rs = np.empty((w.H, w.W), np.float32)
            es = np.empty((w.H, w.W), np.float32)
            V.vd_get_depth_candidates(ctx, rs, es)
            out.append((rs, es))
        for rs, es in out[1:]:
            assert np.array_equal(rs, out[0][0]) and np.array_equal(es, out[0][1])
    finally:
        V.vd_destroy(ctx)


def test_score_launch_shapes_agree_to_rounding(V):
    """Threads per block and blocks per SM of the dense pose scoring only
    regroup float32 partial sums: the per-sample energies agree to rounding."""
    w = window("planes160", 0)
    rng = np.random.default_rng(4)
    ctx = _alone(V, w)
    try:
        from oracle import model as omodel
        P = omodel.problem_from_window(w)
        S = noisy_state(w, P, rng, rel=0.02, qmode="ones")
        energies = []
        for threads, bps in ((256, 1), (256, 2), (256, 4), (512, 1), (512, 3)):
            V.vd_set_tune(ctx, 4, bps, threads)
            push_state(V, ctx, S)
            V.vd_pose_mstep(ctx, 1, 1)
            _, e, _ = V.vd_get_pose_samples(ctx, 64)
            energies.append(np.asarray(e, np.float64))
        for e in energies[1:]:
            ok = np.isfinite(energies[0])
            assert np.array_equal(ok, np.isfinite(e))
            assert np.allclose(e[ok], energies[0][ok], rtol=2e-5, atol=1e-3)
    finally:
        V.vd_destroy(ctx)


def test_bootstrap_restarts_from_the_initial_poses(V):
    """Running bootstrap + EM twice on one context gives the same result:
    the bootstrap starts from the initial poses, not from the last run's."""
    for w in (window("rgbd_batch", 5200, size=(320, 240), N=3), window("planes160", 0)):
        ctx = _alone(V, w)
        try:
            runs = []
            for _ in range(2):
                V.vd_bootstrap(ctx)
                V.vd_run_em(ctx, 2)
                runs.append(_results(V, ctx, w))
            assert _same(runs[0], runs[1]), w.name
        finally:
            V.vd_destroy(ctx)


def test_batch_windows_are_the_chained_oracle_replay(V):
    """A mixed RGB-D batch of the batched workload's kind (uneven size and
    N, the prior with 1 % noise and 10 % holes): every window's bootstrap
    and 3 iterations replayed stage by stage against the float64 oracle at
    the method's bounds (chained.py), and the batch's graph launch gives
    each window bit for bit the replay's depth, rigidness and poses."""
    from oracle import model as omodel
    specs = [((96, 72), 3), ((128, 80), 5), ((80, 64), 4)]
    wins = [window("rgbd_batch", 5300 + i, size=sz, N=n) for i, (sz, n) in enumerate(specs)]
    iters = 3
    b = V.vd_batch_create([(w.W, w.H, w.N, w.intrinsics) for w in wins],
                          [V.vd_params_default(**params_for(w)) for w in wins])
    try:
        for i, w in enumerate(wins):
            _push(V, V.vd_batch_window(b, i), w)
        V.vd_batch_run(b, iters, V.VD_BATCH_BOOTSTRAP, len(wins))
        for i, w in enumerate(wins):
            P = omodel.problem_from_window(w, prior="rgbd")
            assert P.prior_kind == "rgbd"
            rep = chained.replay(V, lambda w=w: _alone(V, w), P, omodel.Params(**params_for(w)),
                                 iters, f"batch window {i} {w.W}x{w.H} N={w.N}")
            print(rep.summary())
            rho, q, G = _results(V, V.vd_batch_window(b, i), w)
            assert np.array_equal(rho, rep.final.rho), i
            assert np.array_equal(q, rep.final.q), i
            assert np.array_equal(np.asarray(G), rep.final.G), i
    finally:
        V.vd_batch_destroy(b)

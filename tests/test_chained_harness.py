"""The chained replay harness (chained.py) on the CPU.

A stand-in for the library that runs the float64 oracle itself must pass
every stage; stand-ins with one planted slip (a rigidness entry 2e-4 off, a
pose 2e-4 rad off, a depth choice outside the tie band, a run that is not
the chained one) must each fail the stage that shows it.
"""
import numpy as np
import pytest

import synth
from oracle import depth as odepth
from oracle import eightpoint as oeight
from oracle import em as oem
from oracle import geometry as ogeo
from oracle import hmm as ohmm
from oracle import model as omodel
from oracle import pose as opose

import chained
from gpu_common import params_for


class OracleLib:
    """The ABI calls the harness makes, answered by the oracle (float32
    storage of the maps, as the library)."""
    VD_OK, VD_WARN_DEGENERATE = 0, 1

    def __init__(self, P, p, slip=None):
        self.P, self.p, self.slip = P, p, slip

    # contexts
    def make(self):
        P = self.P
        return dict(S=omodel.State(rho=np.ones((P.H, P.W), np.float32),
                                   q=np.ones((P.N, P.H, P.W), np.float32),
                                   qhat=np.ones((P.H, P.W), np.float32),
                                   G=np.stack([ogeo.IDENTITY] * (P.N + 1))),
                    C=np.zeros((P.H, P.W), np.float32), star=None, samples=None, n=0, it=0)

    def vd_destroy(self, ctx):
        pass

    def vd_set_poses(self, ctx, G):
        ctx["S"].G = np.array(G, np.float64).reshape(-1, 3, 4)

    def vd_set_state(self, ctx, rho, q=None, qhat=None):
        S = ctx["S"]
        S.rho = np.array(rho, np.float32)
        S.q = np.array(q, np.float32) if q is not None else np.ones_like(S.q)
        S.qhat = np.array(qhat, np.float32) if qhat is not None else np.ones_like(S.qhat)

    def vd_eight_point(self, ctx):
        G1, _ = oeight.bootstrap_pose(self.P, self.p.fisk_alpha0)
        return G1

    def vd_depth_mstep(self, ctx, it, d):
        S = ctx["S"]
        new, _, rs, es = odepth.depth_mstep(self.P, S, it, d, self.p)
        if self.slip == "depth" and it == 0:
            # one pixel keeps its worst candidate (one of its own candidates,
            # far outside the tie band)
            v, u = self.P.H // 2, self.P.W // 2
            c = odepth.hypotheses(self.P, S.rho, it, self.p)[:, v, u]
            E = omodel.energy(self.P, S, np.full(len(c), u), np.full(len(c), v), c, self.p)
            rs = rs.copy()
            rs[v, u] = c[int(np.argmax(E))]
            es = es.copy()
            es[v, u] = np.float32(E.max())
        ctx["star"] = (rs.astype(np.float32), es.astype(np.float32))
        S.rho = new.astype(np.float32)

    def vd_get_depth_candidates(self, ctx, rs, es):
        rs[...] = ctx["star"][0]
        es[...] = ctx["star"][1]

    def vd_get_inv_depth(self, ctx, out):
        out[...] = ctx["S"].rho

    def vd_rigidness_estep(self, ctx, d):
        S = ctx["S"]
        q, qh, C = ohmm.rigidness_estep(self.P, S, S.rho, d, self.p)
        if self.slip == "estep":
            q = q.copy()
            q[0, self.P.H // 2, self.P.W // 3] += np.float32(2e-4)
            C = ((q.astype(np.float64).sum(0)) / self.P.N).astype(np.float32)
        S.q, S.qhat, ctx["C"] = q, qh, C

    def vd_get_rigidness(self, ctx, out):
        out[...] = ctx["S"].q

    def vd_get_prior_rigidness(self, ctx, out):
        out[...] = ctx["S"].qhat

    def vd_get_confidence(self, ctx, out):
        out[...] = ctx["C"]

    def vd_pose_mstep(self, ctx, it, t):
        S = ctx["S"]
        out = opose.pose_mstep_frame(self.P, S, t, it, self.p, detail=True)
        if self.slip == "pose" and it == 0 and t == 1:
            S.G[t] = ogeo.compose(S.G[t], ogeo.se3_exp(np.array([2e-4, 0, 0, 0, 0, 0])))
        poses = np.zeros((self.p.n_pose_samples, 12))
        en = np.full(self.p.n_pose_samples, np.inf)
        for g in range(self.p.n_pose_samples):
            if out["roots"][g]:
                k = int(np.argmin(out["root_scores"][g]))
                poses[g] = out["roots"][g][k].reshape(12)
                en[g] = out["root_scores"][g][k]
        ctx["samples"] = (poses.reshape(-1, 3, 4), en)
        ctx["n"] = out["n_rigid"]
        return self.VD_WARN_DEGENERATE if out["degenerate"] else self.VD_OK

    def vd_get_pose_samples(self, ctx, S):
        return ctx["samples"][0], ctx["samples"][1], ctx["n"]

    def vd_get_poses(self, ctx, N):
        return ctx["S"].G.copy()

    def vd_bootstrap(self, ctx):
        S, _ = oem.bootstrap(self.P, self.p)
        ctx["S"] = S

    def vd_run_em(self, ctx, n):
        S = ctx["S"]
        for it in range(n):
            oem.iteration(self.P, S, it, self.p)
        if self.slip == "run":
            S.rho = (S.rho * np.float32(1.0 + 2e-7)).astype(np.float32)


def _setup():
    win = synth.make_window("planes160", 1)
    kw = params_for(win, n_hyp=8, n_pose_samples=12)
    P = omodel.problem_from_window(win)
    return P, omodel.Params(**kw)


def test_replay_of_the_oracle_passes():
    P, p = _setup()
    lib = OracleLib(P, p)
    rep = chained.replay(lib, lib.make, P, p, 2, "oracle stand-in")
    stages = [r["stage"] for r in rep.rows]
    assert stages[0] == "boot/8pt" and stages[-1] == "run"
    assert len(stages) == 1 + 1 + P.N + 2 * (2 + P.N) + 1


@pytest.mark.parametrize("slip,where", [("depth", "it0/depth"), ("estep", "it0/estep"),
                                        ("pose", "it0/pose1"), ("run", "vd_run_em")])
def test_replay_catches_a_planted_slip(slip, where):
    P, p = _setup()
    lib = OracleLib(P, p, slip=slip)
    with pytest.raises(AssertionError) as e:
        chained.replay(lib, lib.make, P, p, 2, f"slip {slip}")
    assert where in str(e.value), str(e.value)


def test_float32_ranges_hold_the_oracle_and_are_tight_off_edges():
    """term_ranges' intervals contain the oracle's own energy and emission of
    every term; away from flow edges and thresholds they are narrow."""
    P, p = _setup()
    S, _ = oem.bootstrap(P, p)
    iu, iv = omodel.pixel_grid(P)
    tr = chained.term_ranges(P, S.G, iu, iv, S.rho, p)
    ell, e1, _ = omodel.flow_terms(P, S.G, iu, iv, S.rho, p)
    assert np.all(tr["l_lo"] <= ell + 1e-12) and np.all(tr["l_hi"] >= ell - 1e-12)
    assert np.all(tr["e1_lo"] <= e1 * (1 + 1e-12)) and np.all(tr["e1_hi"] >= e1 * (1 - 1e-12))
    calm = ~tr["flipped"] & ~tr["steep"]
    assert calm.mean() > 0.9
    width = (tr["l_hi"] - tr["l_lo"])[calm]
    assert np.median(width) < 1e-4 and np.percentile(width, 99) < 2e-3
    E = omodel.energy(P, S, iu, iv, S.rho, p)
    lo, hi = chained.energy_range(P, S, iu, iv, S.rho, p)
    assert np.all(lo <= E + 1e-12) and np.all(hi >= E - 1e-12)


def test_double_float_ranges_hold_the_oracle_and_leave_no_flips():
    """The ranges of the rigidness emissions (double-float positions) hold
    the oracle's emissions, decide every border and camera-plane test, and
    are narrow enough for the 1e-4 posterior check almost everywhere."""
    P, p = _setup()
    S, _ = oem.bootstrap(P, p)
    iu, iv = omodel.pixel_grid(P)
    tr = chained.term_ranges(P, S.G, iu, iv, S.rho, p, positions="df")
    tr32 = chained.term_ranges(P, S.G, iu, iv, S.rho, p)
    _, e1, _ = omodel.flow_terms(P, S.G, iu, iv, S.rho, p)
    assert np.all(tr["e1_lo"] <= e1 * (1 + 1e-12)) and np.all(tr["e1_hi"] >= e1 * (1 - 1e-12))
    assert not tr["flipped"].any()
    pos = e1 > 0
    rel = (tr["e1_hi"] - tr["e1_lo"])[pos] / e1[pos]
    rel32 = (tr32["e1_hi"] - tr32["e1_lo"])[pos] / e1[pos]
    assert np.percentile(rel, 99) < 2e-4 and rel.max() < 1e-3
    assert np.median(rel) * 20 < np.median(rel32)


def test_chain_posterior_rises_with_every_rigid_emission():
    """The E-step interval check rests on this: with gamma >= 1/2 the
    posterior of every position is non-decreasing in each rigid emission."""
    rng = np.random.default_rng(0)
    for gamma in (0.5, 0.8, 0.95, 0.999):
        for _ in range(20):
            L = int(rng.integers(2, 40))
            e1 = rng.uniform(0, 2, L) * (rng.uniform(size=L) > 0.1)
            e0 = np.full(L, 1.0)
            base = ohmm.forward_backward(e1, e0, gamma)
            j = int(rng.integers(0, L))
            up = e1.copy()
            up[j] = up[j] * 1.5 + 0.1
            assert np.all(ohmm.forward_backward(up, e0, gamma) >= base - 1e-12)


def test_score_range_holds_the_oracle_score():
    P, p = _setup()
    S, _ = oem.bootstrap(P, p)
    rs = opose.rigid_set(P, S, 2, p)
    rng = np.random.default_rng(3)
    for k in range(5):
        G = ogeo.compose(S.G[2], ogeo.se3_exp(rng.normal(size=6) * 0.02 * k))
        E = opose.score(P, G, rs, p)
        lo, hi = chained.score_range(P, G, rs, p)
        assert lo <= E <= hi and (hi - lo) < 2e-3 * E + 1e-6

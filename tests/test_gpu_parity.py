"""Parity of the CUDA library (through the C ABI) with the CPU FP64 oracle.

Tolerances (float32 GPU arithmetic against FP64):
  * interval bounds: the float32 interval contains the FP64 one and is within 4e-6 (1 + |v|) of it
    (FP64 accumulation per layer, outward rounding to float32 at every layer);
  * one-iteration lockstep of the duals: 1e-5 relative, 1e-7 absolute floor, plus the spread of
    the oracle's Adam step over gradients within a float32 summation bound of its own
    (tests/lockstep.py); rows that read an x* or z* decided within that bound are left out and
    counted (none in the drawn states, a small fraction allowed at full size);
  * bounds: 1e-4 absolute, 1e-5 relative where values are large;
  * masks and snapshot bits: bit-exact.
"""
import numpy as np
import pytest

from oracle import active_set as AS
from oracle import dual as du
from oracle import envelope as ev
from oracle import network as nw
from oracle import relaxation as rx
from oracle import saddle as SPm
from paper_2101_05844_gb300 import binding, synth
from tests.helpers import sample_min_output
from tests.lockstep import check_active_set_step
from tests.state_helpers import conv4_full_batch, draw_state, hidden_concat, oracle_bounds_f32, split_hidden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    binding.lib()


def _problems(name, S=None, seed=0):
    prob = synth.problem(name, S=S, seed=seed)
    return prob, nw.problems(prob)


@pytest.mark.parametrize("name,S", [("mlp_tiny", 1), ("small_conv", 3), ("wide_conv_bab", 6),
                                    ("mlp_5_7_6_3", 4)])
def test_interval_bounds_match_oracle(name, S):
    prob, Ps = _problems(name, S)
    ctx = binding.context_for(prob, binding.default_options())
    lh = ctx.get_state(binding.ST_LHAT).reshape(ctx.S, -1)
    uh = ctx.get_state(binding.ST_UHAT).reshape(ctx.S, -1)
    for s, P in enumerate(Ps):
        rl = hidden_concat(P.lhat)
        ru = hidden_concat(P.uhat)
        # sound: the float32 interval (outward rounding at every layer) contains the FP64 one
        assert (lh[s] <= rl + 1e-9 * (1 + np.abs(rl))).all()
        assert (uh[s] >= ru - 1e-9 * (1 + np.abs(ru))).all()
        # and close: a few float32 ulps per layer of propagation
        assert (np.abs(lh[s] - rl) <= 4e-6 * (1 + np.abs(rl))).all()
        assert (np.abs(uh[s] - ru) <= 4e-6 * (1 + np.abs(ru))).all()
    # zero duals: the bound is the interval bound of the output row
    b = ctx.bound()
    for s, P in enumerate(Ps):
        assert b[s] == pytest.approx(P.ibp_output_bound(), abs=1e-4, rel=1e-5)


CASES = [
    # name, S, options, iteration, filled slots
    ("mlp_tiny", 1, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 3, 0),     # Big-M
    ("mlp_tiny", 1, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 7, 2),     # AS, no add
    ("mlp_tiny", 1, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 8, 2),     # AS, adds slot 2
    ("small_conv", 3, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 12, 4),  # adds slot 4
    ("small_conv", 3, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=7), 10, 3),
    ("mlp_5_7_6_3", 4, dict(bigm_iters=2, as_iters=30, omega=4, max_cuts=8), 16, 6),  # adds slot 6
]


@pytest.mark.parametrize("name,S,kw,it,nslots", CASES)
def test_one_iteration_lockstep(name, S, kw, it, nslots):
    prob, _ = _problems(name, S)
    Ps0 = nw.problems(prob)
    lh, uh = oracle_bounds_f32(Ps0)
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), Ps0[0].widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), Ps0[0].widths)[1:])
                                   for s in range(len(Ps0))])
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, **kw), bounds=(lh, uh))
    solvers = draw_state(Ps, ctx, kw, it, nslots, seed=100 + it)
    # bound at the drawn duals
    gb = ctx.bound()
    for s, sv in enumerate(solvers):
        val, f, g, x, z = du.evaluate(sv.P, sv.st)
        assert gb[s] == pytest.approx(val, abs=1e-4, rel=1e-5)
        # the minimiser is decided (no near-zero coefficient) for the lockstep below
        assert min(np.abs(fk).min() for fk in f if fk is not None) > 1e-5
        for gk in g[1:]:
            assert ((gk == 0) | (np.abs(gk) > 1e-5)).all()
    ctx.as_step(1)
    xstar = ctx.get_state(binding.ST_XSTAR).reshape(S, -1)
    zstar = ctx.get_state(binding.ST_ZSTAR, np.uint8).reshape(S, -1)
    xs = ctx.get_state(binding.ST_XSNAP, np.uint8).reshape(S, -1)
    zs = ctx.get_state(binding.ST_ZSNAP, np.uint8).reshape(S, -1)
    al = ctx.get_state(binding.ST_ALPHA).reshape(S, -1)
    b0 = ctx.get_state(binding.ST_BETA0).reshape(S, -1)
    b1 = ctx.get_state(binding.ST_BETA1).reshape(S, -1)
    sb = ctx.get_state(binding.ST_SLOT_BETA).reshape(S, ctx.cap, -1)
    lam = ctx.get_state(binding.ST_LAMBDA).reshape(S, ctx.cap, -1)
    for s, sv in enumerate(solvers):
        P = sv.P
        _, f, g, x, z = du.evaluate(P, sv.st)
        slots_before = len(sv.st.slots[1])
        np.testing.assert_array_equal(zstar[s], hidden_concat(z).astype(np.uint8))
        res = check_active_set_step(sv, dict(alpha=al[s], beta0=b0[s], beta1=b1[s], slots=sb[s], xstar=xstar[s]))
        assert res["exempt_rows"] == 0 and res["undecided_x"] == 0
        # the new slot's snapshot: the oracle's mask at (x*, z*) (bit-exact)
        nnew = len(sv.st.slots[1])
        if nnew > slots_before:
            b = nnew - 1
            offs = np.cumsum([0] + P.widths)
            for k in range(1, P.n):
                xb = ((xs[s, offs[k - 1]:offs[k]] >> b) & 1).astype(bool)
                zb = ((zs[s, offs[k] - P.widths[0]:offs[k + 1] - P.widths[0]] >> b) & 1).astype(float)
                Igpu = rx.mask(P.W[k], P.lo[k - 1], P.hi[k - 1], np.where(xb, P.hi[k - 1], P.lo[k - 1]), zb)
                np.testing.assert_array_equal(Igpu, sv.st.slots[k][b].I)
            np.testing.assert_allclose(
                lam[s, b], hidden_concat([None] + [sv.st.slots[k][b].lam for k in range(1, P.n)]),
                rtol=1e-5, atol=1e-5)


def _as_margin(sv):
    _, f, g, x, z = du.evaluate(sv.P, sv.st)
    m = min(np.abs(fk).min() for fk in f)
    for gk in g[1:]:
        nz = gk[gk != 0]
        if nz.size:
            m = min(m, np.abs(nz).min())
    return m


def test_small_mlp_active_set_matches_oracle_at_every_iteration():
    """The small MLP workload as specified (8-16-16-1, one subproblem, 100 iterations: 20 Big-M,
    then 80 Active Set with masks added at t = 0, 1, 24, 25, 48, cap 5, omega = 24): the float32
    GPU run and the FP64 oracle agree to 1e-4 at every iteration, with no divergence allowed, and
    the final and best bounds agree to 1e-4."""
    prob, Ps = _problems("mlp_tiny", 1)
    kw = dict(bigm_iters=20, as_iters=80, omega=24, max_cuts=5)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, track_best=1, **kw))
    sv = AS.ActiveSet(Ps[0], AS.Options(**kw))
    worst = 0.0
    for it in range(100):
        ctx.as_step(1)
        sv.step(1)
        d = abs(ctx.bound()[0] - du.evaluate(sv.P, sv.st)[0])
        worst = max(worst, d)
        assert d <= 1e-4, f"iteration {it}: GPU and oracle bounds differ by {d}"
    b, best = ctx.bound(best=True)
    assert b[0] == pytest.approx(sv.bound(), abs=1e-4)
    assert best[0] == pytest.approx(sv.best, abs=1e-4)
    assert [len(sv.st.slots[k]) for k in range(1, sv.P.n)] == [5, 5]
    assert best[0] <= sample_min_output(sv.P, 100_000) + 1e-6


@pytest.mark.parametrize("name,S,kw,iters", [
    ("mlp_5_7_6_3", 4, dict(bigm_iters=30, as_iters=60, omega=20, max_cuts=4), 90),
    ("small_conv", 3, dict(bigm_iters=20, as_iters=40, omega=12, max_cuts=5), 60),
])
def test_free_running_active_set_matches_oracle(name, S, kw, iters):
    """Iteration by iteration: the GPU and oracle bounds agree to 1e-4 until the first iteration
    whose decisions the oracle takes within 1e-3 of a tie, the size float32 drift of the duals
    reaches over tens of iterations (a rounding flip, after which the runs are different valid
    runs, both checked valid). The first 10 iterations must agree."""
    prob, Ps = _problems(name, S)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, track_best=1, **kw))
    sol = [AS.ActiveSet(P, AS.Options(**kw)) for P in Ps]
    live = [True] * S
    for it in range(iters):
        margins = [_as_margin(sv) for sv in sol]
        ctx.as_step(1)
        gb = ctx.bound()
        for s, sv in enumerate(sol):
            if not live[s]:
                continue
            sv.step(1)
            ob = du.evaluate(sv.P, sv.st)[0]
            if abs(gb[s] - ob) > 1e-4:
                assert margins[s] < 1e-3, f"divergence at iteration {it} without a near-tie (margin {margins[s]})"
                assert it >= 10
                live[s] = False
    b, best = ctx.bound(best=True)
    for s, P in enumerate(Ps):
        if live[s]:
            assert b[s] == pytest.approx(sol[s].bound(), abs=1e-4)
            assert best[s] == pytest.approx(sol[s].best, abs=1e-4)
        assert best[s] >= P.ibp_output_bound() - 1e-6
        assert best[s] <= sample_min_output(P, 5000) + 1e-6


def _draw_sp_state(Ps, seed, t):
    """A random Saddle Point iterate for every subproblem (generator only) and its oracle solvers.
    Seeds are tried in order until every decision taken on a sum (f, xhat - x, the choice of
    eq. 12) clears 2e-6, the size of float32 summation error here; the other decisions (mask
    thresholds, the sign of G) are taken by identical float32 operations on both sides."""
    P0 = Ps[0]
    S, widths = len(Ps), P0.widths
    NT = sum(widths)
    NH, n0 = NT - widths[0], widths[0]
    lo = np.stack([np.concatenate(P.lo) for P in Ps]).astype(np.float32)
    hi = np.stack([np.concatenate(P.hi) for P in Ps]).astype(np.float32)
    offs = np.cumsum([0] + widths)
    for trial in range(20):
        rng = synth.SplitMix64(seed + 1000 * trial)
        u = lambda n: rng.uniform(n).astype(np.float32)
        x = (lo + u(S * NT).reshape(S, NT) * (hi - lo)).astype(np.float32)
        x = np.minimum(np.maximum(x, lo), hi)
        z = u(S * NH).reshape(S, NH)
        alpha = (u(S * NH) * 0.3).reshape(S, NH)
        Sb = (u(S * NH) * 0.5).reshape(S, NH)
        G = ((u(S * NH) - 0.5) * 2).reshape(S, NH)
        C = ((u(S * NH) - 0.5) * 0.2).reshape(S, NH)
        Pst = ((u(S * NT) - 0.5) * 0.5).reshape(S, NT)
        Pst[:, NT - widths[-1]:] = 0
        mua = (u(S * NH) * 0.3 + 0.01).reshape(S, NH)
        mub = (u(S * NH) * 0.5 + 0.01).reshape(S, NH)
        sps = []
        for s, P in enumerate(Ps):
            hid = lambda v: [None] + split_hidden(v[s].astype(np.float64), widths)[1:]
            Pk = [None] + [Pst[s, offs[k - 1]:offs[k]].astype(np.float64) for k in range(1, P.n)]
            xs = [x[s, offs[k]:offs[k + 1]].astype(np.float64) for k in range(P.n)]
            sps.append(SPm.SaddlePoint.from_state(P, AS.Options(), hid(alpha), hid(Sb), Pk, hid(G), hid(C),
                                                  hid(mua), hid(mub), xs, hid(z), t))
        if min(sp.decision_margin(sums_only=True) for sp in sps) > 2e-6:
            stats = np.zeros((4, S, NT), np.float32)
            stats[0, :, n0:], stats[1, :, n0:], stats[2, :, n0:], stats[3] = Sb, G, C, Pst
            return sps, dict(x=x, z=z, stats=stats, caps=np.stack([mua, mub]), alpha=alpha)
    raise AssertionError("no well-separated state found")


def _install_sp_state(ctx, st, t):
    ctx.set_state(binding.ST_ITER, np.array([0, t, 1], np.int32))
    ctx.set_state(binding.ST_SP_X, st["x"])
    ctx.set_state(binding.ST_SP_Z, st["z"])
    ctx.set_state(binding.ST_SP_STATS, st["stats"])
    ctx.set_state(binding.ST_SP_CAPS, st["caps"])
    ctx.set_state(binding.ST_ALPHA, st["alpha"])


@pytest.mark.parametrize("name,S,t", [("mlp_tiny", 1, 0), ("small_conv", 3, 4), ("mlp_5_7_6_3", 4, 7),
                                      ("small_conv", 2, 11)])
def test_saddle_point_one_iteration_lockstep(name, S, t):
    """One Saddle Point iteration (Alg. 2) from a random iterate drawn by the generator: bound,
    conditional-gradient choices (exact) and every updated quantity (1e-5 relative)."""
    prob, Ps0 = _problems(name, S)
    lh, uh = oracle_bounds_f32(Ps0)
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), Ps0[0].widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), Ps0[0].widths)[1:])
                                   for s in range(S)])
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0), bounds=(lh, uh))
    sps, st = _draw_sp_state(Ps, 50 + t, t)
    _install_sp_state(ctx, st, t)
    gb = ctx.bound()
    for s, sp in enumerate(sps):
        assert gb[s] == pytest.approx(sp.evaluate()[0], abs=1e-5, rel=1e-5)
    ctx.sp_step(1)
    it = ctx.get_state(binding.ST_ITER, np.int32)
    assert it[1] == t + 1 and it[2] == 1
    sel = ctx.get_state(binding.ST_SP_SEL, np.uint8).reshape(S, -1)
    x = ctx.get_state(binding.ST_SP_X).reshape(S, -1)
    z = ctx.get_state(binding.ST_SP_Z).reshape(S, -1)
    al = ctx.get_state(binding.ST_ALPHA).reshape(S, -1)
    stats = ctx.get_state(binding.ST_SP_STATS).reshape(4, S, -1)
    n0 = ctx.widths[0]
    for s, sp in enumerate(sps):
        sp.step(1)
        np.testing.assert_array_equal(sel[s], hidden_concat(sp.last_sel).astype(np.uint8))
        tol = dict(rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(x[s], np.concatenate(sp.x), **tol)
        np.testing.assert_allclose(z[s], hidden_concat(sp.z), **tol)
        np.testing.assert_allclose(al[s], hidden_concat(sp.alpha), **tol)
        np.testing.assert_allclose(stats[0, s, n0:], hidden_concat(sp.Sb), **tol)
        np.testing.assert_allclose(stats[1, s, n0:], hidden_concat(sp.G), **tol)
        np.testing.assert_allclose(stats[2, s, n0:], hidden_concat(sp.C), **tol)
        np.testing.assert_allclose(stats[3, s, :-ctx.widths[-1]],
                                   np.concatenate([sp.Pst[k] for k in range(1, sp.P.n)]), **tol)


@pytest.mark.parametrize("name,S", [("mlp_tiny", 1), ("small_conv", 3), ("mlp_5_7_6_3", 3)])
def test_saddle_point_conversion_from_active_set_state(name, S):
    """Sufficient statistics (eq. 10), price caps (eq. 16) and the closed-form starting primal
    computed from an Active Set state drawn by the generator."""
    prob, Ps0 = _problems(name, S)
    lh, uh = oracle_bounds_f32(Ps0)
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), Ps0[0].widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), Ps0[0].widths)[1:])
                                   for s in range(S)])
    kw = dict(bigm_iters=2, as_iters=30, omega=3, max_cuts=4, sp_init_steps=0)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, **kw), bounds=(lh, uh))
    solvers = draw_state(Ps, ctx, kw, it=9, nslots=4, seed=21)
    ctx.sp_step(0)
    stats = ctx.get_state(binding.ST_SP_STATS).reshape(4, S, -1)
    caps = ctx.get_state(binding.ST_SP_CAPS).reshape(2, S, -1)
    x = ctx.get_state(binding.ST_SP_X).reshape(S, -1)
    z = ctx.get_state(binding.ST_SP_Z).reshape(S, -1)
    n0 = ctx.widths[0]
    for s, sv in enumerate(solvers):
        sp = SPm.SaddlePoint(sv.P, AS.Options(**kw), sv.st)
        tol = dict(rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(stats[0, s, n0:], hidden_concat(sp.Sb), **tol)
        np.testing.assert_allclose(stats[1, s, n0:], hidden_concat(sp.G), **tol)
        np.testing.assert_allclose(stats[2, s, n0:], hidden_concat(sp.C), **tol)
        np.testing.assert_allclose(stats[3, s, :-ctx.widths[-1]],
                                   np.concatenate([sp.Pst[k] for k in range(1, sp.P.n)]), **tol)
        np.testing.assert_allclose(caps[0, s], hidden_concat(sp.mu_a), **tol)
        np.testing.assert_allclose(caps[1, s], hidden_concat(sp.mu_b), **tol)
        f = sp.coefficients()
        decided = np.concatenate([np.abs(fk) > 1e-5 for fk in f])
        np.testing.assert_array_equal(x[s][decided], np.concatenate(sp.x)[decided].astype(np.float32))
        np.testing.assert_array_equal(z[s], hidden_concat(sp.z).astype(np.float32))


@pytest.mark.parametrize("name,S", [("mlp_tiny", 1), ("small_conv", 2), ("mlp_3_4_4_1", 2)])
def test_free_running_saddle_point_tracks_oracle_until_a_tie(name, S):
    """Big-M initialisation, conversion, primal initialisation and SP iterations on both sides:
    bounds agree to 1e-4 until the oracle meets a decision within 1e-3 of a tie; every GPU bound
    stays a valid lower bound (below the sampled minimum of the network output)."""
    prob, Ps = _problems(name, S)
    kw = dict(bigm_iters=40, as_iters=0, sp_init_steps=20)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, **kw))
    ctx.as_step(40)
    refs = [AS.ActiveSet(P, AS.Options(**kw)).step(40) for P in Ps]
    ctx.sp_step(0)
    sps = [SPm.SaddlePoint(r.P, r.opt, r.st) for r in refs]
    live = [True] * S
    xg = ctx.get_state(binding.ST_SP_X).reshape(S, -1)
    for s, sp in enumerate(sps):
        if np.abs(xg[s] - np.concatenate(sp.x)).max() > 1e-4:
            live[s] = False   # primal initialisation met a tie (checked exactly in the lockstep)
    mins = [sample_min_output(P, 5000) for P in Ps]
    for t in range(30):
        margins = [sp.decision_margin() for sp in sps]
        ctx.sp_step(1)
        gb = ctx.bound()
        for s, sp in enumerate(sps):
            assert gb[s] <= mins[s] + 1e-6
            if not live[s]:
                continue
            sp.step(1)
            ob = sp.evaluate()[0]
            if abs(gb[s] - ob) > 1e-4:
                assert margins[s] < 1e-3, f"divergence at SP iteration {t} without a near-tie ({margins[s]})"
                live[s] = False


@pytest.mark.parametrize("name,S", [("mlp_5_7_6_3", 3), ("small_conv", 2)])
def test_bound_backward_matches_envelope_gradient(name, S):
    prob, Ps0 = _problems(name, S)
    lh, uh = oracle_bounds_f32(Ps0)
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), Ps0[0].widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), Ps0[0].widths)[1:])
                                   for s in range(S)])
    kw = dict(bigm_iters=2, as_iters=30, omega=3, max_cuts=4)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, **kw), bounds=(lh, uh))
    solvers = draw_state(Ps, ctx, kw, it=9, nslots=4, seed=7)
    rng = synth.SplitMix64(3)
    gb = rng.uniform(S) + 0.5
    net = prob["net"]
    dW = [np.zeros_like(L["W"]) for L in net]
    db = [np.zeros_like(L["b"]) for L in net]
    dlo = np.zeros_like(prob["lo"])
    dhi = np.zeros_like(prob["hi"])
    ctx.backward(gb, dW, db, dlo, dhi)
    refW = [np.zeros(L["W"].shape) for L in net]
    refb = [np.zeros(L["b"].shape) for L in net]
    for s, sv in enumerate(solvers):
        g = ev.envelope_gradient(sv.P, sv.st)
        for k, L in enumerate(net[:-1], start=1):
            if L["kind"] == "linear":
                refW[k - 1] += gb[s] * g["dW"][k]
            else:
                refW[k - 1] += gb[s] * ev.filter_gradient(g["dW"][k], sv.P.taps[k], L["W"].shape)
            refb[k - 1] += gb[s] * ev.bias_gradient(g["db"][k], L)
        refW[-1] += gb[s] * np.outer(prob["C"][s], g["dW"][sv.P.n][0])
        refb[-1] += gb[s] * prob["C"][s]
        np.testing.assert_allclose(dlo[s], gb[s] * g["dlo0"], rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(dhi[s], gb[s] * g["dhi0"], rtol=1e-4, atol=1e-5)
    for k in range(len(net)):
        np.testing.assert_allclose(dW[k], refW[k], rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(db[k], refb[k], rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("name,S,with_splits", [("mlp_5_7_6_3", 3, False), ("small_conv", 2, False),
                                                ("mlp_5_7_6_3", 3, True)])
def test_bound_backward_through_interval_propagation_matches_chain_gradient(name, S, with_splits):
    """as_bound_backward_ibp against the oracle's chain gradient: the context computes its own
    interval bounds (with split clamps); the oracle's Problems hold its float64 interval bounds
    rounded outward to float32 per layer. Tolerance as the fixed-bound backward: 1e-4 relative."""
    prob = synth.problem(name, S=S, seed=0)
    if with_splits:
        P0 = nw.problems(prob)
        NH = sum(L["n_out"] for L in prob["net"][:-1])
        sp = np.zeros((S, NH), np.int8)
        for s, P in enumerate(P0):
            l, u = np.concatenate(P.lhat[1:]), np.concatenate(P.uhat[1:])
            amb = np.flatnonzero((l < 0) & (u > 0))
            sp[s, amb[::3]] = 1
            sp[s, amb[1::3]] = -1
        prob = dict(prob, splits=sp)
    Ps0 = nw.problems(prob)
    lh, uh = oracle_bounds_f32(Ps0)
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), Ps0[0].widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), Ps0[0].widths)[1:])
                                   for s in range(S)])
    kw = dict(bigm_iters=2, as_iters=30, omega=3, max_cuts=4)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, **kw))
    solvers = draw_state(Ps, ctx, kw, it=9, nslots=4, seed=7)
    gb = synth.SplitMix64(3).uniform(S) + 0.5
    net = prob["net"]
    dW = [np.zeros_like(L["W"]) for L in net]
    db = [np.zeros_like(L["b"]) for L in net]
    dlo, dhi = np.zeros_like(prob["lo"]), np.zeros_like(prob["hi"])
    ctx.backward(gb, dW, db, dlo, dhi, through_bounds=True)
    refW = [np.zeros(L["W"].shape) for L in net]
    refb = [np.zeros(L["b"].shape) for L in net]
    for s, sv in enumerate(solvers):
        g = ev.chain_gradient(sv.P, sv.st, None if not with_splits else prob["splits"][s])
        for k, L in enumerate(net[:-1], start=1):
            if L["kind"] == "linear":
                refW[k - 1] += gb[s] * g["dW"][k]
            else:
                refW[k - 1] += gb[s] * ev.filter_gradient(g["dW"][k], sv.P.taps[k], L["W"].shape)
            refb[k - 1] += gb[s] * ev.bias_gradient(g["db"][k], L)
        refW[-1] += gb[s] * np.outer(prob["C"][s], g["dW"][sv.P.n][0])
        refb[-1] += gb[s] * prob["C"][s]
        np.testing.assert_allclose(dlo[s], gb[s] * g["dlo0"], rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(dhi[s], gb[s] * g["dhi0"], rtol=1e-4, atol=1e-5)
    for k in range(len(net)):
        np.testing.assert_allclose(dW[k], refW[k], rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(db[k], refb[k], rtol=1e-4, atol=1e-5)
    # caller-given bounds have no interval propagation to differentiate
    ctx2 = binding.context_for(prob, binding.default_options(graph_chunk=0, **kw), bounds=(lh, uh))
    with pytest.raises(binding.CBError):
        ctx2.backward(gb, dW, db, dlo, dhi, through_bounds=True)


def test_invalid_arguments_are_rejected_before_any_kernel():
    prob = synth.problem("mlp_tiny", seed=0)
    bad = dict(prob)
    bad["lo"] = prob["hi"] + 1.0
    with pytest.raises(binding.CBError) as e:
        binding.context_for(bad)
    assert e.value.code == binding.AS_ERR_ARG
    with pytest.raises(binding.CBError) as e:
        binding.context_for(prob, binding.default_options(max_cuts=9))
    assert e.value.code == binding.AS_ERR_ARG
    ctx = binding.context_for(prob, binding.default_options(bigm_iters=2, as_iters=2))
    ctx.as_step(2)
    ctx.sp_step(1)
    with pytest.raises(binding.CBError) as e:
        ctx.as_step(1)
    assert e.value.code == binding.AS_ERR_STATE


def test_runs_are_deterministic():
    prob = synth.problem("small_conv", S=3, seed=2)
    out = []
    for _ in range(2):
        ctx = binding.context_for(prob, binding.default_options(bigm_iters=10, as_iters=30, omega=8, max_cuts=4))
        ctx.as_step(40)
        out.append((ctx.bound(), ctx.get_state(binding.ST_SLOT_BETA).tobytes()))
    assert (out[0][0] == out[1][0]).all() and out[0][1] == out[1][1]


@pytest.mark.parametrize("it,nslots", [(236, 4), (240, 4)])
def test_full_size_wide_conv_lockstep_on_sampled_subproblems(it, nslots):
    """The bench workload at full size (Wide conv net, 9 properties), in the bench's launch
    configuration: one Active Set iteration from a drawn state with 4 filled slots (omega 20:
    iteration 236 is ordinary, 240 adds slot 4), every dual of two sampled subproblems against the
    oracle (the oracle's dense conv operators are large)."""
    prob = synth.problem("wide_conv", seed=0)
    dense = nw.dense_layers(prob["net"])
    Ps0 = nw.problems(prob, dense=dense)
    lh, uh = oracle_bounds_f32(Ps0)
    widths = Ps0[0].widths
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), widths)[1:]) for s in range(9)],
                     dense=dense)
    kw = dict(bigm_iters=200, as_iters=800, omega=20, max_cuts=5)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=25, **kw), bounds=(lh, uh))
    sample = {0, 5}
    solvers = draw_state(Ps, ctx, kw, it, nslots, seed=300 + it, subset=sample)
    gb = ctx.bound()
    for s, sv in solvers.items():
        assert gb[s] == pytest.approx(du.evaluate(sv.P, sv.st)[0], abs=1e-4, rel=1e-5)
    ctx.as_step(1)
    S = 9
    st = {key: ctx.get_state(code).reshape(S, -1) for key, code in
          (("alpha", binding.ST_ALPHA), ("beta0", binding.ST_BETA0), ("beta1", binding.ST_BETA1),
           ("xstar", binding.ST_XSTAR))}
    sb = ctx.get_state(binding.ST_SLOT_BETA).reshape(S, ctx.cap, -1)
    for s, sv in solvers.items():
        # wide rows (fan-in up to 2048) widen the float32 bound: at least 80% of the entries are
        # checked at the rounding tolerance itself, the rest within the spread it allows
        res = check_active_set_step(sv, dict(alpha=st["alpha"][s], beta0=st["beta0"][s], beta1=st["beta1"][s],
                                             slots=sb[s], xstar=st["xstar"][s]), min_tight=0.8)
        assert res["checked"] >= 0.9 * 3 * res["rows"]


C4_KW = dict(bigm_iters=100, as_iters=400, omega=120, max_cuts=5)   # the default bench schedule


@pytest.mark.parametrize("it,nslots", [(340, 4)])
def test_full_size_conv4_lockstep_on_sampled_boxes(it, nslots):
    """The default bench workload at full size (conv4 net, 1024 boxes) in the float32 form and the
    bench's launch configuration: one Active Set iteration from a drawn state with 4 filled slots
    (omega 120: iteration 340 adds slot 4), every dual of two sampled boxes against the oracle."""
    sample = {0, 777}
    ctx, Ps = conv4_full_batch(32, C4_KW, sample)
    solvers = draw_state(Ps, ctx, C4_KW, it, nslots, seed=500 + it, subset=sample)
    gb = ctx.bound()
    for s, sv in solvers.items():
        assert gb[s] == pytest.approx(du.evaluate(sv.P, sv.st)[0], abs=1e-4, rel=1e-5)
    ctx.as_step(1)
    S = ctx.S
    st = {key: ctx.get_state(code).reshape(S, -1) for key, code in
          (("alpha", binding.ST_ALPHA), ("beta0", binding.ST_BETA0), ("beta1", binding.ST_BETA1),
           ("xstar", binding.ST_XSTAR))}
    sb = ctx.get_state(binding.ST_SLOT_BETA).reshape(S, ctx.cap, -1)
    for s, sv in solvers.items():
        # conv rows have fan-in 27-576 and FC rows 4096: at least 80% of the entries are checked at
        # the rounding tolerance itself, the rest within the spread it allows
        res = check_active_set_step(sv, dict(alpha=st["alpha"][s], beta0=st["beta0"][s], beta1=st["beta1"][s],
                                             slots=sb[s], xstar=st["xstar"][s]), min_tight=0.8)
        assert res["checked"] >= 0.9 * 3 * res["rows"]


def test_batched_subdomains_lockstep_with_splits_and_caps():
    """The batching workload at full size: 4096 branch-and-bound subdomains of the Wide conv
    net with random ReLU splits and per-subdomain caps of 1-5 masks, in the bench's graph launch
    configuration. Interval bounds with the splits, and one Active Set iteration (an addition
    iteration, so that capped subdomains must skip the new slot) from a drawn state, checked on
    sampled subdomains of different caps."""
    prob = synth.problem("wide_conv_bab", S=4096, seed=0)
    caps = prob["caps"]
    sample = sorted({int(np.argmax(caps == c)) for c in (1, 2, 3, 5)})
    dense = nw.dense_layers(prob["net"])
    sub = dict(prob)
    for key in ("lo", "hi", "C", "splits"):
        sub[key] = prob[key][sample]
    Ps_s = nw.problems(sub, dense=dense)       # interval bounds with the splits, sampled only
    kw = dict(bigm_iters=100, as_iters=400, omega=20, max_cuts=5)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=25, **kw))
    lh = ctx.get_state(binding.ST_LHAT).reshape(4096, -1)
    uh = ctx.get_state(binding.ST_UHAT).reshape(4096, -1)
    for q, s in enumerate(sample):
        rl, ru = hidden_concat(Ps_s[q].lhat), hidden_concat(Ps_s[q].uhat)
        assert (lh[s] <= rl + 1e-9 * (1 + np.abs(rl))).all() and (uh[s] >= ru - 1e-9 * (1 + np.abs(ru))).all()
        assert (np.abs(lh[s] - rl) <= 4e-6 * (1 + np.abs(rl))).all()
        assert (np.abs(uh[s] - ru) <= 4e-6 * (1 + np.abs(ru))).all()
    # the oracle on the sampled subdomains, with the GPU's own interval bounds reproduced in FP64
    # by the oracle above (rounded outward to float32 as both sides use them)
    lh32, uh32 = oracle_bounds_f32(Ps_s)
    widths = Ps_s[0].widths
    Ps = [nw.Problem(prob["net"], prob["lo"][s], prob["hi"][s], prob["C"][s],
                     bounds=(split_hidden(lh32[q].astype(np.float64), widths)[1:],
                             split_hidden(uh32[q].astype(np.float64), widths)[1:]), dense=dense)
          for q, s in enumerate(sample)]
    it = 140   # t = 40: adds slot 4 (omega 20), which only caps of 5 accept
    full_ps = [None] * 4096
    for q, s in enumerate(sample):
        full_ps[s] = Ps[q]
    # install the same float32 bounds on the sampled subdomains of the GPU side
    lh2, uh2 = lh.copy(), uh.copy()
    lh2[sample], uh2[sample] = lh32, uh32
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=25, **kw), bounds=(lh2, uh2))
    solvers = draw_state(full_ps, ctx, kw, it, 4, seed=41, subset=set(sample))
    sbeta = ctx.get_state(binding.ST_SLOT_BETA).reshape(4096, ctx.cap, -1)
    for s in range(4096):
        sbeta[s, int(caps[s]):] = 0.0          # a subdomain never holds slots beyond its cap
    ctx.set_state(binding.ST_SLOT_BETA, sbeta)
    for s, sv in solvers.items():
        sv.cap = int(caps[s])
        # slots beyond a subdomain's cap were never added: drop them on the oracle side too
        for k in range(1, sv.P.n):
            del sv.st.slots[k][int(caps[s]):]
    ctx.as_step(1)
    st = {key: ctx.get_state(code).reshape(4096, -1) for key, code in
          (("alpha", binding.ST_ALPHA), ("beta0", binding.ST_BETA0), ("beta1", binding.ST_BETA1),
           ("xstar", binding.ST_XSTAR))}
    sb = ctx.get_state(binding.ST_SLOT_BETA).reshape(4096, ctx.cap, -1)
    for s, sv in solvers.items():
        # wide rows (fan-in up to 2048) widen the float32 bound: at least 80% of the entries are
        # checked at the rounding tolerance itself, the rest within the spread it allows
        res = check_active_set_step(sv, dict(alpha=st["alpha"][s], beta0=st["beta0"][s], beta1=st["beta1"][s],
                                             slots=sb[s], xstar=st["xstar"][s]), min_tight=0.8)
        assert res["checked"] >= 0.9 * 3 * res["rows"]
        nslots = len(sv.st.slots[1])
        assert nslots == min(int(caps[s]), 5)
        for b in range(nslots, ctx.cap):
            assert (sb[s, b] == 0).all()      # capped: the slot stays empty


def test_autotune_picks_a_candidate_and_starts_from_zero_duals():
    """as_options.autotune times team-size targets with real iterations at init, then reloads the
    batch: the context starts at zero duals (the interval bound) and iterates to valid bounds."""
    prob, Ps = _problems("small_conv", 3)
    kw = dict(bigm_iters=10, as_iters=30, omega=8, max_cuts=5)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, autotune=1, **kw))
    cands = {5000, 10000, 20000, 40000, 80000, 160000, 320000}
    row, col = ctx.team_targets()
    assert row in cands and col in cands
    b0 = ctx.bound()
    for s, P in enumerate(Ps):
        assert b0[s] == pytest.approx(P.ibp_output_bound(), abs=1e-4, rel=1e-5)
    ctx.as_step(40)
    b = ctx.bound()
    for s, P in enumerate(Ps):
        assert b0[s] - 1e-6 <= b[s] <= sample_min_output(P, 5000) + 1e-6
    plain = binding.context_for(prob, binding.default_options(graph_chunk=0, **kw))
    assert plain.team_targets() == (40000, 40000)

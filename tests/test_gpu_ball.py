"""Parity of the ellipsoid (l2-ball) input set, as_options.input_l2, with the oracle.

Tolerances as for the box (tests/test_gpu_parity.py): interval bounds contain the FP64 ones and are
within 4e-6 (1 + |v|); one-iteration lockstep of the duals 1e-5 relative where the update direction
is decided; bounds 1e-4 absolute / 1e-5 relative. x_0* is no longer a box vertex: it is compared
to 1e-5 relative (float32 f_0 against FP64), the hidden layers' x*, z* exactly.
"""
import numpy as np
import pytest

from oracle import active_set as AS
from oracle import bab
from oracle import dual as du
from oracle import envelope as ev
from oracle import network as nw
from oracle import relaxation as rx
from paper_2101_05844_gb300 import binding, synth
from tests.state_helpers import draw_state, hidden_concat, oracle_bounds_f32, split_hidden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    binding.lib()


def _ball(name, S, seed=0, equal=False):
    prob = synth.problem(name, S=S, seed=seed)
    lo, hi = prob["lo"].astype(np.float64), prob["hi"].astype(np.float64)
    c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
    if not equal:
        e = e * (0.5 + synth.SplitMix64(seed + 7).uniform(e.size).reshape(e.shape))
    return dict(prob, lo=(c - e).astype(np.float32), hi=(c + e).astype(np.float32), ball=True)


def _opts(**kw):
    return binding.default_options(graph_chunk=0, input_l2=1, **kw)


@pytest.mark.parametrize("name,S", [("mlp_5_7_6_3", 3), ("small_conv", 2)])
def test_interval_bounds_over_the_ellipsoid(name, S):
    prob = _ball(name, S)
    ctx = binding.context_for(prob, _opts())
    lh = ctx.get_state(binding.ST_LHAT).reshape(S, -1)
    uh = ctx.get_state(binding.ST_UHAT).reshape(S, -1)
    for s, P in enumerate(nw.problems(prob)):
        rl, ru = hidden_concat(P.lhat), hidden_concat(P.uhat)
        assert np.all(lh[s] <= rl) and np.all(uh[s] >= ru)
        np.testing.assert_allclose(lh[s], rl, rtol=0, atol=4e-6 * (1 + np.abs(rl)).max())
        np.testing.assert_allclose(uh[s], ru, rtol=0, atol=4e-6 * (1 + np.abs(ru)).max())
    box = binding.context_for(dict(prob, ball=False), binding.default_options(graph_chunk=0))
    assert np.all(lh >= box.get_state(binding.ST_LHAT).reshape(S, -1))


CASES = [
    ("mlp_tiny", 1, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 3, 0),     # Big-M
    ("mlp_tiny", 1, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 8, 2),     # adds slot 2
    ("small_conv", 3, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 12, 4),  # adds slot 4
    ("mlp_5_7_6_3", 4, dict(bigm_iters=2, as_iters=30, omega=4, max_cuts=8), 16, 6),  # adds slot 6
]


@pytest.mark.parametrize("name,S,kw,it,nslots", CASES)
def test_one_iteration_lockstep(name, S, kw, it, nslots):
    prob = _ball(name, S)
    Ps0 = nw.problems(prob)
    lh, uh = oracle_bounds_f32(Ps0)
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), Ps0[0].widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), Ps0[0].widths)[1:])
                                   for s in range(S)])
    ctx = binding.context_for(prob, _opts(**kw), bounds=(lh, uh))
    solvers = draw_state(Ps, ctx, kw, it, nslots, seed=200 + it, interior0=True)
    gb = ctx.bound()
    for s, sv in enumerate(solvers):
        assert gb[s] == pytest.approx(du.evaluate(sv.P, sv.st)[0], abs=1e-4, rel=1e-5)
    ctx.as_step(1)
    xstar = ctx.get_state(binding.ST_XSTAR).reshape(S, -1)
    zstar = ctx.get_state(binding.ST_ZSTAR, np.uint8).reshape(S, -1)
    al = ctx.get_state(binding.ST_ALPHA).reshape(S, -1)
    b0 = ctx.get_state(binding.ST_BETA0).reshape(S, -1)
    b1 = ctx.get_state(binding.ST_BETA1).reshape(S, -1)
    sb = ctx.get_state(binding.ST_SLOT_BETA).reshape(S, ctx.cap, -1)
    lam = ctx.get_state(binding.ST_LAMBDA).reshape(S, ctx.cap, -1)
    kap = ctx.get_state(binding.ST_KAPPA).reshape(S, ctx.cap, -1)
    n0 = Ps[0].widths[0]
    for s, sv in enumerate(solvers):
        P = sv.P
        _, f, g, x, z = du.evaluate(P, sv.st)
        grads = du.supergradient(P, sv.st, x, z)
        before = len(sv.st.slots[1])
        sv.step(1)
        np.testing.assert_allclose(xstar[s, :n0], x[0], rtol=1e-5, atol=1e-6)
        np.testing.assert_array_equal(xstar[s, n0:], np.concatenate([x[k] for k in range(1, P.n)]).astype(np.float32))
        np.testing.assert_array_equal(zstar[s], hidden_concat(z).astype(np.uint8))
        if len(sv.st.slots[1]) > before:   # the new slot's lambda, kappa (float32 recompute)
            b = before
            ref_l = hidden_concat([None] + [sv.st.slots[k][b].lam for k in range(1, P.n)])
            ref_k = hidden_concat([None] + [sv.st.slots[k][b].lam + sv.st.slots[k][b].mu + P.b[k]
                                            for k in range(1, P.n)])
            np.testing.assert_allclose(lam[s, b], ref_l, rtol=1e-5, atol=1e-5)
            np.testing.assert_allclose(kap[s, b], ref_k, rtol=1e-5, atol=1e-5)
            I1 = sv.st.slots[1][b].I   # interior x_0*: the layer-1 mask is z (or 1 where W = 0)
            np.testing.assert_array_equal(I1, (z[1][:, None] > 0) | (P.W[1] == 0) | (P.lo[0] == P.hi[0])[None, :])

        def check(gpu, ref, gref):
            decided = (np.abs(gref) > 1e-4) | (gref == 0)
            np.testing.assert_allclose(gpu[decided], ref[decided], rtol=1e-5, atol=1e-7)
            assert (gpu >= 0).all() and decided.mean() > 0.9
        check(al[s], hidden_concat(sv.st.alpha), hidden_concat(grads["galpha"]))
        check(b0[s], hidden_concat(sv.st.beta0), hidden_concat(grads["gbeta0"]))
        check(b1[s], hidden_concat(sv.st.beta1), hidden_concat(grads["gbeta1"]))
        for b in range(before):
            check(sb[s, b], hidden_concat([None] + [sv.st.slots[k][b].beta for k in range(1, P.n)]),
                  hidden_concat([None] + [grads["gslots"][k][b] for k in range(1, P.n)]))


def _as_margin(sv):
    _, f, g, x, z = du.evaluate(sv.P, sv.st)
    m = min(np.abs(fk).min() for fk in f[1:]) if len(f) > 1 else np.inf
    for gk in g[1:]:
        nz = gk[gk != 0]
        if nz.size:
            m = min(m, np.abs(nz).min())
    return m


@pytest.mark.parametrize("name,S,kw,iters", [
    ("mlp_tiny", 1, dict(bigm_iters=20, as_iters=80, omega=24, max_cuts=5), 100),
    ("mlp_5_7_6_3", 4, dict(bigm_iters=30, as_iters=60, omega=20, max_cuts=4), 90),
    ("small_conv", 3, dict(bigm_iters=20, as_iters=40, omega=12, max_cuts=5), 60),
])
def test_free_running_active_set_matches_oracle(name, S, kw, iters):
    """Iteration by iteration from zero duals: bounds within 1e-4 until the oracle takes a decision
    within 1e-3 of a tie (then both runs go on as different valid runs); every bound lies below
    the sampled minimum over the ellipsoid."""
    prob = _ball(name, S)
    Ps0 = nw.problems(prob)
    lh, uh = oracle_bounds_f32(Ps0)
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), Ps0[0].widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), Ps0[0].widths)[1:])
                                   for s in range(S)])
    ctx = binding.context_for(prob, _opts(track_best=1, **kw), bounds=(lh, uh))
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
            if abs(gb[s] - du.evaluate(sv.P, sv.st)[0]) > 1e-4:
                assert margins[s] < 1e-3, f"divergence at iteration {it} without a near-tie"
                assert it >= 10
                live[s] = False
    b, best = ctx.bound(best=True)
    dense = nw.dense_layers(prob["net"])
    rng = synth.SplitMix64(4)
    for s, P in enumerate(Ps):
        lo, hi = P.lo[0], P.hi[0]
        c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
        g = rng.normal(2000 * lo.size).reshape(2000, lo.size)
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        X = c + e * g * (rng.uniform(2000) ** (1.0 / lo.size))[:, None]
        m = min(float(prob["C"][s] @ bab.forward(dense, x)) for x in X)
        assert best[s] <= m + 1e-5


@pytest.mark.parametrize("chain", [False, True])
def test_backward_over_the_ellipsoid_matches_oracle(chain):
    """dW, db, dlo, dhi of the bound over the ellipsoid against the oracle's envelope gradient (the
    box endpoints give c and e), with the intermediate bounds held (caller bounds) or carried
    through interval propagation (the context's own bounds, layer 1 over the ellipsoid): 1e-4
    relative, as for the box."""
    name, S = "mlp_5_7_6_3", 3
    prob = _ball(name, S)
    Ps0 = nw.problems(prob)
    lh, uh = oracle_bounds_f32(Ps0)
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), Ps0[0].widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), Ps0[0].widths)[1:])
                                   for s in range(S)])
    kw = dict(bigm_iters=2, as_iters=30, omega=3, max_cuts=4)
    ctx = binding.context_for(prob, _opts(**kw), bounds=None if chain else (lh, uh))
    solvers = draw_state(Ps, ctx, kw, it=9, nslots=4, seed=7, interior0=True)
    gb = synth.SplitMix64(3).uniform(S) + 0.5
    net = prob["net"]
    dW = [np.zeros_like(L["W"]) for L in net]
    db = [np.zeros_like(L["b"]) for L in net]
    dlo, dhi = np.zeros_like(prob["lo"]), np.zeros_like(prob["hi"])
    ctx.backward(gb, dW, db, dlo, dhi, through_bounds=chain)
    refW = [np.zeros(L["W"].shape) for L in net]
    refb = [np.zeros(L["b"].shape) for L in net]
    for s, sv in enumerate(solvers):
        g = ev.chain_gradient(sv.P, sv.st) if chain else ev.envelope_gradient(sv.P, sv.st)
        for k in range(1, len(net)):
            refW[k - 1] += gb[s] * g["dW"][k]
            refb[k - 1] += gb[s] * g["db"][k]
        refW[-1] += gb[s] * np.outer(prob["C"][s], g["dW"][sv.P.n][0])
        refb[-1] += gb[s] * prob["C"][s]
        np.testing.assert_allclose(dlo[s], gb[s] * g["dlo0"], rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(dhi[s], gb[s] * g["dhi0"], rtol=1e-4, atol=1e-5)
    for k in range(len(net)):
        np.testing.assert_allclose(dW[k], refW[k], rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(db[k], refb[k], rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("name,S,kw", [
    ("mlp_5_7_6_3", 4, dict(bigm_iters=30, as_iters=60, omega=20, max_cuts=4)),
    ("small_conv", 3, dict(bigm_iters=20, as_iters=40, omega=12, max_cuts=5)),
])
def test_bf16_form_over_the_ellipsoid(name, S, kw):
    """The BF16 form over the ellipsoid: the bound (re-evaluated in float32) lies below the sampled
    minimum over the ellipsoid and within 1e-2 (per unit of 1 + |bound|) of the oracle's FP64 run,
    the bound the BF16 suite sets for the box; graph replay equals plain launches."""
    prob = _ball(name, S)
    Ps = nw.problems(prob)
    iters = kw["bigm_iters"] + kw["as_iters"]
    ctx = binding.context_for(prob, _opts(precision=16, **kw))
    ctx.as_step(iters)
    b = ctx.bound()
    dense = nw.dense_layers(prob["net"])
    rng = synth.SplitMix64(12)
    for s, P in enumerate(Ps):
        ref = AS.ActiveSet(P, AS.Options(**kw)).step(iters).bound()
        assert abs(b[s] - ref) / (1 + abs(ref)) <= 1e-2
        n0 = P.widths[0]
        c, e = 0.5 * (P.lo[0] + P.hi[0]), 0.5 * (P.hi[0] - P.lo[0])
        g = rng.normal(2000 * n0).reshape(2000, n0)
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        X = c + e * g * (rng.uniform(2000) ** (1.0 / n0))[:, None]
        assert b[s] <= min(float(prob["C"][s] @ bab.forward(dense, x)) for x in X) + 1e-6
    g = binding.context_for(prob, binding.default_options(graph_chunk=10, input_l2=1, precision=16, **kw))
    a = binding.context_for(prob, _opts(precision=16, **kw))
    g.as_step(iters)
    a.as_step(iters)
    np.testing.assert_array_equal(a.bound(), g.bound())


@pytest.mark.parametrize("name,S", [("mlp_tiny", 1), ("small_conv", 2), ("mlp_5_7_6_3", 3)])
def test_saddle_point_over_the_ellipsoid_tracks_oracle_until_a_tie(name, S):
    """Big-M, conversion, primal initialisation (x_0 retracted into the ellipsoid) and Saddle Point
    iterations on both sides: bounds agree to 1e-4 until the oracle meets a decision within 1e-3 of
    a tie; x_0 stays in the ellipsoid and every bound below the sampled minimum over it."""
    from oracle import saddle as SPm
    prob = _ball(name, S)
    Ps = nw.problems(prob)
    kw = dict(bigm_iters=40, as_iters=0, sp_init_steps=20)
    ctx = binding.context_for(prob, _opts(**kw))
    ctx.as_step(40)
    refs = [AS.ActiveSet(P, AS.Options(**kw)).step(40) for P in Ps]
    ctx.sp_step(0)
    sps = [SPm.SaddlePoint(r.P, r.opt, r.st) for r in refs]
    n0 = Ps[0].widths[0]
    xg = ctx.get_state(binding.ST_SP_X).reshape(S, -1)
    live = [bool(np.abs(xg[s] - np.concatenate(sp.x)).max() <= 1e-4) for s, sp in enumerate(sps)]
    assert any(live)
    dense = nw.dense_layers(prob["net"])
    rng = synth.SplitMix64(6)
    mins = []
    for s, P in enumerate(Ps):
        c, e = 0.5 * (P.lo[0] + P.hi[0]), 0.5 * (P.hi[0] - P.lo[0])
        g = rng.normal(2000 * n0).reshape(2000, n0)
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        X = c + e * g * (rng.uniform(2000) ** (1.0 / n0))[:, None]
        mins.append(min(float(prob["C"][s] @ bab.forward(dense, x)) for x in X))
    for t in range(30):
        margins = [sp.decision_margin() for sp in sps]
        ctx.sp_step(1)
        gb = ctx.bound()
        xg = ctx.get_state(binding.ST_SP_X).reshape(S, -1)
        for s, sp in enumerate(sps):
            P = Ps[s]
            c, e = 0.5 * (P.lo[0] + P.hi[0]), 0.5 * (P.hi[0] - P.lo[0])
            assert np.sum(((xg[s, :n0] - c) / e) ** 2) <= 1 + 1e-4
            assert gb[s] <= mins[s] + 1e-6
            if not live[s]:
                continue
            sp.step(1)
            if abs(gb[s] - sp.evaluate()[0]) > 1e-4:
                assert margins[s] < 1e-3, f"divergence at SP iteration {t} without a near-tie ({margins[s]})"
                live[s] = False


def test_intermediate_bounds_over_the_ellipsoid_match_oracle():
    """Layer 2 (solves over the interval bounds of layer 1, the same on both sides) within
    1e-4 (1 + max |v|). Over an ellipsoid x_0* moves continuously with f_0, so the float32 runs drift
    from the FP64 ones by the float32 rounding of f_0 at every iteration, where box vertices absorb
    it; deeper layers start from layer-2 bounds that already carry that drift, amplified by the
    weights (sum |w| about 8 on the conv net's FC layer): 5e-3 (1 + max |v|) there. Every bound
    holds the pre-activations of inputs sampled in the ellipsoid."""
    from oracle import intermediate as IM
    kw = dict(bigm_iters=12, as_iters=8, omega=4, max_cuts=3)
    for name, S in (("mlp_4_3_3_3_1", 2), ("small_conv", 2)):
        prob = _ball(name, S, seed=3)
        lh, uh = binding.intermediate_bounds(prob["net"], prob["lo"], prob["hi"], None, _opts(**kw))
        rl, ru = IM.batch(prob, AS.Options(**kw))
        widths = [L["n_out"] for L in prob["net"][:-1]]
        o1, o2 = widths[0], widths[0] + widths[1]
        for g, r in ((lh, rl), (uh, ru)):
            np.testing.assert_allclose(g[:, :o2], r[:, :o2], rtol=0, atol=1e-4 * (1 + np.abs(r[:, :o2])).max())
            np.testing.assert_allclose(g[:, o2:], r[:, o2:], rtol=0, atol=5e-3 * (1 + np.abs(r[:, o2:])).max())
        dense = nw.dense_layers(prob["net"])
        rng = synth.SplitMix64(9)
        for s in range(S):
            lo, hi = prob["lo"][s].astype(np.float64), prob["hi"][s].astype(np.float64)
            c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
            g = rng.normal(1000 * lo.size).reshape(1000, lo.size)
            g /= np.linalg.norm(g, axis=1, keepdims=True)
            h = (c + e * g * (rng.uniform(1000) ** (1.0 / lo.size))[:, None]).T
            pre = []
            for W, b, _ in dense[:-1]:
                a = W @ h + b[:, None]
                pre.append(a)
                h = np.maximum(a, 0.0)
            a = np.concatenate(pre)
            assert np.all(a.min(axis=1) >= lh[s] - 1e-5) and np.all(a.max(axis=1) <= uh[s] + 1e-5)


@pytest.mark.parametrize("seed,verdict", [(4, "verified"), (4, "falsified"), (7, "verified")])
def test_branch_and_bound_over_the_ellipsoid_matches_oracle(seed, verdict):
    prob = _ball("mlp_4_5_5_1", 1, seed=seed)
    lo, hi = prob["lo"][0].astype(np.float64), prob["hi"][0].astype(np.float64)
    dense = nw.dense_layers(prob["net"])
    rng = synth.SplitMix64(seed)
    c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
    g = rng.normal(4000 * lo.size).reshape(4000, lo.size)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    X = c + e * g * (rng.uniform(4000) ** (1.0 / lo.size))[:, None]
    vals = np.array([bab.forward(dense, x)[0] for x in X])
    t = vals.min() - 0.1 * np.ptp(vals) if verdict == "verified" else 0.5 * (vals.min() + vals.max())
    net = [dict(L) for L in prob["net"]]
    net[-1]["b"] = (net[-1]["b"].astype(np.float64) - t).astype(np.float32)
    loose = dict(bigm_iters=100, as_iters=0, input_l2=1)
    tight = dict(bigm_iters=50, as_iters=100, omega=30, max_cuts=3, input_l2=1)
    res = binding.bab(net, prob["lo"][0], prob["hi"][0], None,
                      binding.bab_default_options(loose=loose, tight=tight, batch=8, max_domains=600, cost_ratio=4.0))
    ref = bab.BaB(net, lo, hi, np.ones(1), bab.BabOptions(
        loose=AS.Options(bigm_iters=100), tight=AS.Options(bigm_iters=50, as_iters=100, omega=30, max_cuts=3),
        batch=8, max_domains=600), ball=True).run()
    assert ref["status"] == verdict and res["status"] == verdict
    if verdict == "falsified":
        x = res["x"].astype(np.float64)
        assert np.sum(((x - c) / e) ** 2) <= 1 + 1e-5
        assert bab.forward(nw.dense_layers(net), x)[0] < 0
    else:
        assert res["lower"] > 0

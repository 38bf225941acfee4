"""Pins of the oracle's Saddle Point (Alg. 2), its sufficient statistics (eq. 10, Fact 3), the
envelope gradient, and the dense conv operators."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import active_set as AS
from oracle import dual as du
from oracle import envelope as ev
from oracle import network as nw
from oracle import saddle as SPm
from paper_2101_05844_gb300 import synth
from tests.helpers import fig4_problem, netlp_for, sample_min_output


def test_sufficient_statistics_equal_explicit_beta_sums():
    """Fact 3: the statistics carried by Saddle Point equal the sums over the explicit (sparse)
    list of beta variables, after conversion from an Active Set state and after SP steps."""
    prob = synth.problem("mlp_4_5_5_1", seed=1)
    P = nw.problems(prob)[0]
    s = AS.ActiveSet(P, AS.Options(bigm_iters=30, as_iters=30, omega=10, max_cuts=3)).step(60)
    sp = SPm.SaddlePoint(P, s.opt, s.st, explicit=True)
    for steps in (0, 25):
        sp.step(steps)
        Sb, Pk, G, C = sp.explicit_stats()
        for k in range(1, P.n):
            np.testing.assert_allclose(Sb[k], sp.Sb[k], rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(Pk[k], sp.Pst[k], rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(G[k], sp.G[k], rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(C[k], sp.C[k], rtol=1e-12, atol=1e-12)


def test_saddle_point_bound_from_statistics_equals_active_set_bound_at_conversion():
    prob = synth.problem("small_conv", seed=2)
    P = nw.problems(prob)[0]
    s = AS.ActiveSet(P, AS.Options(bigm_iters=20, as_iters=20, omega=8, max_cuts=3)).step(40)
    sp = SPm.SaddlePoint(P, s.opt, s.st)
    # duals unchanged by conversion and primal init: same bound from the statistics
    assert sp.evaluate()[0] == pytest.approx(s.bound(), rel=1e-12, abs=1e-12)


def test_saddle_point_bounds_are_valid_and_below_lp():
    prob = synth.problem("mlp_3_4_4_1", seed=8)
    P = nw.problems(prob)[0]
    vA = float(netlp_for(P).solve("A", P.W[P.n][0], P.b[P.n][0]))
    s = AS.ActiveSet(P, AS.Options(bigm_iters=200)).step(200)
    sp = SPm.SaddlePoint(P, s.opt, s.st).step(300)
    sp.bound()
    assert max(sp.trace) <= vA + 1e-9 and sp.best <= vA + 1e-9
    assert sp.best <= sample_min_output(P, 20000) + 1e-9


def test_saddle_point_conditional_gradient_is_a_vertex_of_the_capped_domain():
    """eqs. (11)-(12): alpha_bar in {0, mu_alpha}; per neuron at most one beta at mu_beta."""
    prob = synth.problem("mlp_tiny", seed=3)
    P = nw.problems(prob)[0]
    s = AS.ActiveSet(P, AS.Options(bigm_iters=50)).step(50)
    sp = SPm.SaddlePoint(P, s.opt, s.st)
    sb0 = [None] + [sp.Sb[k].copy() for k in range(1, P.n)]
    sp.step(1)
    g = 1.0 / sp.opt.sp_gamma0
    for k in range(1, P.n):
        sbar = (sp.Sb[k] - (1 - g) * sb0[k]) / g
        ok = np.isclose(sbar, 0, atol=1e-12) | np.isclose(sbar, sp.mu_b[k], rtol=1e-10)
        assert ok.all()
        assert (sp.Sb[k] <= sp.mu_b[k] * (1 + 1e-12) + 1e-15).all()


@pytest.mark.parametrize("name", ["mlp_4_5_5_1", "small_conv"])
def test_envelope_gradient_matches_finite_differences(name):
    prob = synth.problem(name, seed=4)
    P = nw.problems(prob)[0]
    s = AS.ActiveSet(P, AS.Options(bigm_iters=30, as_iters=30, omega=10, max_cuts=3)).step(60)
    st = s.st
    grad = ev.envelope_gradient(P, st)
    rng = synth.SplitMix64(7)
    h = 1e-6

    def bound_with(mod):
        Q = nw.Problem.__new__(nw.Problem)
        Q.__dict__.update(P.__dict__)
        Q.W = [None if w is None else w.copy() for w in P.W]
        Q.b = [None if w is None else w.copy() for w in P.b]
        Q.lo = [v.copy() for v in P.lo]
        Q.hi = [v.copy() for v in P.hi]
        mod(Q)
        st2 = du.DualState(st.alpha, st.beta0, st.beta1, [[] for _ in range(P.n)])
        for k in range(1, P.n):
            for sl in st.slots[k]:
                du.add_slot(Q, st2, k, sl.I, beta=sl.beta)
        return du.evaluate(Q, st2)[0]

    checks = 0
    for k in range(1, P.n + 1):
        for _ in range(4):
            i = int(rng.integers(1, 0, P.W[k].shape[0] - 1)[0])
            j = int(rng.integers(1, 0, P.W[k].shape[1] - 1)[0])
            if P.W[k][i, j] == 0 or abs(P.W[k][i, j]) < 10 * h:
                continue

            def m(Q, d):
                Q.W[k][i, j] += d
            fd = (bound_with(lambda Q: m(Q, h)) - bound_with(lambda Q: m(Q, -h))) / (2 * h)
            assert fd == pytest.approx(grad["dW"][k][i, j], rel=1e-5, abs=1e-7)
            checks += 1
        i = int(rng.integers(1, 0, P.W[k].shape[0] - 1)[0])

        def mb(Q, d):
            Q.b[k][i] += d
        fd = (bound_with(lambda Q: mb(Q, h)) - bound_with(lambda Q: mb(Q, -h))) / (2 * h)
        assert fd == pytest.approx(grad["db"][k][i], rel=1e-5, abs=1e-7)
    for j in range(min(6, P.widths[0])):
        def ml(Q, d):
            Q.lo[0][j] += d

        def mh(Q, d):
            Q.hi[0][j] += d
        fd = (bound_with(lambda Q: ml(Q, h)) - bound_with(lambda Q: ml(Q, -h))) / (2 * h)
        assert fd == pytest.approx(grad["dlo0"][j], rel=1e-5, abs=1e-7)
        fd = (bound_with(lambda Q: mh(Q, h)) - bound_with(lambda Q: mh(Q, -h))) / (2 * h)
        assert fd == pytest.approx(grad["dhi0"][j], rel=1e-5, abs=1e-7)
    assert checks >= 4


def test_dense_conv_operator_equals_library_convolution():
    """The oracle's dense conv matrix applied to an input equals torch's conv2d (float64)."""
    layers = synth.small_convnet()
    net = synth.make_net(layers, 3)
    rng = synth.SplitMix64(4)
    for L in net:
        if L["kind"] != "conv":
            continue
        W, b, taps = nw.conv_dense(L)
        x = rng.uniform(L["n_in"]) - 0.5
        ref = F.conv2d(torch.from_numpy(x.reshape(1, *L["in_shape"])),
                       torch.from_numpy(L["W"].astype(np.float64)),
                       torch.from_numpy(L["b"].astype(np.float64)),
                       stride=L["stride"], padding=L["pad"]).numpy().ravel()
        np.testing.assert_allclose(W @ x + b, ref, rtol=1e-12, atol=1e-12)
        assert len(taps) == np.count_nonzero(W)


def test_interval_bounds_contain_sampled_preactivations_and_respect_splits():
    prob = synth.problem("wide_conv_bab", S=4, seed=0)
    dense = nw.dense_layers(prob["net"])
    Ps = nw.problems(prob, dense=dense)
    rng = synth.SplitMix64(1)
    for s, P in enumerate(Ps):
        X = P.lo[0][None, :] + rng.uniform(20 * 3072).reshape(20, 3072) * (P.hi[0] - P.lo[0])
        h = X.T
        off = 0
        for k in range(1, P.n):
            pre = P.W[k] @ h + P.b[k][:, None]
            sp = prob["splits"][s][off:off + P.widths[k]]
            free = sp == 0
            assert (pre[free] >= P.lhat[k][free, None] - 1e-9).all()
            assert (pre[free] <= P.uhat[k][free, None] + 1e-9).all()
            assert (P.lhat[k] <= P.uhat[k]).all()
            h = np.maximum(pre, 0)
            off += P.widths[k]


def _chain_bound(P, st, splits, mod):
    """The bound at fixed duals and masks, with interval propagation redone after mod(Q)."""
    Q = nw.Problem.__new__(nw.Problem)
    Q.__dict__.update(P.__dict__)
    Q.W = [None if w is None else w.copy() for w in P.W]
    Q.b = [None if w is None else w.copy() for w in P.b]
    lo0, hi0 = P.lo[0].copy(), P.hi[0].copy()
    Q.lo, Q.hi = [lo0], [hi0]
    mod(Q)
    lh, uh, lo, hi = nw.ibp(Q.W[1:Q.n], Q.b[1:Q.n], Q.lo[0], Q.hi[0], splits)
    Q.lhat, Q.uhat, Q.lo, Q.hi = lh, uh, lo, hi
    st2 = du.DualState(st.alpha, st.beta0, st.beta1, [[] for _ in range(P.n)])
    for k in range(1, P.n):
        for sl in st.slots[k]:
            du.add_slot(Q, st2, k, sl.I, beta=sl.beta)
    return du.evaluate(Q, st2)[0]


@pytest.mark.parametrize("name,with_splits", [("mlp_4_5_5_1", False), ("small_conv", False),
                                              ("mlp_3_4_4_4_1", True)])
def test_chain_gradient_matches_finite_differences(name, with_splits):
    """Central differences of the bound with the intermediate bounds recomputed by interval
    propagation at every perturbed point; the chain gradient differs from the fixed-bound one."""
    prob = synth.problem(name, seed=4)
    splits = None
    if with_splits:
        NH = sum(L["n_out"] for L in prob["net"][:-1])
        P0 = nw.problems(prob)[0]
        lh = np.concatenate(P0.lhat[1:])
        uh = np.concatenate(P0.uhat[1:])
        amb = np.flatnonzero((lh < 0) & (uh > 0))
        splits = np.zeros(NH, np.int8)
        splits[amb[0]] = 1
        splits[amb[-1]] = -1
        prob = dict(prob, splits=splits[None, :].repeat(prob["lo"].shape[0], 0))
    P = nw.problems(prob)[0]
    s = AS.ActiveSet(P, AS.Options(bigm_iters=30, as_iters=30, omega=10, max_cuts=3)).step(60)
    st = s.st
    grad = ev.chain_gradient(P, st, splits)
    base = ev.envelope_gradient(P, st)
    rng = synth.SplitMix64(11)
    h = 1e-6

    def fd(mod):
        return (_chain_bound(P, st, splits, lambda Q: mod(Q, h)) -
                _chain_bound(P, st, splits, lambda Q: mod(Q, -h))) / (2 * h)

    checks, differs = 0, 0
    for k in range(1, P.n + 1):
        for _ in range(5):
            i = int(rng.integers(1, 0, P.W[k].shape[0] - 1)[0])
            j = int(rng.integers(1, 0, P.W[k].shape[1] - 1)[0])
            if abs(P.W[k][i, j]) < 10 * h:
                continue

            def m(Q, d):
                Q.W[k][i, j] += d
            assert fd(m) == pytest.approx(grad["dW"][k][i, j], rel=1e-5, abs=1e-7)
            differs += abs(grad["dW"][k][i, j] - base["dW"][k][i, j]) > 1e-4
            checks += 1
        i = int(rng.integers(1, 0, P.W[k].shape[0] - 1)[0])

        def mb(Q, d):
            Q.b[k][i] += d
        assert fd(mb) == pytest.approx(grad["db"][k][i], rel=1e-5, abs=1e-7)
    for j in range(min(6, P.widths[0])):
        def ml(Q, d):
            Q.lo[0][j] += d

        def mh(Q, d):
            Q.hi[0][j] += d
        assert fd(ml) == pytest.approx(grad["dlo0"][j], rel=1e-5, abs=1e-7)
        assert fd(mh) == pytest.approx(grad["dhi0"][j], rel=1e-5, abs=1e-7)
        differs += abs(grad["dlo0"][j] - base["dlo0"][j]) > 1e-4
    assert checks >= 8 and differs >= 2

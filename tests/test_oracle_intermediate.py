"""Pins of the intermediate-bounds oracle (App. E) against the paper's Fig. 4 example, exact LPs,
interval propagation at zero duals, and sampled pre-activations."""
import json
import os

import numpy as np
import pytest

from oracle import active_set as AS
from oracle import intermediate as IM
from oracle import lp
from oracle import network as nw
from paper_2101_05844_gb300 import synth
from tests.helpers import fig4_net

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig4_lp.json")))["printed"]


def test_fig4_zero_iterations_give_the_printed_interval_values():
    """Zero duals bound each neuron by interval propagation (App. B.3): post-activation
    l_1 = [0, 0], u_1 = [1, 3] and M+_2[1] = 3 as App. F.1 prints them."""
    Ws, bs, w3, b3, lo0, hi0 = lp.fig4_network()
    lh, uh = IM.intermediate_bounds(fig4_net(), lo0, hi0, AS.Options())
    np.testing.assert_array_equal(np.maximum(lh[1], 0), GOLD["l_1"])
    np.testing.assert_array_equal(np.maximum(uh[1], 0), GOLD["u_1"])
    assert uh[2][1] == GOLD["M^+_2[1]"]


def test_fig4_solves_reach_the_printed_lp_bound_from_outside():
    """Big-M solves of the layer-2 problems approach the LP value uhat_2[1] = 2.25 of App. F.1
    from above (a dual bound never crosses the LP optimum), and every layer-2 bound brackets the
    exact LP bounds of problem (App. E) with C_k = M_k within 1e-3."""
    Ws, bs, w3, b3, lo0, hi0 = lp.fig4_network()
    lh, uh = IM.intermediate_bounds(fig4_net(), lo0, hi0, AS.Options(bigm_iters=2000))
    assert GOLD["uhat_2[1]"] <= uh[2][1] <= GOLD["uhat_2[1]"] + 1e-3
    lm, um, _, _ = lp.layer_bounds_lp(Ws, bs, lo0, hi0, "M")
    assert np.all(lh[2] <= lm[2] + 1e-12) and np.all(lh[2] >= lm[2] - 1e-3)
    assert np.all(uh[2] >= um[2] - 1e-12) and np.all(uh[2] <= um[2] + 1e-3)
    np.testing.assert_array_equal(lh[1], lm[1])
    np.testing.assert_array_equal(uh[1], um[1])


@pytest.mark.parametrize("name,seed", [("mlp_4_3_3_3_1", 2), ("small_conv", 1)])
def test_zero_iterations_equal_interval_propagation(name, seed):
    prob = synth.problem(name, S=2, seed=seed)
    dense = nw.dense_layers(prob["net"])
    for s in range(2):
        lh, uh = IM.intermediate_bounds(prob["net"], prob["lo"][s], prob["hi"][s], AS.Options(), dense=dense)
        ih, iu, _, _ = nw.ibp([d[0] for d in dense[:-1]], [d[1] for d in dense[:-1]], prob["lo"][s],
                              prob["hi"][s])
        for k in range(1, len(lh)):
            np.testing.assert_allclose(lh[k], ih[k], rtol=0, atol=1e-12)
            np.testing.assert_allclose(uh[k], iu[k], rtol=0, atol=1e-12)


def _preacts(prob, s, n_samples, seed):
    """Pre-activations of every hidden layer at random points of box s and at its vertices."""
    rng = synth.SplitMix64(seed)
    lo, hi = prob["lo"][s].astype(np.float64), prob["hi"][s].astype(np.float64)
    n0 = lo.size
    X = lo[None] + rng.uniform(n_samples * n0).reshape(n_samples, n0) * (hi - lo)[None]
    if n0 <= 12:
        V = np.array(np.meshgrid(*[[0, 1]] * n0)).reshape(n0, -1).T
        X = np.vstack([X, np.where(V == 1, hi, lo)])
    h = X.T
    out = []
    for W, b, _ in nw.dense_layers(prob["net"])[:-1]:
        a = W @ h + b[:, None]
        out.append(a)
        h = np.maximum(a, 0.0)
    return out


def test_bounds_contain_sampled_preactivations_and_tighten_interval_bounds():
    prob = synth.problem("mlp_4_3_3_3_1", S=2, seed=2)
    opt = AS.Options(bigm_iters=300, as_iters=200, omega=50, max_cuts=4)
    dense = nw.dense_layers(prob["net"])
    gained = 0.0
    for s in range(2):
        lh, uh = IM.intermediate_bounds(prob["net"], prob["lo"][s], prob["hi"][s], opt, dense=dense)
        ih, iu, _, _ = nw.ibp([d[0] for d in dense[:-1]], [d[1] for d in dense[:-1]], prob["lo"][s],
                              prob["hi"][s])
        for k, a in enumerate(_preacts(prob, s, 4000, 11 + s), start=1):
            assert np.all(a.min(axis=1) >= lh[k] - 1e-12)
            assert np.all(a.max(axis=1) <= uh[k] + 1e-12)
            assert np.all(lh[k] >= ih[k]) and np.all(uh[k] <= iu[k])
            gained += float(np.sum(iu[k] - ih[k]) - np.sum(uh[k] - lh[k]))
    assert gained > 0.0


def test_deeper_layers_use_the_tightened_bounds_of_earlier_layers():
    """With converged Big-M solves, each layer's bounds reach the exact LP over C_k = M_k built
    on the bounds this procedure produced for the earlier layers (within 2e-4) and never cross
    it; the same LP over interval-propagated layer-2 bounds is lower by more than 2e-3 on some
    layer-3 neuron, so a procedure that skipped the earlier tightening would fail here."""
    prob = synth.problem("mlp_4_3_3_3_1", S=1, seed=2)
    lo0, hi0 = prob["lo"][0], prob["hi"][0]
    dense = nw.dense_layers(prob["net"])
    Ws, bs = [d[0] for d in dense[:-1]], [d[1] for d in dense[:-1]]
    lh, uh = IM.intermediate_bounds(prob["net"], lo0, hi0, AS.Options(bigm_iters=3000), dense=dense)
    lo = [np.asarray(lo0, np.float64)] + [np.maximum(v, 0) for v in lh[1:]]
    hi = [np.asarray(hi0, np.float64)] + [np.maximum(v, 0) for v in uh[1:]]
    for k in range(2, len(lh)):
        sub = lp.NetLP(Ws[:k - 1], bs[:k - 1], lh[:k], uh[:k], lo[:k], hi[:k])
        W, b = Ws[k - 1], bs[k - 1]
        for i in range(W.shape[0]):
            vl = float(sub.solve("M", W[i], b[i], sense=1))
            vu = float(sub.solve("M", W[i], b[i], sense=-1))
            assert vl - 2e-4 <= lh[k][i] <= vl + 1e-9
            assert vu - 1e-9 <= uh[k][i] <= vu + 2e-4
    # the layer-3 LP over interval-propagated layer-2 bounds is looser somewhere
    ih, iu, ilo, ihi = nw.ibp(Ws, bs, lo0, hi0)
    looser = lp.NetLP(Ws[:2], bs[:2], [None, lh[1], ih[2]], [None, uh[1], iu[2]], [lo[0], lo[1], ilo[2]],
                      [hi[0], hi[1], ihi[2]])
    W3, b3 = Ws[2], bs[2]
    gap = [lh[3][i] - float(looser.solve("M", W3[i], b3[i], sense=1)) for i in range(W3.shape[0])]
    assert max(gap) > 2e-3


def test_split_clamps_a_straddling_neuron():
    prob = synth.problem("mlp_4_3_3_3_1", S=1, seed=2)
    lo0, hi0 = prob["lo"][0], prob["hi"][0]
    opt = AS.Options(bigm_iters=50)
    lh, uh = IM.intermediate_bounds(prob["net"], lo0, hi0, opt)
    amb = [(k, i) for k in range(2, len(lh)) for i in range(lh[k].size) if lh[k][i] < 0 < uh[k][i]]
    assert amb
    widths = [v.size for v in lh[1:]]
    offs = np.cumsum([0] + widths)
    for sgn in (1, -1):
        k, i = amb[0]
        sp = np.zeros(offs[-1], np.int8)
        sp[offs[k - 1] + i] = sgn
        lh2, uh2 = IM.intermediate_bounds(prob["net"], lo0, hi0, opt, splits=sp)
        if sgn > 0:
            assert lh2[k][i] == 0.0 and uh2[k][i] > 0
        else:
            assert uh2[k][i] == 0.0 and lh2[k][i] < 0
        for kk in range(1, k + 1):   # layers up to k are unchanged elsewhere
            for ii in range(lh[kk].size):
                if (kk, ii) != (k, i):
                    assert lh2[kk][ii] == lh[kk][ii] and uh2[kk][ii] == uh[kk][ii]

"""Pins of the branch-and-bound oracle (Sec. 6.2): the subtree-size estimate at hand-evaluated
points, and verdicts against the exact minimum of small networks, found by enumerating every
ReLU activation pattern and solving each linear region's LP exactly."""
import math

import numpy as np
import pytest

from oracle import active_set as AS
from oracle import bab
from oracle import intermediate as IM
from oracle import network as nw
from paper_2101_05844_gb300 import synth
from tests.helpers import exact_min, net_with_shifted_output as _case


def _opts(**kw):
    o = dict(loose=AS.Options(bigm_iters=100), tight=AS.Options(bigm_iters=50, as_iters=100, omega=30, max_cuts=3),
             batch=8, max_domains=600)
    o.update(kw)
    return bab.BabOptions(**o)


def test_subtree_ratio_at_hand_evaluated_points():
    # l = -2, i = 1: a_l grows 2^3 - 1 = 7 nodes; with l_{a_t-a_l} = 1, a_t grows 2^2 - 1 = 3
    assert bab.subtree_ratio(-2.0, 1.0, 1.0) == pytest.approx(7 / 3)
    # l_{a_t-a_l} = 2.5: a_t grows 2^0.5 - 1 nodes
    assert bab.subtree_ratio(-2.0, 2.5, 1.0) == pytest.approx(7 / (math.sqrt(2) - 1))
    # a_t would prune the child at once
    assert bab.subtree_ratio(-2.0, 4.0, 1.0) == math.inf
    # deep trees: the ratio tends to 2^(l_{a_t-a_l} / i)
    assert bab.subtree_ratio(-1000.0, 3.0, 1.0) == pytest.approx(8.0)
    assert bab.subtree_ratio(-50.0, 3.0, 2.0) == pytest.approx((2 ** 26 - 1) / (2 ** 24.5 - 1))
    assert not bab.is_hard(-2.0, 1.0, None, 1.0)
    assert bab.is_hard(-2.0, 1.0, 0.0, 1.0) and not bab.is_hard(-2.0, -1.0, 0.0, 1.0)
    assert bab.is_hard(-2.0, 1.0, 1.0, 2.0) and not bab.is_hard(-2.0, 1.0, 1.0, 2.5)


def test_branch_neuron_takes_the_largest_relaxation_gap():
    lh = [None, np.array([-1.0, -3.0, 0.5]), np.array([-2.0, -1.0])]
    uh = [None, np.array([1.0, 1.0, 2.0]), np.array([2.0, -0.5])]
    # gaps -l u / (u - l): 0.5, 0.75, (not ambiguous), 1.0, (not ambiguous)
    assert bab.branch_neuron(lh, uh, np.zeros(5, np.int8)) == 3
    assert bab.branch_neuron(lh, uh, np.array([0, 0, 0, 1, 0], np.int8)) == 1
    assert bab.branch_neuron(lh, uh, np.array([1, 1, 0, 1, 0], np.int8)) == -1


def test_exact_minimum_is_below_every_sample_and_reached_by_one():
    prob = synth.problem("mlp_4_3_3_1", S=1, seed=1)
    m = exact_min(prob["net"], prob["lo"][0], prob["hi"][0], np.ones(1))
    rng = synth.SplitMix64(3)
    lo, hi = prob["lo"][0].astype(np.float64), prob["hi"][0].astype(np.float64)
    X = lo + rng.uniform(20000 * 4).reshape(20000, 4) * (hi - lo)
    dense = nw.dense_layers(prob["net"])
    vals = np.array([bab.forward(dense, x)[0] for x in X])
    assert vals.min() >= m - 1e-9
    assert vals.min() - m <= 0.02 * (vals.max() - vals.min())


@pytest.mark.parametrize("name,seed,margin,expect", [
    ("mlp_4_3_3_1", 3, -0.03, bab.VERIFIED), ("mlp_4_5_5_1", 4, -0.03, bab.VERIFIED),
    ("mlp_4_5_5_1", 7, -0.03, bab.VERIFIED), ("mlp_3_4_4_4_1", 6, -0.03, bab.VERIFIED),
    ("mlp_4_3_3_1", 1, 0.03, bab.FALSIFIED), ("mlp_4_5_5_1", 2, 0.03, bab.FALSIFIED),
    ("mlp_3_4_4_4_1", 4, 0.03, bab.FALSIFIED)])
def test_verdict_matches_the_exact_minimum(name, seed, margin, expect):
    """The property f(x) - t > 0 with t 3% of the output's range over the box below / above its
    exact minimum: verified / falsified (with a counterexample inside the box whose float64 value
    is negative), the reported bounds bracketing the exact minimum. Some cases need branching
    (up to 41 domains), some only the root."""
    net, lo, hi, m_t = _case(name, seed, margin)
    res = bab.BaB(net, lo, hi, np.ones(1), _opts()).run()
    assert res["status"] == expect
    if expect == bab.VERIFIED:
        assert 0 < res["lower"] <= m_t + 1e-9
    else:
        x = res["x"]
        assert np.all(x >= lo - 1e-12) and np.all(x <= hi + 1e-12)
        assert bab.forward(nw.dense_layers(net), x)[0] < 0
        assert res["lower"] <= m_t + 1e-9 <= res["upper"] + 2e-9


def test_stratification_switches_only_when_the_estimate_says_so():
    net, lo, hi, _ = _case("mlp_4_5_5_1", 4, -0.03)
    ones = np.ones(1)
    never = bab.BaB(net, lo, hi, ones, _opts(cost_ratio=1e30)).run()
    always = bab.BaB(net, lo, hi, ones, _opts(cost_ratio=0.0)).run()
    plain = bab.BaB(net, lo, hi, ones, _opts(stratify=False)).run()
    assert never["status"] == always["status"] == plain["status"] == bab.VERIFIED
    assert never["hard_bounded"] == 1                     # the root's a_t solve only
    assert plain["hard_bounded"] == plain["bounded"]      # a_t everywhere
    assert always["hard_bounded"] > 1


def test_warm_start_and_root_intermediate_bounds_prune_sooner():
    """Starting each child from its parent's duals (Sec. 8.2) verifies the property within the
    domain budget that cold starts exhaust; tighter root intermediate bounds (App. E) verify it
    with fewer domains."""
    net, lo, hi, _ = _case("mlp_4_5_5_1", 4, -0.03)
    ones = np.ones(1)
    warm = bab.BaB(net, lo, hi, ones, _opts()).run()
    cold = bab.BaB(net, lo, hi, ones, _opts(warm_start=False, max_domains=60)).run()
    assert warm["status"] == bab.VERIFIED and warm["bounded"] < 60
    assert cold["status"] == bab.UNKNOWN
    rb = IM.intermediate_bounds(net, lo, hi, AS.Options(bigm_iters=200))
    tight = bab.BaB(net, lo, hi, ones, _opts(), root_bounds=rb).run()
    assert tight["status"] == bab.VERIFIED and tight["bounded"] < warm["bounded"]


def test_unsplittable_domains_are_bounded_again_from_their_own_duals():
    """A root with no ambiguous neuron is an exact LP; its first solve stops short of the exact
    minimum and re-solves from its own duals reach a positive bound."""
    net, lo, hi, m_t = _case("mlp_4_5_5_1", 1, -0.03)
    ones = np.ones(1)
    once = bab.BaB(net, lo, hi, ones, _opts(leaf_rebounds=0)).run()
    again = bab.BaB(net, lo, hi, ones, _opts()).run()
    assert once["status"] == bab.UNKNOWN and once["bounded"] == 2
    assert again["status"] == bab.VERIFIED and 2 < again["bounded"] <= 10
    assert 0 < again["lower"] <= m_t + 1e-9


@pytest.mark.parametrize("seed,shift", [(3, False), (2, True)])
def test_conv_net_verdicts_agree_with_sampled_points(seed, shift):
    """The small conv net (every layer kind) with a three-output property row: a falsified verdict
    comes with a point of the box whose float64 value is negative (seed 3 after branching). With
    the property moved below a valid lower bound of a long solve (sampled values are no guide in
    72 input dimensions: the search finds points far below them), it is verified."""
    prob = synth.problem("small_conv", S=1, seed=seed)
    net, lo, hi, c = prob["net"], prob["lo"][0], prob["hi"][0], prob["C"][0].astype(np.float64)
    dense = nw.dense_layers(net)
    rng = synth.SplitMix64(seed)
    X = lo + rng.uniform(3000 * lo.size).reshape(3000, lo.size) * (hi - lo)
    vals = np.array([c @ bab.forward(dense, x) for x in X])
    if shift:
        P = nw.Problem(net, lo, hi, c, dense=dense)
        lb = AS.solve(P, AS.Options(bigm_iters=300, as_iters=300, omega=60, max_cuts=3))[1]
        t = lb - 0.02 * abs(lb)
        net = [dict(L) for L in net]
        net[-1]["b"] = (net[-1]["b"].astype(np.float64) - t * c / (c @ c)).astype(np.float32)
        dense = nw.dense_layers(net)
        vals = np.array([c @ bab.forward(dense, x) for x in X])
    res = bab.BaB(net, lo, hi, c, _opts(max_domains=200)).run()
    if shift:
        assert res["status"] == bab.VERIFIED and 0 < res["lower"] <= vals.min()
    else:
        assert res["status"] == bab.FALSIFIED and res["bounded"] > 2
        x = res["x"]
        assert np.all(x >= lo) and np.all(x <= hi) and c @ bab.forward(dense, x) < 0
        assert res["lower"] <= vals.min()

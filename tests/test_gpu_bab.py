"""as_bab (Sec. 6.2 branch and bound, Sec. 8.2 warm starts) against the oracle's branch and bound
and the exact minimum of small networks.

What is unique is compared: the verdict, and the bracketing lower <= exact minimum <= upper. The
trees themselves may differ (float32 bounds against float64 ones decide the order of domains, the
branching neuron among near-equal gaps and the moment a bound turns positive), so their sizes are
only checked for the behaviour each option is for."""
import numpy as np
import pytest

from oracle import active_set as AS
from oracle import bab as obab
from oracle import network as nw
from paper_2101_05844_gb300 import binding, synth
from tests.helpers import net_with_shifted_output

pytestmark = pytest.mark.gpu

LOOSE = dict(bigm_iters=100, as_iters=0)
TIGHT = dict(bigm_iters=50, as_iters=100, omega=30, max_cuts=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    binding.lib()


def _gpu(**kw):
    base = dict(batch=8, max_domains=600, cost_ratio=4.0, ema_weight=0.3, leaf_rebounds=8)
    base.update(kw)
    return binding.bab_default_options(loose=LOOSE, tight=TIGHT, **base)


def _oracle(**kw):
    o = dict(loose=AS.Options(**LOOSE), tight=AS.Options(**TIGHT), batch=8, max_domains=600, cost_ratio=4.0)
    o.update(kw)
    return obab.BabOptions(**o)


CASES = [("mlp_4_3_3_1", 3, -0.03, "verified"), ("mlp_4_5_5_1", 4, -0.03, "verified"),
         ("mlp_4_5_5_1", 7, -0.03, "verified"), ("mlp_3_4_4_4_1", 6, -0.03, "verified"),
         ("mlp_4_3_3_1", 1, 0.03, "falsified"), ("mlp_4_5_5_1", 2, 0.03, "falsified"),
         ("mlp_3_4_4_4_1", 4, 0.03, "falsified")]


@pytest.mark.parametrize("name,seed,margin,expect", CASES)
def test_verdict_matches_oracle_and_exact_minimum(name, seed, margin, expect):
    net, lo, hi, m_t = net_with_shifted_output(name, seed, margin)
    res = binding.bab(net, lo, hi, None, _gpu())
    ref = obab.BaB(net, lo, hi, np.ones(1), _oracle()).run()
    assert ref["status"] == expect
    assert res["status"] == expect
    assert res["lower"] <= m_t + 1e-6 * (1 + abs(m_t))
    if expect == "verified":
        assert res["lower"] > 0 and res["frontier"] == 0
    else:
        x = res["x"].astype(np.float64)
        assert np.all(x >= lo) and np.all(x <= hi)
        assert obab.forward(nw.dense_layers(net), x)[0] == pytest.approx(res["upper"], abs=1e-12)
        assert res["upper"] < 0 and m_t <= res["upper"] + 1e-9


def test_stratification_switch():
    net, lo, hi, _ = net_with_shifted_output("mlp_4_5_5_1", 4, -0.03)
    never = binding.bab(net, lo, hi, None, _gpu(cost_ratio=1e30))
    always = binding.bab(net, lo, hi, None, _gpu(cost_ratio=1e-30))
    plain = binding.bab(net, lo, hi, None, _gpu(stratify=0))
    assert never["status"] == always["status"] == plain["status"] == "verified"
    assert never["hard_bounded"] == 1
    assert always["hard_bounded"] > 1
    assert plain["hard_bounded"] == plain["bounded"]
    measured = binding.bab(net, lo, hi, None, _gpu(cost_ratio=0.0))
    assert measured["status"] == "verified" and measured["cost_ratio"] > 1.0   # a_t runs more iterations


def test_warm_start_and_root_intermediate_bounds():
    net, lo, hi, _ = net_with_shifted_output("mlp_4_5_5_1", 4, -0.03)
    warm = binding.bab(net, lo, hi, None, _gpu())
    cold = binding.bab(net, lo, hi, None, _gpu(warm_start=0, max_domains=60))
    assert warm["status"] == "verified" and warm["bounded"] < 60
    assert cold["status"] == "unknown"
    tight = binding.bab(net, lo, hi, None, _gpu(root_intermediate=1, intermediate=dict(bigm_iters=200, as_iters=0)))
    assert tight["status"] == "verified" and tight["bounded"] < warm["bounded"]


def test_unsplittable_root_is_solved_again():
    net, lo, hi, m_t = net_with_shifted_output("mlp_4_5_5_1", 1, -0.03)
    once = binding.bab(net, lo, hi, None, _gpu(leaf_rebounds=0))
    again = binding.bab(net, lo, hi, None, _gpu())
    assert once["status"] == "unknown" and once["bounded"] == 2 and once["frontier"] == 1
    assert again["status"] == "verified" and 0 < again["lower"] <= m_t + 1e-6


def test_limits_and_errors():
    net, lo, hi, _ = net_with_shifted_output("mlp_3_4_4_4_1", 6, -0.03)
    r = binding.bab(net, lo, hi, None, _gpu(max_domains=5))
    assert r["status"] == "unknown" and r["frontier"] > 0 and r["lower"] <= 0
    with pytest.raises(binding.CBError):
        binding.bab(net, lo, hi, None, _gpu(batch=7))
    with pytest.raises(binding.CBError):
        binding.bab(net, hi + 1.0, hi, None, _gpu())


def test_conv_net_multi_output_property_is_decided_consistently():
    """The small conv net (every layer kind) and a runner-up property row: a verdict of "verified"
    must hold at sampled points, a "falsified" one must come with a real counterexample."""
    prob = synth.problem("small_conv", S=1, seed=2)
    net, lo, hi, c = prob["net"], prob["lo"][0], prob["hi"][0], prob["C"][0]
    res = binding.bab(net, lo, hi, c, _gpu(batch=16, max_domains=400))
    dense = nw.dense_layers(net)
    rng = synth.SplitMix64(5)
    X = lo + rng.uniform(3000 * lo.size).reshape(3000, lo.size) * (hi - lo)
    vals = np.array([c @ obab.forward(dense, x) for x in X])
    assert res["lower"] <= vals.min() + 1e-5
    if res["status"] == "verified":
        assert vals.min() > 0
    elif res["status"] == "falsified":
        assert c @ obab.forward(dense, res["x"].astype(np.float64)) < 0
    assert res["upper"] >= res["lower"]

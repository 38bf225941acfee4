"""Parity of as_intermediate_bounds (App. E, batched sub-network solves) with the oracle.

Tolerances: every bound within 1e-4 (1 + |v|) of the FP64 oracle (float32 solves of a few
iterations, bounds of earlier layers feeding later ones, outward rounding); validity (sampled
pre-activations inside the bounds, inside interval propagation) exactly.
"""
import numpy as np
import pytest

from oracle import active_set as AS
from oracle import intermediate as IM
from oracle import network as nw
from paper_2101_05844_gb300 import binding, synth

pytestmark = pytest.mark.gpu

KW = dict(bigm_iters=12, as_iters=8, omega=4, max_cuts=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    binding.lib()


def _opts(**kw):
    return binding.default_options(graph_chunk=0, **kw)


def _ibp(prob, s):
    dense = nw.dense_layers(prob["net"])
    sp = None if prob.get("splits") is None else prob["splits"][s]
    lh, uh, _, _ = nw.ibp([d[0] for d in dense[:-1]], [d[1] for d in dense[:-1]], prob["lo"][s],
                          prob["hi"][s], sp)
    return np.concatenate(lh[1:]), np.concatenate(uh[1:])


def _preacts(prob, s, n, seed):
    rng = synth.SplitMix64(seed)
    lo, hi = prob["lo"][s].astype(np.float64), prob["hi"][s].astype(np.float64)
    X = lo[None] + rng.uniform(n * lo.size).reshape(n, lo.size) * (hi - lo)[None]
    h, out = X.T, []
    for W, b, _ in nw.dense_layers(prob["net"])[:-1]:
        a = W @ h + b[:, None]
        out.append(a)
        h = np.maximum(a, 0.0)
    return np.concatenate(out, axis=0)


def _with_splits(prob, seed):
    prob = dict(prob)
    S = prob["lo"].shape[0]
    NH = sum(L["n_out"] for L in prob["net"][:-1])
    rng = synth.SplitMix64(seed)
    sp = np.zeros((S, NH), np.int8)
    idx = rng.integers(S * 3, 0, NH).reshape(S, 3)
    sgn = np.where(rng.uniform(S * 3).reshape(S, 3) < 0.5, 1, -1)
    for s in range(S):
        sp[s, idx[s]] = sgn[s]
    prob["splits"] = sp
    return prob


@pytest.mark.parametrize("name,S,splits", [("mlp_4_3_3_3_1", 3, False), ("mlp_5_7_6_3", 2, True),
                                           ("small_conv", 2, False)])
def test_matches_oracle(name, S, splits):
    prob = synth.problem(name, S=S, seed=3)
    if splits:
        prob = _with_splits(prob, 5)
    lh, uh = binding.intermediate_bounds(prob["net"], prob["lo"], prob["hi"], prob.get("splits"), _opts(**KW))
    rl, ru = IM.batch(prob, AS.Options(**KW))
    np.testing.assert_allclose(lh, rl, rtol=0, atol=1e-4 * (1 + np.abs(rl)).max())
    np.testing.assert_allclose(uh, ru, rtol=0, atol=1e-4 * (1 + np.abs(ru)).max())
    for s in range(S):
        il, iu = _ibp(prob, s)
        assert np.all(lh[s] >= il - 1e-6 * (1 + np.abs(il))) and np.all(uh[s] <= iu + 1e-6 * (1 + np.abs(iu)))
        if not splits:
            a = _preacts(prob, s, 2000, 7 + s)
            assert np.all(a.min(axis=1) >= lh[s] - 1e-6) and np.all(a.max(axis=1) <= uh[s] + 1e-6)
    assert np.sum(uh - lh) < np.sum([np.sum(_ibp(prob, s)[1] - _ibp(prob, s)[0]) for s in range(S)])


def test_chunked_batches_agree_with_one_batch():
    """max_batch splits each layer's subproblems over several contexts (a ragged last one, pairs
    kept whole); per-subproblem arithmetic does not depend on the batch."""
    prob = synth.problem("small_conv", S=3, seed=4)
    one = binding.intermediate_bounds(prob["net"], prob["lo"], prob["hi"], None, _opts(**KW))
    many = binding.intermediate_bounds(prob["net"], prob["lo"], prob["hi"], None, _opts(**KW), max_batch=17)
    for a, b in zip(one, many):
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6)


def test_zero_iterations_return_interval_bounds():
    prob = synth.problem("small_conv", S=2, seed=6)
    lh, uh = binding.intermediate_bounds(prob["net"], prob["lo"], prob["hi"], None, _opts(bigm_iters=0, as_iters=0))
    for s in range(2):
        il, iu = _ibp(prob, s)
        tol = 4e-6 * (1 + np.abs(il))
        assert np.all(lh[s] <= il + tol) and np.all(lh[s] >= il - tol)
        tol = 4e-6 * (1 + np.abs(iu))
        assert np.all(uh[s] <= iu + tol) and np.all(uh[s] >= iu - tol)


def test_invalid_arguments():
    prob = synth.problem("mlp_4_3_3_3_1", S=1, seed=0)
    with pytest.raises(binding.CBError):
        binding.intermediate_bounds(prob["net"], prob["hi"] + 1.0, prob["lo"], None, _opts(**KW))
    with pytest.raises(binding.CBError):
        binding.intermediate_bounds(prob["net"], prob["lo"], prob["hi"], None, _opts(**KW), max_batch=-1)


def test_full_size_wide_conv_sampled_neurons():
    """The 3x32x32 wide conv net, one box: layer 2 (2048 conv neurons, 4096 subproblems of the
    sub-network conv16 -> conv32-as-dense) and layer 3 (100 neurons over both convs). Sampled
    layer-2 neurons match oracle solves; every bound is valid for sampled inputs and inside
    interval propagation."""
    prob = synth.problem("wide_conv", seed=0)
    prob = dict(prob, lo=prob["lo"][:1], hi=prob["hi"][:1], C=prob["C"][:1])
    kw = dict(bigm_iters=3, as_iters=2, omega=2, max_cuts=2)
    lh, uh = binding.intermediate_bounds(prob["net"], prob["lo"], prob["hi"], None, _opts(**kw))
    net = prob["net"]
    dense = nw.dense_layers(net)
    Ws, bs = [d[0] for d in dense[:-1]], [d[1] for d in dense[:-1]]
    il, iu, _, _ = nw.ibp(Ws, bs, prob["lo"][0], prob["hi"][0])
    n1, n2 = Ws[0].shape[0], Ws[1].shape[0]
    rng = synth.SplitMix64(21)
    for i in rng.integers(6, 0, n2):
        i = int(i)
        vals = []
        for sign in (1.0, -1.0):
            crow = np.zeros(n2)
            crow[i] = sign
            P = nw.Problem(net[:2], prob["lo"][0], prob["hi"][0], crow, bounds=([il[1]], [iu[1]]), dense=dense[:2])
            vals.append(AS.solve(P, AS.Options(**kw))[0])
        rl, ru = max(il[2][i], vals[0]), min(iu[2][i], -vals[1])
        assert lh[0, n1 + i] == pytest.approx(rl, abs=1e-4 * (1 + abs(rl)))
        assert uh[0, n1 + i] == pytest.approx(ru, abs=1e-4 * (1 + abs(ru)))
    ilc, iuc = np.concatenate(il[1:]), np.concatenate(iu[1:])
    assert np.all(lh[0] >= ilc - 1e-6 * (1 + np.abs(ilc))) and np.all(uh[0] <= iuc + 1e-6 * (1 + np.abs(iuc)))
    a = _preacts(prob, 0, 200, 3)
    assert np.all(a.min(axis=1) >= lh[0] - 1e-5) and np.all(a.max(axis=1) <= uh[0] + 1e-5)
    assert np.sum(uh[0, n1:] - lh[0, n1:]) < np.sum(iuc[n1:] - ilc[n1:])

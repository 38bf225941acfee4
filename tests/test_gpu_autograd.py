"""Differentiation (the MLP 784-1024x3-10 workload): the envelope gradient through torch.autograd.

1. Finite differences through the GPU path itself: the bound at fixed duals and masks is linear
   in each weight where the primal minimiser does not change, so a central difference of two
   contexts with perturbed weights (same duals, snapshots and intermediate bounds installed via
   the state API) must equal the autograd gradient.
2. The full-size MLP 784-1024-1024-1024-10 with 256 boxes: gradients at a drawn state match the
   oracle's envelope gradient on sampled entries (the oracle computes them from its own masks).
"""
import numpy as np
import pytest

from oracle import envelope as ev
from oracle import network as nw
from paper_2101_05844_gb300 import binding, synth
from tests.state_helpers import draw_state, oracle_bounds_f32, split_hidden

pytestmark = pytest.mark.gpu

STATE = [binding.ST_ITER, binding.ST_ALPHA, binding.ST_BETA0, binding.ST_BETA1, binding.ST_XSNAP,
         binding.ST_ZSNAP, binding.ST_SLOT_BETA]


def _copy_state(src, dst):
    for w in STATE:
        dtype = np.int32 if w == binding.ST_ITER else (np.uint8 if w in (binding.ST_XSNAP, binding.ST_ZSNAP)
                                                        else np.float32)
        dst.set_state(w, src.get_state(w, dtype))


def test_autograd_gradient_equals_finite_differences_of_the_gpu_bound():
    torch = pytest.importorskip("torch")
    from paper_2101_05844_gb300.autograd import bound

    prob = synth.problem("mlp_12_20_20_5", S=3, seed=3)
    kw = dict(bigm_iters=30, as_iters=60, omega=20, max_cuts=4, graph_chunk=0)
    ctx = binding.context_for(prob, binding.default_options(**kw))
    ctx.as_step(75)
    lh = ctx.get_state(binding.ST_LHAT).reshape(ctx.S, -1)
    uh = ctx.get_state(binding.ST_UHAT).reshape(ctx.S, -1)
    dev = torch.device("cuda")
    params = []
    for L in prob["net"]:
        params += [torch.tensor(L["W"], device=dev, requires_grad=True),
                   torch.tensor(L["b"], device=dev, requires_grad=True)]
    lo = torch.tensor(prob["lo"], device=dev, requires_grad=True)
    hi = torch.tensor(prob["hi"], device=dev, requires_grad=True)
    weights = torch.tensor(synth.SplitMix64(5).uniform(ctx.S) + 0.5, device=dev)
    (bound(ctx, lo, hi, params) * weights).sum().backward()

    ctx.bound()
    xstar0 = ctx.get_state(binding.ST_XSTAR)
    zstar0 = ctx.get_state(binding.ST_ZSTAR, np.uint8)

    def perturbed(k, kind, idx, h):
        """Bound sum with one weight moved by h, and whether the minimiser stayed the same."""
        net = [dict(L) for L in prob["net"]]
        arr = net[k][kind].copy()
        arr.flat[idx] += h
        net[k] = dict(net[k], **{kind: arr})
        c2 = binding.Context(net, prob["lo"], prob["hi"], prob["C"], lh, uh, options=binding.default_options(**kw))
        _copy_state(ctx, c2)
        v = float((c2.bound() * weights.cpu().numpy()).sum())
        same = (c2.get_state(binding.ST_XSTAR) == xstar0).all() and \
            (c2.get_state(binding.ST_ZSTAR, np.uint8) == zstar0).all()
        c2.close()
        return v, same

    rng = synth.SplitMix64(9)
    checked = 0
    for k in range(len(prob["net"])):
        for kind, grad in (("W", params[2 * k].grad), ("b", params[2 * k + 1].grad)):
            n = prob["net"][k][kind].size
            for _ in range(4):
                idx = int(rng.integers(1, 0, n - 1)[0])
                h = 1e-2 * max(1.0, abs(float(prob["net"][k][kind].flat[idx])))
                (vp, sp), (vm, sm) = perturbed(k, kind, idx, h), perturbed(k, kind, idx, -h)
                if not (sp and sm):
                    continue          # the minimiser moved: the bound is not linear across +-h
                fd = (vp - vm) / (2 * h)
                g = float(grad.flatten()[idx])
                assert fd == pytest.approx(g, rel=2e-3, abs=2e-3), (k, kind, idx)
                checked += 1
    assert checked >= 16


def test_full_size_mlp_gradient_matches_oracle_on_sampled_entries():
    torch = pytest.importorskip("torch")
    prob = synth.problem("mlp_wide", S=256, seed=0)
    dense = nw.dense_layers(prob["net"])
    Ps0 = nw.problems(prob, dense=dense)
    lh, uh = oracle_bounds_f32(Ps0)
    widths = Ps0[0].widths
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), widths)[1:]) for s in range(256)],
                     dense=dense)
    kw = dict(bigm_iters=50, as_iters=250, omega=75, max_cuts=5, graph_chunk=0)
    ctx = binding.context_for(prob, binding.default_options(**kw), bounds=(lh, uh))
    sample = [0, 37, 101, 255]   # the oracle evaluates these subproblems; the rest get weight 0
    solvers = draw_state(Ps, ctx, kw, it=130, nslots=4, seed=77, subset=set(sample))
    gb = np.zeros(256)
    gb[sample] = [1.0, 0.5, 2.0, 1.5]
    dev = torch.device("cuda")
    dW = [torch.zeros(L["W"].shape, device=dev) for L in prob["net"]]
    db = [torch.zeros(L["b"].shape, device=dev) for L in prob["net"]]
    dlo = torch.zeros(prob["lo"].shape, device=dev)
    dhi = torch.zeros(prob["hi"].shape, device=dev)
    ctx.backward(gb, dW, db, dlo, dhi)
    torch.cuda.synchronize()
    refW = [np.zeros(L["W"].shape) for L in prob["net"]]
    refb = [np.zeros(L["b"].shape) for L in prob["net"]]
    for s in sample:
        g = ev.envelope_gradient(solvers[s].P, solvers[s].st)
        for k in range(1, solvers[s].P.n):
            refW[k - 1] += gb[s] * g["dW"][k]
            refb[k - 1] += gb[s] * g["db"][k]
        refW[-1] += gb[s] * np.outer(prob["C"][s], g["dW"][solvers[s].P.n][0])
        refb[-1] += gb[s] * prob["C"][s]
        np.testing.assert_allclose(dlo[s].cpu().numpy(), gb[s] * g["dlo0"], rtol=1e-4, atol=1e-4)
        np.testing.assert_allclose(dhi[s].cpu().numpy(), gb[s] * g["dhi0"], rtol=1e-4, atol=1e-4)
    for k in range(len(prob["net"])):
        np.testing.assert_allclose(dW[k].cpu().numpy(), refW[k], rtol=1e-4, atol=2e-4)
        np.testing.assert_allclose(db[k].cpu().numpy(), refb[k], rtol=1e-4, atol=2e-4)


def test_values_other_than_the_contexts_are_refused():
    """A training loop that updated a weight, or a box other than the one the context bounds, gets
    an error instead of the gradient of the context's stale copies."""
    torch = pytest.importorskip("torch")
    from paper_2101_05844_gb300.autograd import bound

    prob = synth.problem("mlp_4_5_5_1", S=2, seed=1)
    ctx = binding.context_for(prob, binding.default_options(bigm_iters=5, as_iters=5, graph_chunk=0))
    ctx.as_step(10)
    dev = torch.device("cuda")
    params = []
    for L in prob["net"]:
        params += [torch.tensor(L["W"], device=dev, requires_grad=True),
                   torch.tensor(L["b"], device=dev, requires_grad=True)]
    lo = torch.tensor(prob["lo"], device=dev, requires_grad=True)
    hi = torch.tensor(prob["hi"], device=dev, requires_grad=True)
    bound(ctx, lo, hi, params).sum().backward()      # the context's own values: accepted
    with torch.no_grad():
        params[2][0, 0] += 1e-3                        # an optimiser step on W_2
    with pytest.raises(ValueError, match="W_2"):
        bound(ctx, lo, hi, params)
    with torch.no_grad():
        params[2][0, 0] -= 1e-3
        lo2 = lo.detach().clone()
        lo2[0, 0] -= 0.01
    with pytest.raises(ValueError, match="box"):
        bound(ctx, lo2, hi, params)
    ctx.reset(lo2, hi, torch.tensor(prob["C"], device=dev))   # reset to the new box: accepted
    ctx.as_step(10)
    assert torch.isfinite(bound(ctx, lo2, hi, params)).all()

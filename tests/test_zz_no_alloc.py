"""The allocation-free interval-bound entry point, as_ibp_noalloc.

It serves callers that cannot call cudaMalloc: a verifier embedded in a process whose device
memory belongs to another allocator (a framework's caching allocator, a serving engine's fixed
pool), or a latency-critical caller that cannot take the implicit synchronisation of
cudaMalloc / cudaFree. These tests call it through the C ABI and check its bounds against the
ones the context path (as_init) computes, bit for bit, on consecutive calls, and against the
oracle's float64 interval propagation; that it refuses a
problem larger than its fixed scratch, host pointers, and (where a second GPU exists) memory of
another device, by its host-side checks alone.
"""
import numpy as np
import pytest

from oracle import network as nw
from paper_2101_05844_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _device_net(net, torch):
    out = []
    for L in net:
        L = dict(L)
        L["W"] = torch.from_numpy(np.ascontiguousarray(L["W"], np.float32)).cuda()
        L["b"] = torch.from_numpy(np.ascontiguousarray(L["b"], np.float32)).cuda()
        out.append(L)
    return out


def _context_bounds(prob, S):
    ctx = binding.context_for(prob, binding.default_options())
    lh = ctx.get_state(binding.ST_LHAT).reshape(S, -1)
    uh = ctx.get_state(binding.ST_UHAT).reshape(S, -1)
    ctx.close()
    return lh, uh


def _noalloc_bounds(prob, S, torch):
    net = _device_net(prob["net"], torch)
    lo = torch.from_numpy(prob["lo"]).cuda()
    hi = torch.from_numpy(prob["hi"]).cuda()
    splits = None if prob.get("splits") is None else torch.from_numpy(prob["splits"]).cuda()
    NH = sum(L["n_out"] for L in prob["net"][:-1])
    lh = torch.full((S, NH), float("nan"), device="cuda")
    uh = torch.full((S, NH), float("nan"), device="cuda")
    rc = binding.ibp_noalloc(net, lo, hi, lh, uh, splits, stream=torch.cuda.current_stream().cuda_stream)
    assert rc == binding.AS_OK
    torch.cuda.synchronize()
    return lh.cpu().numpy(), uh.cpu().numpy()


def test_noalloc_bounds_equal_context_bounds_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    binding.lib()
    cases = [("wide_conv_bab", 6, 0), ("small_conv", 3, 1), ("wide_conv_bab", 6, 0)]
    for name, S, seed in cases:   # consecutive calls share the scratch; the third repeats the first
        prob = synth.problem(name, S=S, seed=seed)
        lh_ref, uh_ref = _context_bounds(prob, S)
        lh, uh = _noalloc_bounds(prob, S, torch)
        assert np.isfinite(lh).all() and np.isfinite(uh).all()
        # the same compensated accumulation in the same lane order and the same outward rounding as
        # the context's interval bounds: bit for bit
        np.testing.assert_array_equal(lh, lh_ref)
        np.testing.assert_array_equal(uh, uh_ref)
        # and against the oracle's float64 interval propagation (App. E): sound (the float32 interval
        # contains it) and within a few float32 ulps per layer
        for s, P in enumerate(nw.problems(prob)):
            rl = np.concatenate([np.asarray(P.lhat[k]) for k in range(1, P.n)])
            ru = np.concatenate([np.asarray(P.uhat[k]) for k in range(1, P.n)])
            assert (lh[s] <= rl + 1e-9 * (1 + np.abs(rl))).all() and (uh[s] >= ru - 1e-9 * (1 + np.abs(ru))).all()
            assert (np.abs(lh[s] - rl) <= 4e-6 * (1 + np.abs(rl))).all()
            assert (np.abs(uh[s] - ru) <= 4e-6 * (1 + np.abs(ru))).all()
        if prob.get("splits") is not None:
            # the split branch runs: some split neurons were clamped to zero at one end
            sp = prob["splits"]
            assert ((lh == 0) & (sp > 0)).sum() + ((uh == 0) & (sp < 0)).sum() > 0


def test_noalloc_refuses_problems_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    layers = synth.arch("conv4")
    net = synth.make_net(layers, 1)
    S = 64                                   # 4 x 64 x 32768 floats > the 4 Mi-float scratch
    assert 4 * S * max(L["n_out"] for L in layers[:-1]) > binding.NOALLOC_SCRATCH_FLOATS
    dnet = _device_net(net, torch)
    lo = torch.zeros((S, 3072), device="cuda")
    hi = torch.ones((S, 3072), device="cuda")
    NH = sum(L["n_out"] for L in layers[:-1])
    lh = torch.empty((S, NH), device="cuda")
    uh = torch.empty((S, NH), device="cuda")
    assert binding.ibp_noalloc(dnet, lo, hi, lh, uh) == binding.AS_ERR_SCRATCH
    # host pointers are refused too: the call cannot copy them without allocating
    assert binding.ibp_noalloc(dnet[:1] + dnet[1:], lo.cpu(), hi.cpu(), lh, uh) == binding.AS_ERR_ARG


def test_noalloc_refuses_memory_of_another_device():
    """Buffers on a device other than the current one are refused before any launch (the kernels
    could reach them only through peer access). Needs a second GPU; the check is host-side."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: no memory of another device to pass")
    prob = synth.problem("small_conv", S=2, seed=1)
    torch.cuda.set_device(0)
    net = _device_net(prob["net"], torch)
    NH = sum(L["n_out"] for L in prob["net"][:-1])
    other = torch.device("cuda", 1)
    lo = torch.from_numpy(prob["lo"]).to(other)
    hi = torch.from_numpy(prob["hi"]).to(other)
    lh = torch.empty((2, NH), device=other)
    uh = torch.empty((2, NH), device=other)
    assert binding.ibp_noalloc(net, lo, hi, lh, uh) == binding.AS_ERR_ARG

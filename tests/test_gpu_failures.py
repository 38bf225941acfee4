"""Failure paths of the C ABI, each made on the host, so that no GPU faults, traps or hangs:

  * AS_ERR_NUMERIC: weights with a NaN give a non-finite bound, which as_bound reports;
  * AS_ERR_OOM: the library's allocation hook (environment CB_FAIL_ALLOC_AT = n) refuses the n-th
    device allocation of a context as if the device were full; as_init then fails cleanly, frees
    what it had allocated, and the next context is unaffected;
  * AS_ERR_TIMEOUT: the tensor-core GEMMs' stage waits given a limit of zero rounds (environment
    CB_TC_STAGE_WAIT_LIMIT = 0) give up at once; the CTA then waits for its last commit with the
    full limit (no MMA in flight), frees its tensor memory, sets the status word, and the next
    as_bound returns AS_ERR_TIMEOUT. A context made without the hook runs normally afterwards.
"""
import os

import numpy as np
import pytest

from paper_2101_05844_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    binding.lib()


class _env:
    def __init__(self, key, value):
        self.key, self.value = key, value

    def __enter__(self):
        os.environ[self.key] = self.value

    def __exit__(self, *a):
        os.environ.pop(self.key, None)


def test_nan_weight_gives_a_numeric_error():
    prob = synth.problem("mlp_tiny", seed=0)
    prob["net"][1]["W"] = prob["net"][1]["W"].copy()
    prob["net"][1]["W"][0, 0] = np.nan
    ctx = binding.context_for(prob, binding.default_options(bigm_iters=3, as_iters=3, graph_chunk=0))
    ctx.as_step(4)
    with pytest.raises(binding.CBError) as e:
        ctx.bound()
    assert e.value.code == binding.AS_ERR_NUMERIC


def test_refused_allocations_fail_cleanly():
    import torch
    prob = synth.problem("small_conv", S=3, seed=1)
    opt = binding.default_options(bigm_iters=4, as_iters=6, omega=3, max_cuts=3, graph_chunk=0)
    ok = binding.context_for(prob, opt)          # warm: the library's module and torch's context are up
    ok.as_step(10)
    ref = ok.bound()
    ok.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    refused = 0
    for n in (1, 2, 5, 9, 14, 20, 30):
        with _env("CB_FAIL_ALLOC_AT", str(n)):
            try:
                c = binding.context_for(prob, opt)
            except binding.CBError as e:
                assert e.code == binding.AS_ERR_OOM
                refused += 1
            else:
                c.close()
    assert refused >= 4
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 64 << 20   # what the failed inits took is freed
    c = binding.context_for(prob, opt)
    c.as_step(10)
    np.testing.assert_array_equal(c.bound(), ref)


def test_tensor_core_wait_limit_reports_a_timeout_and_the_gpu_stays_usable():
    prob = synth.problem("conv4", S=2, seed=0)
    opt = binding.default_options(bigm_iters=2, as_iters=4, omega=2, max_cuts=2, graph_chunk=0, precision=16)
    with _env("CB_TC_STAGE_WAIT_LIMIT", "0"):
        ctx = binding.context_for(prob, opt)
    ctx.as_step(2)
    with pytest.raises(binding.CBError) as e:
        ctx.bound()
    assert e.value.code == binding.AS_ERR_TIMEOUT
    ctx.close()
    good = binding.context_for(prob, opt)
    good.as_step(6)
    assert np.isfinite(good.bound()).all()

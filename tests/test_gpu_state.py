"""Whole-state export and import (as_export_state / as_import_state): a context continued from an
imported blob follows the exporting one; lambda, kappa are recomputed in float32 on import, so the
bounds agree to 1e-5 relative, not bit for bit. Mismatched contexts and foreign blobs are refused."""
import numpy as np
import pytest

from paper_2101_05844_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    binding.lib()


@pytest.mark.parametrize("name,S", [("small_conv", 3), ("mlp_5_7_6_3", 2)])
def test_active_set_and_saddle_point_continue_from_an_imported_state(name, S):
    prob = synth.problem(name, S=S, seed=2)
    opt = binding.default_options(graph_chunk=0, bigm_iters=10, as_iters=60, omega=8, max_cuts=4, sp_init_steps=10)
    a = binding.context_for(prob, opt)
    a.as_step(27)                       # mid Active Set, slots filled
    blob = a.export_state()
    b = binding.context_for(prob, opt)
    b.import_state(blob)
    np.testing.assert_allclose(b.bound(), a.bound(), rtol=1e-5, atol=1e-6)
    a.as_step(20)
    b.as_step(20)
    np.testing.assert_allclose(b.bound(), a.bound(), rtol=1e-5, atol=1e-5)
    a.sp_step(5)
    blob = a.export_state()
    c = binding.context_for(prob, opt)
    c.import_state(blob)
    np.testing.assert_allclose(c.bound(), a.bound(), rtol=1e-5, atol=1e-6)
    a.sp_step(5)
    c.sp_step(5)
    np.testing.assert_allclose(c.bound(), a.bound(), rtol=1e-5, atol=1e-5)


def test_mismatched_imports_are_refused():
    prob = synth.problem("mlp_tiny", S=1, seed=0)
    a = binding.context_for(prob, binding.default_options(graph_chunk=0, max_cuts=4))
    a.as_step(5)
    blob = a.export_state()
    other = binding.context_for(prob, binding.default_options(graph_chunk=0, max_cuts=5))
    with pytest.raises(binding.CBError):
        other.import_state(blob)
    with pytest.raises(binding.CBError):
        a.import_state(np.zeros_like(blob))


def test_a_refused_import_leaves_the_context_unchanged():
    """A blob of another batch size passes the iteration counter's section but not the duals': the
    import is refused before any buffer is written, so the context goes on as if never touched."""
    prob = synth.problem("small_conv", S=3, seed=2)
    opt = binding.default_options(graph_chunk=0, bigm_iters=10, as_iters=60, omega=8, max_cuts=4)
    a = binding.context_for(prob, opt)
    a.as_step(23)
    ref = binding.context_for(prob, opt)
    ref.as_step(23)
    small = synth.problem("small_conv", S=2, seed=2)
    other = binding.context_for(small, opt)
    other.as_step(5)
    blob = other.export_state()
    with pytest.raises(binding.CBError) as e:
        a.import_state(blob)
    assert e.value.code == binding.AS_ERR_SHAPE
    a.as_step(9)
    ref.as_step(9)
    np.testing.assert_array_equal(a.bound(), ref.bound())
    np.testing.assert_array_equal(a.get_state(binding.ST_ITER, np.int32), ref.get_state(binding.ST_ITER, np.int32))

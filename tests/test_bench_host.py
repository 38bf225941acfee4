"""Host-side pieces of bench.py that need no GPU: the committed DRAM-traffic record and its source
check, the algorithmic work and byte models of the roofline, the slot schedule, and the oracle
sample code the CPU baselines run."""
import hashlib
import json
import os

import pytest

import bench
from paper_2101_05844_gb300 import binding, synth


def test_traffic_record_scales_with_the_batch_and_names_its_sources():
    """A committed capture names the sources it was taken on; while they are unchanged the bench
    reports its bytes scaled from the captured batch to the timed one, and a changed or missing
    source reports none."""
    path = os.path.join(bench.ROOT, "profiles", "dram_traffic_conv4.json")
    if not os.path.exists(path):
        pytest.skip("no DRAM capture committed for the conv4 workload")
    rec = json.load(open(path))
    fresh = all(hashlib.sha256(open(os.path.join(bench.ROOT, s["path"]), "rb").read()).hexdigest() == s["sha256"]
                for s in rec["sources"])
    for k, v in rec["dram_bytes_per_launch"].items():
        got = bench.captured_traffic("conv4", k, 2 * rec["subproblems"])
        assert got == (pytest.approx(2 * v) if fresh else None)
    assert bench.captured_traffic("conv4", "no_such_kernel", 8) is None
    assert bench.captured_traffic("no_such_workload", "as_colA", 8) is None


def test_slot_schedule_of_the_default_workload():
    """100 Big-M then 400 Active Set iterations, masks added at t = 0, 1, 120, 121, 240 (cap 5): the
    col pass consumes the slots added before its iteration, the row pass those after."""
    opt = binding.Options()
    for k, v in dict(bigm_iters=100, as_iters=400, omega=120, vars_per_add=2, max_cuts=5).items():
        setattr(opt, k, v)
    col, row = bench.conv4_slots(opt)
    assert len(col) == len(row) == 500
    assert col[:101] == [0] * 101 and row[:100] == [0] * 100
    assert row[100] == 1 and col[101] == 1 and row[101] == 2 and col[102] == 2
    assert col[220] == 2 and row[220] == 3 and row[221] == 4 and col[340] == 4 and row[340] == 5
    assert col[-1] == row[-1] == 5


def test_byte_and_flop_models_grow_with_slots():
    net = synth.problem("conv4", S=1, seed=0)["net"]
    b0, b5 = bench.colA_bf16_bytes(net, 0, 5), bench.colA_bf16_bytes(net, 5, 5)
    # 8 bytes per slot product and 8 per slot (beta, kappa) on every hidden input: 16 per slot there
    nh_in = sum(L["n_in"] for L in net[1:-1])
    assert b5 - b0 == 5 * 8 * sum(L["n_in"] for L in net[:-1]) + 5 * 8 * sum(L["n_in"] for L in net[1:])
    assert nh_in > 0
    r0, r5 = bench.rowB_bf16_bytes(net, 0, 5), bench.rowB_bf16_bytes(net, 5, 5)
    assert r5 - r0 == 5 * 36 * sum(L["n_out"] for L in net[:-1])
    assert bench.tc_flops(net, 5) == pytest.approx(6 * bench.tc_flops(net, 0))


def test_dense_nnz_counts_the_taps_inside_the_image():
    """The nonzeros of a conv layer's operator: one per (output, input) pair its filter connects, the
    zero padding left out (the oracle's dense operator lists them)."""
    from oracle import network as nw
    for L in synth.problem("small_conv", seed=0)["net"]:
        if L["kind"] == "conv":
            assert bench.dense_nnz(L) == len(nw.conv_dense(L)[2])
        else:
            assert bench.dense_nnz(L) == L["n_in"] * L["n_out"]


def test_algorithmic_flops_scale_with_subproblems_launches_and_slots():
    net = synth.problem("wide_conv", seed=0)["net"]
    sched = [0] * 10
    f1 = bench.algorithmic_flops(net, 9, "as_colA", sched, 10)
    assert f1 > 0
    assert bench.algorithmic_flops(net, 18, "as_colA", sched, 10) == pytest.approx(2 * f1)
    assert bench.algorithmic_flops(net, 9, "as_colA", sched, 20) == pytest.approx(2 * f1)
    assert bench.algorithmic_flops(net, 9, "as_colA", [3] * 10, 10) > f1


@pytest.mark.parametrize("workload,variant", [("wide_conv", ""), ("wide_conv", "l2"), ("wide_conv", "layer2"),
                                              ("conv4", "")])
def test_oracle_sample_code_compiles_for_every_variant(workload, variant):
    compile(bench._oracle_sample_code(workload, 0, 1.0, variant), "<sample>", "exec")

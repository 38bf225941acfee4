"""Host-side pieces of bench.py that need no GPU: the committed DRAM-traffic record and its source
check, the HBM side of the roofline built from it, the algorithmic work model, and the oracle
sample code the CPU baselines run."""
import json
import os

import pytest

import bench


def test_traffic_record_matches_the_current_kernel_source():
    """The committed capture names the source it was taken on; while that source is unchanged the
    bench reports its bytes, and a changed source reports none."""
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "dram_traffic_wide_conv.json")))
    for k, v in rec["dram_bytes_per_launch"].items():
        assert bench.captured_traffic("wide_conv", k) == v
    assert bench.captured_traffic("wide_conv", "no_such_kernel") is None
    assert bench.captured_traffic("no_such_workload", "as_colA") is None


def test_hbm_rooflines_from_captured_bytes_and_live_durations():
    kt = {"as_colA": (25.0, 1000), "as_rowB": (0.0, 0), "sp_rowB": (30.0, 1000)}
    out = bench.hbm_rooflines("wide_conv", kt)
    assert set(out) == {"as_colA"}   # no launches: skipped; no capture: skipped
    r = out["as_colA"]
    t = bench.captured_traffic("wide_conv", "as_colA")
    assert r["launch_us"] == pytest.approx(25.0)
    assert r["achieved"] == pytest.approx(t / 25e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_algorithmic_flops_scale_with_subproblems_launches_and_slots():
    from paper_2101_05844_gb300 import synth
    net = synth.problem("wide_conv", seed=0)["net"]
    sched = [0] * 10
    f1 = bench.algorithmic_flops(net, 9, "as_colA", sched, 10)
    assert f1 > 0
    assert bench.algorithmic_flops(net, 18, "as_colA", sched, 10) == pytest.approx(2 * f1)
    assert bench.algorithmic_flops(net, 9, "as_colA", sched, 20) == pytest.approx(2 * f1)
    assert bench.algorithmic_flops(net, 9, "as_colA", [3] * 10, 10) > f1


@pytest.mark.parametrize("variant", ["", "l2", "layer2"])
def test_oracle_sample_code_compiles_for_every_variant(variant):
    compile(bench._oracle_sample_code("wide_conv", 0, 1.0, variant), "<sample>", "exec")

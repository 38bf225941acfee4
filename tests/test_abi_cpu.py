"""Host-side checks without a GPU: the library builds, loads and exports every declared symbol;
the generator is deterministic; argument validation happens before any kernel runs."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_2101_05844_gb300 import binding, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2101_05844_gb300 import build
    build.build()
    return binding.lib()


def test_library_exports_every_declared_function(built):
    hdr = open(os.path.join(ROOT, "include", "convex_barrier.h")).read()
    names = set(re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(\w+)\s*\(", hdr, re.M))
    assert {"as_init", "as_step", "sp_step", "as_bound", "as_bound_backward"} <= names
    for n in names:
        assert hasattr(built, n), n
    assert set(binding.EXPORTS) == names


def test_default_options_are_the_papers(built):
    o = binding.default_options()
    assert (o.bigm_lr0, o.bigm_lr1, o.as_lr0, o.as_lr1) == (1e-2, 1e-4, 1e-3, 1e-6)
    assert (o.omega, o.vars_per_add, o.max_cuts, o.sp_gamma0, o.sp_init_steps) == (450, 2, 7, 10.0, 100)


STRUCTS = [("as_options", binding.Options), ("as_layer", binding.Layer), ("as_net", binding.Net),
           ("as_bab_options", binding.BabOptions), ("as_bab_result", binding.BabResult)]


def test_struct_layouts_match_header(tmp_path):
    """sizeof and field offsets of every ABI struct, from the C compiler, equal the binding's."""
    import subprocess
    src = tmp_path / "probe.c"
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "convex_barrier.h"', 'int main(void){']
    for cname, py in STRUCTS:
        body.append(f'printf("%zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            body.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    body.append('return 0;}')
    src.write_text("\n".join(body))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    expect = []
    for _, py in STRUCTS:
        expect.append(ct.sizeof(py))
        expect += [getattr(py, f).offset for f, _ in py._fields_]
    assert out == expect


def test_generator_is_deterministic_and_seeded():
    a = synth.problem("small_conv", seed=3)
    b = synth.problem("small_conv", seed=3)
    c = synth.problem("small_conv", seed=4)
    for La, Lb in zip(a["net"], b["net"]):
        assert (La["W"] == Lb["W"]).all()
    assert (a["lo"] == b["lo"]).all() and not (a["lo"] == c["lo"]).all()
    u = synth.SplitMix64(0).uniform(100000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    n = synth.SplitMix64(1).normal(200000)
    assert abs(n.mean()) < 0.01 and abs(n.std() - 1) < 0.01


def test_splitmix64_reference_values():
    # SplitMix64 with state 0 (first outputs published with the algorithm's reference code)
    r = synth.SplitMix64(0)
    v = r.bits(3)
    assert [int(x) for x in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_workload_shapes():
    p = synth.problem("wide_conv", seed=0)
    assert [L["n_out"] for L in p["net"]] == [4096, 2048, 100, 10]
    assert p["C"].shape == (9, 10) and p["lo"].shape == (9, 3072)
    q = synth.problem("wide_conv_bab", S=16, seed=0)
    assert q["splits"].shape == (16, 6244) and ((q["caps"] >= 1) & (q["caps"] <= 5)).all()

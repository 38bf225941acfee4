"""Benchmark of the batched Active Set / Saddle Point hot path on one or more GB300 GPUs.

Default workload (the precision configuration, the largest that fits one GPU): the conv net
3x32x32 -> 4 conv 3x3 (32, 32, 64, 64 channels; strides 1, 2, 1, 2; padding 1) -> FC512 -> FC10 on
1024 L-infinity boxes of half-width 8/255 around U[0,1] images, one property per box (the top logit
at the centre against the runner-up); synthetic He-initialised weights. One step bounds the whole
batch end to end through the C ABI and covers every step of the hot path:
  the BF16 form of Big-M then Active Set (100 Big-M + 400 Active Set iterations; masks added at
  Active Set iterations 0, 1, 120, 121, 240, cap 5: S1-S6 of the path), the bound re-evaluated in
  float32 with float64 summation (S8); then Saddle Point continuing from those duals (AS-SP, S7:
  conversion, 10 primal-initialisation steps, 20 iterations) and its bound.
value = subproblem-iterations per second of the step (520 per box), inputs resident in HBM; e2e =
the same with the batch in pinned host memory and both bounds read back, copies inside the timed
region. forms = the same Active Set schedule in the plain float32 form and the BF16 form on the same
batch and GPU: subproblem-iterations/s and the time each takes to reach the float32 form's final
bound (minus 1e-4, absolute and relative). roofline = the dominant kernel of a profiled step against
its bound (HBM bytes, tensor or FP32 ALU flops); cpu_baseline = the CPU oracle on a bounded sample.
wide_conv = the Wide conv net's 9 properties (Active Set and Saddle Point solves on two streams), the
earlier headline, as an extra key. --impl reference times the CPU oracle as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Active-Set subproblem-iters/s & time-to-bound vs plain FP32; % HBM roofline"
UNIT = "subproblem-iters/s"
L2_BYTES = 129 * 1024 * 1024
FP32_LANES_PER_SM = 128

# the default workload's schedule (conv4, 1024 boxes)
C4_S, C4_BIGM, C4_AS, C4_OMEGA, C4_CAP = 1024, 100, 400, 120, 5
C4_SP_INIT, C4_SP_ITERS = 10, 20
# the Wide conv net's (the extra key)
AS_BIGM, AS_ITERS, SP_BIGM, SP_ITERS = 200, 800, 200, 1000


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def fp32_peak_tflops(torch, dev):
    """FP32 ALU peak: SMs (queried at run time) x 128 FP32 lanes x 2 flop x the maximum SM clock
    (MEASURED_PEAKS.json, else nvidia-smi, else 2.07 GHz)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = measured_peaks().get("sm_max_mhz")
    src = "MEASURED_PEAKS.json sm_max_mhz"
    if not mhz:
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(dev.index or 0), "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            mhz, src = float(out.stdout.strip().splitlines()[0]), "nvidia-smi clocks.max.sm"
        except (OSError, ValueError, IndexError, subprocess.SubprocessError):
            mhz, src = 2070.0, "nominal 2.07 GHz"
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, f"{sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz ({src})"


# the BF16 contexts time their products' plans at as_init (as_options.autotune), before any timing
TC_AUTOTUNE = int(os.environ.get("CB_BENCH_TC_AUTOTUNE", "1"))


def conv4_options(binding, precision, profile=0, graph_chunk=25, bigm=C4_BIGM, as_iters=C4_AS, omega=C4_OMEGA):
    return binding.default_options(bigm_iters=bigm, as_iters=as_iters, omega=omega, max_cuts=C4_CAP,
                                   graph_chunk=graph_chunk, profile=profile, precision=precision,
                                   sp_init_steps=C4_SP_INIT, autotune=TC_AUTOTUNE if precision == 16 else 0)


def conv4_step(ctx, batch, out_as, out_sp, events=None):
    """One step of the default workload on one context: reset, Big-M + Active Set, bound, Saddle
    Point continuation, bound. events: three CUDA events recorded before, between and after the
    two solves (on the current stream, which the context's stream is)."""
    lo, hi, C = batch
    if events:
        events[0].record()
    ctx.reset(lo, hi, C)
    ctx.as_step(C4_BIGM + C4_AS)
    ctx.bound_into(64, out_as)
    if events:
        events[1].record()
    ctx.sp_step(C4_SP_ITERS)
    ctx.bound_into(64, out_sp)
    if events:
        events[2].record()


def workload_options(binding, profile=0):
    # autotune: each context times its passes' team sizes on its own net and batch at creation
    as_opt = binding.default_options(bigm_iters=AS_BIGM, as_iters=AS_ITERS, omega=round(0.3 * AS_ITERS),
                                     max_cuts=5, graph_chunk=25, profile=profile, autotune=1)
    sp_opt = binding.default_options(bigm_iters=SP_BIGM, as_iters=0, max_cuts=5, graph_chunk=25,
                                     profile=profile, autotune=1)
    return as_opt, sp_opt


def wide_step(ctx_as, ctx_sp, batch, out_as, out_sp):
    """The Wide conv net's step: the Active Set solve and the Saddle Point solve of the batch, on
    contexts on different streams, so their launches overlap on the GPU."""
    lo, hi, C = batch
    ctx_as.reset(lo, hi, C)
    ctx_as.as_step(AS_BIGM + AS_ITERS)
    ctx_sp.reset(lo, hi, C)
    ctx_sp.as_step(SP_BIGM)
    ctx_sp.sp_step(SP_ITERS)
    ctx_as.bound_into(64, out_as)
    ctx_sp.bound_into(64, out_sp)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_flops(net, S, kernel, n_slots_per_iter, launches):
    """Algorithmic FP32 flops of all launches of a kernel over one step (2 per multiply-add).

    nnz_k = weights touched per layer application (the dense operator's nonzeros). Active Set
    row pass: (1 + slots) multiply-adds per (subproblem, nonzero) of every hidden layer, once per
    iteration; col pass: the same over hidden layers plus the output row, once per iteration and
    once more for the final bound (at the last iteration's slots). Saddle Point, per launch: row
    pass 3 per hidden nonzero (W x, the masked product, the mask row sum); phase A alone 1 per
    nonzero (W^T alpha); phase C fused with the next phase A 2 per hidden nonzero (the masked
    backward and W^T alpha)."""
    nnz = []
    for L in net:
        if L["kind"] == "linear":
            nnz.append(L["n_in"] * L["n_out"])
        else:
            c, h, w = L["in_shape"]
            oc, oh, ow = L["out_shape"]
            cnt = 0
            for oy in range(oh):
                for ky in range(L["kh"]):
                    y = oy * L["stride"] - L["pad"] + ky
                    if 0 <= y < h:
                        cnt += 1
            cntx = 0
            for ox in range(ow):
                for kx in range(L["kw"]):
                    x = ox * L["stride"] - L["pad"] + kx
                    if 0 <= x < w:
                        cntx += 1
            nnz.append(oc * c * cnt * cntx)
    hid = sum(nnz[:-1])
    out_row = net[-1]["n_in"]
    if kernel == "as_rowB":
        return sum(2.0 * S * hid * (1 + k) for k in n_slots_per_iter)
    if kernel == "as_colA":
        per = [2.0 * S * (hid * (1 + k) + out_row) for k in n_slots_per_iter]
        return sum(per) + per[-1] * max(0, launches - len(per))
    if kernel == "sp_rowB":
        return 2.0 * S * hid * 3 * launches
    if kernel == "sp_colA":
        return 2.0 * S * (hid + out_row) * launches
    if kernel == "sp_colC":
        return 2.0 * S * hid * 2 * launches
    return 0.0


def slots_schedule(opt):
    """Active-set size at every iteration of the Active Set context (global schedule)."""
    out = []
    for it in range(opt.bigm_iters + opt.as_iters):
        if it < opt.bigm_iters:
            out.append(0)
            continue
        t = it - opt.bigm_iters
        q, r = divmod(t, opt.omega)
        before = min(q * opt.vars_per_add + min(r, opt.vars_per_add), opt.max_cuts)
        add = 1 if (r < opt.vars_per_add and q * opt.vars_per_add + r < opt.max_cuts) else 0
        out.append(before + add)
    return out


def batched_run(binding, torch, dev, stream, rank):
    """The batching workload: the Wide conv net on 4096 branch-and-bound subdomains (random
    ReLU splits, caps of 1-5 masks), 100 Big-M + 400 Active Set iterations, one timed run after a
    warm-up, and a profiled run for the dominant kernel's rate."""
    from paper_2101_05844_gb300 import synth
    prob = synth.problem("wide_conv_bab", S=4096, seed=rank)
    S = 4096
    opt = binding.default_options(bigm_iters=100, as_iters=400, omega=120, max_cuts=5, graph_chunk=25, autotune=1)
    t = {k: torch.from_numpy(prob[k]).to(dev) for k in ("lo", "hi", "C", "splits", "caps")}
    ctx = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], splits=prob["splits"],
                          caps=prob["caps"], options=opt, stream=stream)
    out = torch.zeros(S, dtype=torch.float64, device=dev)

    def run(c):
        c.reset(t["lo"], t["hi"], t["C"], None, None, t["splits"], t["caps"])
        c.as_step(500)
        c.bound_into(64, out)

    run(ctx)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run(ctx)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    prof = binding.default_options(bigm_iters=100, as_iters=400, omega=120, max_cuts=5, profile=1, autotune=1)
    pc = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], splits=prob["splits"],
                         caps=prob["caps"], options=prof, stream=stream)
    kt0 = pc.kernel_times()   # as_init's own launches are not the run's
    run(pc)
    kt = {k: (v[0] - kt0[k][0], v[1] - kt0[k][1]) for k, v in pc.kernel_times().items()}
    top = max(kt, key=lambda k: kt[k][0])
    sched = slots_schedule(opt)
    # per-subdomain caps: the mean active-set size follows min(slots, cap)
    caps = prob["caps"].astype(float)
    mean_slots = [float(np.minimum(k, caps).mean()) for k in sched]
    flops = algorithmic_flops(prob["net"], S, top, mean_slots, kt[top][1])
    peak, _ = fp32_peak_tflops(torch, dev)
    achieved = flops / (kt[top][0] / 1e3) / 1e12
    teams = ctx.team_targets()
    ctx.close()
    pc.close()
    # the same run in the BF16 form (tensor-core products), for comparison
    o16 = binding.default_options(bigm_iters=100, as_iters=400, omega=120, max_cuts=5, graph_chunk=25, precision=16)
    c16 = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], splits=prob["splits"],
                          caps=prob["caps"], options=o16, stream=stream)
    run(c16)
    torch.cuda.synchronize()
    e0.record()
    run(c16)
    e1.record()
    e1.synchronize()
    ms16 = e0.elapsed_time(e1)
    c16.close()
    return {"workload": "wide_conv_bab", "subproblems": S, "iterations": 500, "value": S * 500 / (ms / 1e3),
            "team_targets": {"row": teams[0], "col": teams[1]},
            "bf16": {"value": S * 500 / (ms16 / 1e3), "ms": ms16},
            "unit": UNIT, "ms": ms, "roofline": {"bound": "alu", "kernel": top, "achieved": achieved, "peak": peak,
                                                 "unit": "TFLOP/s", "frac": achieved / peak},
            "kernel_ms": {k: v[0] for k, v in kt.items() if v[1]}}


def differentiation_run(binding, torch, dev, stream, rank):
    """The differentiation workload: MLP 784-1024-1024-1024-10 on 256 boxes of half-width 0.1,
    60 Big-M + 240 Active Set iterations in float32 (timed after a warm-up), then the bound and its
    envelope gradient with respect to W, b and the box endpoints (as_bound_backward, timed)."""
    from paper_2101_05844_gb300 import synth
    prob = synth.problem("mlp_wide", S=256, seed=rank)
    S, iters = 256, 300
    opt = binding.default_options(bigm_iters=60, as_iters=240, omega=72, max_cuts=5, graph_chunk=25)
    t = {k: torch.from_numpy(prob[k]).to(dev) for k in ("lo", "hi", "C")}
    ctx = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=opt, stream=stream)
    dW = [torch.zeros(L["W"].shape, device=dev) for L in prob["net"]]
    db = [torch.zeros(L["b"].shape, device=dev) for L in prob["net"]]
    dlo, dhi = torch.zeros(t["lo"].shape, device=dev), torch.zeros(t["hi"].shape, device=dev)
    g = torch.ones(S, dtype=torch.float64, device=dev)
    bound = torch.zeros(S, dtype=torch.float64, device=dev)

    def run():
        ctx.reset(t["lo"], t["hi"], t["C"])
        ctx.as_step(iters)

    run()
    ctx.backward(g, dW, db, dlo, dhi)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    run()
    e[1].record()
    ctx.bound_into(64, bound)
    ctx.backward(g, dW, db, dlo, dhi)
    e[2].record()
    e[2].synchronize()
    ms_it, ms_bw = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    b32 = bound.cpu().numpy().copy()
    ctx.close()
    # the same iterations in the BF16 form (the gradient is taken in float32 either way)
    opt16 = binding.default_options(bigm_iters=60, as_iters=240, omega=72, max_cuts=5, graph_chunk=25, precision=16)
    c16 = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=opt16, stream=stream)
    c16.reset(t["lo"], t["hi"], t["C"])
    c16.as_step(iters)
    torch.cuda.synchronize()
    c16.reset(t["lo"], t["hi"], t["C"])
    e[0].record()
    c16.as_step(iters)
    e[1].record()
    e[1].synchronize()
    ms16 = e[0].elapsed_time(e[1])
    c16.bound_into(64, bound)
    b16 = bound.cpu().numpy()
    c16.close()
    return {"workload": {"net": "mlp_784_1024x3_10", "subproblems": S, "iterations": iters, "eps": 0.1},
            "value": S * iters / (ms_it / 1e3), "unit": UNIT, "ms_iterations": ms_it,
            "ms_bound_and_backward": ms_bw, "mean_final_bound": float(b32.mean()),
            "bf16": {"value": S * iters / (ms16 / 1e3), "ms_iterations": ms16, "mean_final_bound": float(b16.mean()),
                     "minus_fp32_final_bound_mean": float((b16 - b32).mean())}}


def intermediate_run(binding, torch, dev, stream, rank):
    """Intermediate bounds by batched sub-network solves (App. E) on the wide conv net, one box:
    layer 2 (2048 conv neurons: 4096 subproblems of conv16 -> conv32 as a dense map) and layer 3
    (100 neurons: 200 subproblems of conv16 -> conv32 -> FC100), 100 Big-M + 100 Active Set
    iterations each (timed after a warm-up call); then the headline Active Set schedule on the 9
    properties of the box, once over interval bounds and once over the tightened bounds."""
    import numpy as np
    from paper_2101_05844_gb300 import synth
    prob = synth.problem("wide_conv", seed=rank)
    net, S9 = prob["net"], prob["lo"].shape[0]
    lo1, hi1 = prob["lo"][:1], prob["hi"][:1]
    ib_bigm, ib_as = 100, 100
    opt = binding.default_options(bigm_iters=ib_bigm, as_iters=ib_as, omega=40, max_cuts=3, graph_chunk=25,
                                  autotune=1)
    binding.intermediate_bounds(net, lo1, hi1, None, opt, stream=stream)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    lh, uh = binding.intermediate_bounds(net, lo1, hi1, None, opt, stream=stream)
    e[1].record()
    e[1].synchronize()
    ms = e[0].elapsed_time(e[1])
    widths = [L["n_out"] for L in net[:-1]]
    units = sum(2 * w for w in widths[1:]) * (ib_bigm + ib_as)
    # interval bounds for comparison: a context over the whole net computes them at creation
    ci = binding.Context(net, lo1, hi1, prob["C"][:1], options=binding.default_options(graph_chunk=0))
    il, iu = ci.get_state(binding.ST_LHAT).reshape(1, -1), ci.get_state(binding.ST_UHAT).reshape(1, -1)
    ci.close()
    offs = np.cumsum([0] + widths)
    width_ratio = {f"layer{k}": float(np.sum(uh[0, offs[k - 1]:offs[k]] - lh[0, offs[k - 1]:offs[k]]) /
                                      np.sum(iu[0, offs[k - 1]:offs[k]] - il[0, offs[k - 1]:offs[k]]))
                   for k in range(1, len(widths) + 1)}
    final = {}
    aopt, _ = workload_options(binding)
    for tag, (L, U) in (("interval", (il, iu)), ("tightened", (lh, uh))):
        c = binding.Context(net, prob["lo"], prob["hi"], prob["C"], np.repeat(L, S9, 0), np.repeat(U, S9, 0),
                            options=aopt, stream=stream)
        c.as_step(AS_BIGM + AS_ITERS)
        final[tag] = [float(v) for v in c.bound()]
        c.close()
    gain = np.array(final["tightened"]) - np.array(final["interval"])
    return {"workload": {"net": "wide_conv 3x32x32 conv16-conv32-FC100-FC10", "boxes": 1, "eps": 2.0 / 255.0,
                         "subproblems": {"layer2": 2 * widths[1], "layer3": 2 * widths[2]},
                         "iterations": {"bigm": ib_bigm, "active_set": ib_as, "max_cuts": 3}},
            "value": units / (ms / 1e3), "unit": UNIT, "ms": ms,
            "cpu_baseline": oracle_rate("wide_conv", "layer2") if rank == 0 else None,
            "width_over_interval_width": width_ratio,
            "final_bound_9_properties": {"schedule": f"{AS_BIGM} Big-M + {AS_ITERS} Active Set",
                                         "interval_bounds_mean": float(np.mean(final["interval"])),
                                         "tightened_bounds_mean": float(np.mean(final["tightened"])),
                                         "gain_min": float(gain.min()), "gain_mean": float(gain.mean())}}


def bab_run(binding, torch, dev, stream, rank, time_limit):
    """Branch and bound with stratified bounding (Sec. 6.2) on the wide conv net's box and each of
    its 9 properties in turn: a_l = 180 Big-M iterations, a_t = the same followed by 100 Active Set
    iterations (Sec. 8.2), 256 children per batch, warm starts from the parent, root intermediate
    bounds by 100 Big-M + 100 Active Set iterations; time_limit seconds per property."""
    from paper_2101_05844_gb300 import synth
    prob = synth.problem("wide_conv", seed=rank)
    net, lo, hi = prob["net"], prob["lo"][0], prob["hi"][0]
    opt = binding.bab_default_options(batch=256, time_limit=time_limit, root_intermediate=1,
                                      intermediate=dict(bigm_iters=100, as_iters=100, omega=40, max_cuts=3))
    keys = ("status", "lower", "upper", "bounded", "hard_bounded", "batches", "max_depth", "frontier", "seconds",
            "cost_ratio")
    rows, units, secs = [], 0, 0.0
    it_l = opt.loose.bigm_iters + opt.loose.as_iters
    it_t = opt.tight.bigm_iters + opt.tight.as_iters
    for s in range(prob["C"].shape[0]):
        r = binding.bab(net, lo, hi, prob["C"][s], opt, stream=stream)
        rows.append({k: r[k] for k in keys})
        units += (r["bounded"] - r["hard_bounded"]) * it_l + r["hard_bounded"] * it_t
        secs += r["seconds"]
    verdicts = {v: sum(1 for x in rows if x["status"] == v) for v in ("verified", "falsified", "unknown")}
    return {"workload": {"net": "wide_conv 3x32x32 conv16-conv32-FC100-FC10", "boxes": 1, "eps": 2.0 / 255.0,
                         "properties": len(rows), "batch": 256, "time_limit_s": time_limit,
                         "a_l": f"Big-M {it_l}", "a_t": f"Big-M {opt.tight.bigm_iters} + Active Set {opt.tight.as_iters}"},
            "verdicts": verdicts, "domains_per_s": sum(x["bounded"] for x in rows) / secs,
            "value": units / secs, "unit": UNIT + " (solved domains only, root intermediate bounds included in time)",
            "seconds": secs, "properties": rows}


def l2_run(binding, torch, dev, stream, rank):
    """The headline's Active Set schedule on the wide conv net's 9 properties with the input set the
    l2 ball inscribed in the box (radius eps, as_options.input_l2), timed after a warm-up run,
    beside the same run over the box: subproblem-iterations/s and the final bounds."""
    import numpy as np
    from paper_2101_05844_gb300 import synth
    prob = synth.problem("wide_conv", seed=rank)
    S = prob["lo"].shape[0]
    iters = AS_BIGM + AS_ITERS
    out = {}
    for tag, l2 in (("l2_ball", 1), ("box", 0)):
        opt = binding.default_options(bigm_iters=AS_BIGM, as_iters=AS_ITERS, omega=round(0.3 * AS_ITERS),
                                      max_cuts=5, graph_chunk=25, autotune=1, input_l2=l2)
        ctx = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=opt, stream=stream)
        ctx.as_step(iters)
        ctx.reset(prob["lo"], prob["hi"], prob["C"])
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        ctx.as_step(iters)
        e[1].record()
        e[1].synchronize()
        ms = e[0].elapsed_time(e[1])
        b = ctx.bound()
        ctx.close()
        out[tag] = {"value": S * iters / (ms / 1e3), "ms": ms, "mean_final_bound": float(np.mean(b)),
                    "final_bounds": [float(v) for v in b]}
    return {"workload": {"net": "wide_conv 3x32x32 conv16-conv32-FC100-FC10", "subproblems": S,
                         "iterations": iters, "input_set": "l2 ball of radius 2/255 inscribed in the l_inf box"},
            "unit": UNIT, "cpu_baseline": oracle_rate("wide_conv", "l2") if rank == 0 else None, **out}


def dense_nnz(L):
    """Nonzeros of a layer's dense operator (taps inside the zero padding left out)."""
    if L["kind"] == "linear":
        return L["n_in"] * L["n_out"]
    c, h, w = L["in_shape"]
    oc, oh, ow = L["out_shape"]
    cy = sum(1 for oy in range(oh) for ky in range(L["kh"]) if 0 <= oy * L["stride"] - L["pad"] + ky < h)
    cx = sum(1 for ox in range(ow) for kx in range(L["kw"]) if 0 <= ox * L["stride"] - L["pad"] + kx < w)
    return oc * c * cy * cx


def conv4_slots(opt):
    """Slots each Active Set iteration's col pass (before its addition) and row pass (after it)
    consume, per global iteration (Alg. 1's addition schedule, one mask per iteration)."""
    col, row = [], []
    for it in range(opt.bigm_iters + opt.as_iters):
        if it < opt.bigm_iters:
            col.append(0)
            row.append(0)
            continue
        t = it - opt.bigm_iters
        q, r = divmod(t, opt.omega)
        before = min(q * opt.vars_per_add + min(r, opt.vars_per_add), opt.max_cuts)
        add = 1 if (r < opt.vars_per_add and q * opt.vars_per_add + r < opt.max_cuts) else 0
        col.append(before)
        row.append(before + add)
    return col, row


def colA_bf16_bytes(net, ns, cap):
    """Algorithmic DRAM bytes per subproblem of one BF16-form col-pass launch with ns slots: per input
    j of every layer k (neuron layer k - 1): its box (8), snapshot and fixed bytes (2), x*, f written
    (8); where layer k is hidden, the (1 + ns) W+ / W- products read (8 (1 + ns)) and the operand
    planes written (2 signs x (1 + cap) slots x 2); where j is hidden, alpha, beta_0, beta_1, uhat,
    lhat (20), the slots' beta and kappa (8 ns), z snapshot and z* (2); the output row's weight (4)."""
    total = 0
    n = len(net)
    for k, L in enumerate(net, start=1):
        per = 18
        if k <= n - 1:
            per += 8 * (1 + ns) + 4 * (1 + cap)
        else:
            per += 4
        if k - 1 >= 1:
            per += 22 + 8 * ns
        total += per * L["n_in"]
    return total


def rowB_bf16_bytes(net, ns, cap):
    """Algorithmic DRAM bytes per subproblem of one BF16-form row-pass launch with ns slots: per
    hidden neuron, the (1 + ns) products (4 each), x* (4), z*, z snapshot (2), uhat, lhat (8), alpha,
    beta_0, beta_1 and their six Adam moments read and written (72), the slots' beta, moments,
    lambda, kappa read (20 ns) and beta, moments written (12 ns), the col pass's operand planes
    written (2 (1 + cap))."""
    nh = sum(L["n_out"] for L in net[:-1])
    return nh * (4 * (1 + ns) + 4 + 2 + 8 + 72 + 32 * ns + 2 * (1 + cap))


def tc_flops(net, ns):
    """Algorithmic flops per subproblem of one launch group of the BF16 form's tensor-core products
    (all hidden layers): W x* and the ns masked products, 2 (1 + ns) nnz (the sign split and the
    channel padding the GEMMs also multiply are not counted)."""
    return 2.0 * (1 + ns) * sum(dense_nnz(L) for L in net[:-1])


def conv4_roofline(binding, torch, dev, net, S, kt, opt):
    """The dominant kernel of a profiled step (per-kernel CUDA events) against its roofline."""
    col, row = conv4_slots(opt)
    peaks = measured_peaks()
    total_ms = sum(v[0] for v in kt.values())
    top = max(kt, key=lambda k: kt[k][0])
    tms, n = kt[top]
    out = {"kernel": top, "launches": n, "kernel_ms": tms,
           "share_of_kernel_time": tms / total_ms if total_ms else None}
    if top in ("as_colA", "as_rowB"):
        if top == "as_colA":
            ns_list = col + [col[-1]] * max(0, n - len(col))   # the bound's launch: the last slots
            per = [colA_bf16_bytes(net, k, C4_CAP) for k in ns_list[:n]]
        else:
            per = [rowB_bf16_bytes(net, k, C4_CAP) for k in row[:n]]
        algo = S * float(sum(per))
        gbs = algo / (tms / 1e3) / 1e9
        peak = float(peaks.get("hbm_gbs", 6800.0))
        out.update({"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                    "bytes_per_launch": algo / n,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
                    else "fallback 6.8 TB/s (of fallback)",
                    "traffic": captured_traffic("conv4", top, S),
                    # the captured launch has all C4_CAP slots in use: its algorithmic bytes, to
                    # compare the traffic with (bytes_per_launch averages over the slot schedule)
                    "traffic_launch": f"Active Set iteration with {C4_CAP} slots, captured at 128 boxes, "
                                      "scaled to the batch",
                    "traffic_algorithmic": S * float((colA_bf16_bytes if top == "as_colA" else rowB_bf16_bytes)(
                        net, C4_CAP, C4_CAP))})
    elif top in ("tc_col", "tc_row"):
        nsl = col if top == "tc_col" else row
        layers = len(net) - 1
        per_launch = [tc_flops(net, k) / layers for k in nsl for _ in range(layers)]
        algo = S * float(sum(per_launch[:n]))
        tf = algo / (tms / 1e3) / 1e12
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        out.update({"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured; timed inside a long step)",
                    "traffic": captured_traffic("conv4", top, S)})
    else:
        flops = algorithmic_flops(net, S, top, row, n)
        peak, src = fp32_peak_tflops(torch, dev)
        tf = flops / (tms / 1e3) / 1e12 if tms > 0 else None
        out.update({"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                    "frac": tf / peak if tf else None, "peak_source": src + " (derived)",
                    "traffic": captured_traffic("conv4", top, S)})
    return out


def run_chunks(torch, ctx, batch, iters, chunk, bound):
    """Iterations of a reset context in chunks, CUDA events around each chunk, the bound evaluated
    after each (not timed): (elapsed ms, [(ms so far, bounds)] after every chunk)."""
    lo, hi, C = batch
    ctx.reset(lo, hi, C)
    hist, elapsed = [], 0.0
    for c0 in range(0, iters, chunk):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.as_step(min(chunk, iters - c0))
        e1.record()
        e1.synchronize()
        elapsed += e0.elapsed_time(e1)
        ctx.bound_into(64, bound)
        hist.append((elapsed, bound.cpu().numpy().copy()))
    return elapsed, hist


def reach_summary(hist, targets):
    """Per target: how many subproblems' bounds reached it, and the median and largest time at which
    they first did."""
    out = {}
    for k, tg in targets.items():
        r = np.full(tg.size, np.nan)
        for ms, b in hist:
            r[np.isnan(r) & (b >= tg)] = ms
        done = ~np.isnan(r)
        out[k] = {"reached": int(done.sum()), "of": int(r.size),
                  "median_ms": float(np.median(r[done])) if done.any() else None,
                  "max_ms": float(np.max(r[done])) if done.any() else None}
    return out


def forms_compare(binding, torch, prob, batch, S, stream):
    """The plain float32 form and the BF16 form of the same Active Set schedule on the same batch:
    subproblem-iterations/s (sums of chunk times) and the time to reach the float32 form's final
    bound minus 1e-4 (absolute, and relative to 1 + |bound|: bounds here are 1e4-1e5, where 1e-4
    is below a float32 ulp); the BF16 form also on an 800-iteration schedule of its own (160 Big-M
    + 640 Active Set, omega 192), which it runs in less time than the float32 form's 500."""
    iters, chunk = C4_BIGM + C4_AS, 25
    bound = torch.zeros(S, dtype=torch.float64, device="cuda")
    runs = {}
    for key, opt, n in (("fp32", conv4_options(binding, 32), iters), ("bf16", conv4_options(binding, 16), iters),
                        ("bf16_800", conv4_options(binding, 16, bigm=160, as_iters=640, omega=192), 800)):
        ctx = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=opt, stream=stream)
        runs[key] = (n,) + run_chunks(torch, ctx, batch, n, chunk, bound)
        ctx.close()
    fin32 = runs["fp32"][2][-1][1]
    targets = {"abs_1e-4": fin32 - 1e-4, "rel_1e-4": fin32 - 1e-4 * (1 + np.abs(fin32))}
    out = {}
    for key, (n, ms, hist) in runs.items():
        fin = hist[-1][1]
        gap = fin - fin32
        out[key] = {"value": S * n / (ms / 1e3), "unit": UNIT, "ms": ms, "iterations": n,
                    "mean_final_bound": float(fin.mean()), "time_to_bound": reach_summary(hist, targets),
                    "minus_fp32_final_bound": {"mean": float(gap.mean()), "min": float(gap.min()),
                                               "max": float(gap.max())}}
    t32 = out["fp32"]["time_to_bound"]["rel_1e-4"]["max_ms"]
    t16 = out["bf16_800"]["time_to_bound"]["rel_1e-4"]
    out["time_to_bound"] = {
        "target": "every box's float32-form final bound minus 1e-4 (1 + |bound|), bound re-evaluated in float32",
        "fp32_ms": t32, "bf16_ms": t16["max_ms"] if t16["reached"] == S else None,
        "bf16_reached": t16["reached"], "of": S,
        "speedup": (t32 / t16["max_ms"]) if (t32 and t16["reached"] == S) else None}
    return out


def captured_traffic(workload, kernel, S=None):
    """DRAM bytes per launch of `kernel` from the committed ncu capture of this workload (scaled from
    the captured batch to S subproblems: the traffic of these passes grows with the batch), or None
    when there is none or the kernel source has changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src["path"]), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != src["sha256"]:
                    return None
        v = rec["dram_bytes_per_launch"].get(kernel)
        if v is None:
            return None
        return v * (S / rec["subproblems"]) if S else v
    except (OSError, KeyError, ValueError, TypeError):
        return None


def slowest_rank(values, dist, device):
    """Element-wise maximum of per-rank timings over all ranks (the job is as slow as its slowest
    replica); with one process the values themselves."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(units_per_rank_step, world, ms_per_step):
    """Whole-job subproblem-iterations per second: every rank does units_per_rank_step
    subproblem-iterations per step in ms_per_step (the slowest rank's)."""
    return units_per_rank_step * world / (ms_per_step / 1e3)


SAMPLE_SCHEDULES = {
    # (Big-M iterations, Active Set schedule length, omega, iterations at most) of the oracle sample
    "wide_conv": (4, 200, 15, 40),
    "conv4": (2, 200, 15, 3),
}


def _oracle_sample_code(prob_name, s, seconds_budget, variant=""):
    """A bounded oracle run on subproblem s: variant "" the workload itself, "l2" over the l2 ball
    inscribed in its box, "layer2" the intermediate-bounds subproblem of layer 2's first neuron
    (the sub-network up to the second layer, property row +e_0)."""
    bigm, asi, omega, cap_it = SAMPLE_SCHEDULES.get(prob_name, SAMPLE_SCHEDULES["wide_conv"])
    return f"""
import os, sys, time, json
import numpy as np
sys.path.insert(0, {ROOT!r})
from oracle import active_set as AS, network as nw
from paper_2101_05844_gb300 import synth
prob = synth.problem({prob_name!r}, S={s} + 1, seed=0)
t0 = time.time()
net = prob["net"]
if {variant!r} == "layer2":
    net = net[:2]
    crow = np.zeros(net[1]["n_out"]); crow[0] = 1.0
else:
    crow = prob["C"][{s}]
dense = nw.dense_layers(net)
P = nw.Problem(net, prob["lo"][{s}], prob["hi"][{s}], crow, dense=dense, ball={variant!r} == "l2")
setup = time.time() - t0
opt = AS.Options(bigm_iters={bigm}, as_iters={asi}, omega={omega}, max_cuts=5)
st = AS.ActiveSet(P, opt)
t0 = time.time(); n = 0
while n < {cap_it} and (time.time() - t0) < {seconds_budget}:
    st.step(1); n += 1
dt = time.time() - t0
print(json.dumps({{"iters": n, "seconds": dt, "setup_s": setup}}))
"""


def oracle_rate(prob_name, variant, seconds_budget=10.0):
    """subproblem-iterations/s of one single-threaded oracle run of _oracle_sample_code."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", _oracle_sample_code(prob_name, 0, seconds_budget, variant)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "kind": "oracle", "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["iters"] / d["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one subproblem, {d['iters']} iterations, FP64 numpy, single thread; {d['seconds']:.1f} s"}


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) / 2 ** 20
    except (OSError, ValueError):
        pass
    return 0.0


def cpu_baseline(prob_name, seconds_budget=20.0, all_cores=True):
    """Times the CPU oracle, single-threaded, on a bounded sample of the workload: one subproblem,
    a few Big-M then Active Set iterations (the first with a mask addition; the dense operators are
    built before the timer starts). As context, the same sample on several subproblems at once, one
    single-threaded process each, on as many host cores as memory allows (fresh interpreters, started
    after the GPU work: nothing is forked from a CUDA process)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", _oracle_sample_code(prob_name, 0, seconds_budget)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    bigm = SAMPLE_SCHEDULES.get(prob_name, SAMPLE_SCHEDULES["wide_conv"])[0]
    out = {"value": d["iters"] / d["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"subproblem 0 of the {prob_name} batch, {d['iters']} iterations ({bigm} Big-M, then Active "
                     f"Set with a mask added at its first iteration), FP64 numpy, dense operators (built in "
                     f"{d['setup_s']:.1f} s, not timed), single thread; {d['seconds']:.1f} s"}
    if not all_cores:
        return out
    per_gb = 10.0 if prob_name == "conv4" else 1.0
    k = max(1, min(os.cpu_count() or 1, int(_mem_available_gb() // per_gb), 16))
    procs = [subprocess.Popen([sys.executable, "-c", _oracle_sample_code(prob_name, q, seconds_budget)],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for q in range(k)]
    rates = []
    for p in procs:
        so, _ = p.communicate(timeout=900)
        if p.returncode == 0:
            e = json.loads(so.strip().splitlines()[-1])
            rates.append(e["iters"] / e["seconds"])
    if len(rates) == k:
        out["all_cores"] = {"value": sum(rates), "unit": UNIT, "cores": k, "host_cores": os.cpu_count(),
                            "sample": f"the same sample on {k} subproblems at once, one single-threaded "
                                      f"process each (as many as the host's memory allows, at most its "
                                      f"cores); the sum of their rates"}
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = cpu_baseline(args.workload, seconds_budget=max(10.0, 25.0 / max(1, args.steps)), all_cores=False)
    S = args.subproblems if args.workload == "conv4" else 9
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "subproblems": S, "note": "CPU oracle, bounded sample"},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def wide_conv_run(binding, torch, dev, rank, steps, warmup, flush):
    """The Wide conv net's 9 properties (one box, the earlier headline): an Active Set solve
    (200 Big-M + 800 Active Set) and a Saddle Point solve (200 Big-M + 1000 Saddle Point) per step
    on two streams, timed like the default workload."""
    from paper_2101_05844_gb300 import synth
    prob = synth.problem("wide_conv", seed=rank)
    S = prob["lo"].shape[0]
    batch = tuple(torch.from_numpy(prob[k]).to(dev) for k in ("lo", "hi", "C"))
    outs = [torch.zeros(S, dtype=torch.float64, device=dev) for _ in range(2)]
    as_opt, sp_opt = workload_options(binding)
    s_as, s_sp = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ctx_as = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=as_opt, stream=s_as.cuda_stream)
    ctx_sp = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=sp_opt, stream=s_sp.cuda_stream)
    main = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        wide_step(ctx_as, ctx_sp, batch, outs[0], outs[1])
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        s_as.wait_event(e0)
        s_sp.wait_event(e0)
        wide_step(ctx_as, ctx_sp, batch, outs[0], outs[1])
        main.wait_stream(s_as)
        main.wait_stream(s_sp)
        e1.record(main)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    iters = AS_BIGM + AS_ITERS + SP_BIGM + SP_ITERS
    out = {"workload": "wide_conv: 3x32x32 -> conv16 4x4/2 -> conv32 4x4/2 -> FC100 -> FC10, one box of "
                       "half-width 2/255, its 9 logit-difference properties",
           "value": S * iters / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "subproblems": S,
           "iterations_per_step": {"active_set": AS_BIGM + AS_ITERS, "big_m_before_sp": SP_BIGM,
                                   "saddle_point": SP_ITERS},
           "bounds": {"active_set": [float(v) for v in outs[0].cpu()], "saddle_point": [float(v) for v in outs[1].cpu()]}}
    ctx_as.close()
    ctx_sp.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="conv4", choices=["conv4", "wide_conv"],
                    help="conv4: the default step (1024 boxes); wide_conv: the reference arm's oracle sample "
                         "on the Wide conv net")
    ap.add_argument("--subproblems", type=int, default=C4_S,
                    help="boxes of the conv4 batch (1024; fewer only for a profiler capture)")
    ap.add_argument("--profile-only", action="store_true",
                    help="only warm-up and timed steps of the conv4 workload, nothing else (profiler captures)")
    ap.add_argument("--form", default="bf16", choices=["bf16", "fp32"],
                    help="form of the conv4 step's Active Set products (bf16: the default line; fp32 only "
                         "with --profile-only, for captures of the float32 passes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the float32 / BF16 comparison")
    ap.add_argument("--no-wide", action="store_true", help="skip the Wide conv extra key")
    ap.add_argument("--differentiation", action="store_true",
                    help="also time the differentiation workload: MLP 784-1024x3-10, 256 boxes, 300 "
                         "Active Set iterations, then the bound and its envelope gradient")
    ap.add_argument("--batched", action="store_true",
                    help="also time the batching workload: 4096 subdomains, 500 Active Set iterations")
    ap.add_argument("--intermediate", action="store_true",
                    help="also time intermediate bounds by batched sub-network solves on the wide conv "
                         "net (one box, layers 2 and 3) and the final bounds they give")
    ap.add_argument("--bab", action="store_true",
                    help="also run branch and bound with stratified bounding on the wide conv net's 9 properties")
    ap.add_argument("--bab-time", type=float, default=10.0, help="time limit per property of --bab (seconds)")
    ap.add_argument("--l2", action="store_true",
                    help="also time the Wide conv Active Set schedule over the l2 ball inscribed in each box")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch

    from paper_2101_05844_gb300 import binding, synth
    from paper_2101_05844_gb300.shard import gather_bounds, shard_batch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    binding.lib()
    dev = torch.device("cuda", local)

    # one batch of world x subproblems boxes; each rank bounds its contiguous slice (weak scaling:
    # the slice stays the same size as ranks are added) and the bounds are gathered once per step
    a, b = shard_batch(args.subproblems * world, world, rank)
    S = b - a
    prob = synth.problem("conv4", S=args.subproblems * world, seed=0, part=(a, b))
    batch_d = tuple(torch.from_numpy(prob[k]).to(dev) for k in ("lo", "hi", "C"))
    batch_h = tuple(torch.from_numpy(prob[k]).pin_memory() for k in ("lo", "hi", "C"))
    out_d = [torch.zeros(S, dtype=torch.float64, device=dev) for _ in range(2)]
    out_h = [torch.zeros(S, dtype=torch.float64).pin_memory() for _ in range(2)]
    stream = torch.cuda.current_stream(dev).cuda_stream
    if args.form == "fp32" and not args.profile_only:
        ap.error("--form fp32 is for profiler captures (--profile-only); the line reports both forms")
    ctx = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"],
                          options=conv4_options(binding, 16 if args.form == "bf16" else 32), stream=stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(batch, outs, k):
        times, parts = [], []
        for _ in range(k):
            flush.fill_(1.0)                      # evict L2 between steps
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            conv4_step(ctx, batch, outs[0], outs[1], ev)
            if dist:     # the job's best bound per box, in batch order, on every rank (its only collective)
                gather_bounds(torch.maximum(outs[0], outs[1]).to(dev), args.subproblems * world, dist)
                ev[2].record()
            ev[2].synchronize()
            times.append(ev[0].elapsed_time(ev[2]))
            parts.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])))
        return times, parts

    for _ in range(args.warmup):
        conv4_step(ctx, batch_d, out_d[0], out_d[1])
    barrier()
    l0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        times, parts = timed(batch_d, out_d, args.steps)
        barrier()
    launches = ctx.launch_count() - l0
    if args.profile_only:
        if rank == 0:
            print(json.dumps({"profile_only": True, "ms_per_step": sum(times) / len(times), "subproblems": S}))
        return
    # end to end through the API with the batch in pinned host memory and the bounds read back
    for _ in range(max(1, args.warmup // 2)):
        conv4_step(ctx, batch_h, out_h[0], out_h[1])
    barrier()
    e2e_times, _ = timed(batch_h, out_h, args.steps)
    barrier()
    bounds_as, bounds_sp = out_h[0].numpy().copy(), out_h[1].numpy().copy()

    per_step = S * (C4_BIGM + C4_AS + C4_SP_ITERS)
    ms, ms_e2e = slowest_rank([sum(times) / len(times), sum(e2e_times) / len(e2e_times)], dist, dev)
    value = job_throughput(per_step, world, ms)
    ms_as = sum(p[0] for p in parts) / len(parts)
    ms_sp = sum(p[1] for p in parts) / len(parts)

    # per-kernel device time of one profiled step (CUDA events around each launch) for the roofline
    popt = conv4_options(binding, 16, profile=1, graph_chunk=0)
    pc = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=popt, stream=stream)
    kt0 = pc.kernel_times()   # as_init's own launches (its batch set-up) are not the step's
    conv4_step(pc, batch_d, out_d[0], out_d[1])
    kt = {k: (v[0] - kt0[k][0], v[1] - kt0[k][1]) for k, v in pc.kernel_times().items() if v[1] > kt0[k][1]}
    pc.close()
    roof = conv4_roofline(binding, torch, dev, prob["net"], S, kt, popt)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "conv4", "net": "3x32x32 -> 4 conv 3x3 (32, 32, 64, 64; s1, s2, s1, s2) -> FC512 -> FC10",
                   "subproblems_per_gpu": S, "eps": "8/255",
                   "iterations_per_step": {"big_m": C4_BIGM, "active_set": C4_AS, "saddle_point": C4_SP_ITERS,
                                           "saddle_point_primal_init_steps": C4_SP_INIT},
                   "form": "BF16 products on the tensor cores, float32 duals and Adam, bound in float32 with "
                           "float64 summation; Saddle Point in float32",
                   "l2": "flushed between timed steps (write of 2x L2); the batch's state is several GB",
                   "parallelism": f"batch sharded over {world} GPU(s): contiguous slices, network replicated, "
                                  f"one gather of the bounds per step"},
        "parts": {"active_set_bf16": {"ms": ms_as, "value": S * (C4_BIGM + C4_AS) / (ms_as / 1e3), "unit": UNIT},
                  "saddle_point": {"ms": ms_sp, "value": S * C4_SP_ITERS / (ms_sp / 1e3), "unit": UNIT,
                                   "note": "conversion, primal initialisation and iterations"}},
        "e2e": {"value": job_throughput(per_step, world, ms_e2e), "unit": UNIT, "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in batch_h),
                "d2h_bytes_per_step": 2 * S * 8},
        "gpu_launches": launches,
        "roofline": roof,
        "kernel_ms_per_step": {k: v[0] for k, v in kt.items()},
        "clocks": clk.summary(),
        "bounds": {"active_set_mean": float(bounds_as.mean()), "saddle_point_mean": float(bounds_sp.mean())},
    }
    ctx.close()
    if not args.no_forms:
        line["forms"] = forms_compare(binding, torch, prob, batch_d, S, stream)
    if not args.no_wide:
        line["wide_conv"] = wide_conv_run(binding, torch, dev, rank, args.steps, args.warmup, flush)
    if args.batched:
        line["batched"] = batched_run(binding, torch, dev, stream, rank)
    if args.differentiation:
        line["differentiation"] = differentiation_run(binding, torch, dev, stream, rank)
    if args.l2:
        line["l2"] = l2_run(binding, torch, dev, stream, rank)
    if args.bab:
        line["bab"] = bab_run(binding, torch, dev, stream, rank, args.bab_time)
    if args.intermediate:
        line["intermediate"] = intermediate_run(binding, torch, dev, stream, rank)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline("conv4", seconds_budget=25.0)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

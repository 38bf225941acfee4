"""Benchmark of the batched Active Set / Saddle Point hot path on one or more GB300 GPUs.

One step bounds one batch of the workload end to end through the C ABI:
  Active Set: reset (interval bounds) + 200 Big-M + 800 Active Set iterations + bound;
  Saddle Point: reset + 200 Big-M + 1000 Saddle Point iterations (conversion and 100 primal
  initialisation steps included) + bound.
Default workload: the paper's "Wide" conv net (3x32x32 -> conv16 4x4/2 -> conv32 4x4/2 -> FC100
-> FC10), one L-infinity box of radius 2/255 around a U[0,1] image, the 9 logit-difference
properties as 9 subproblems; synthetic He-initialised weights.

Output: one JSON line (rank 0). value = subproblem-iterations per second over the whole step,
inputs resident on the device; e2e = the same with the batch in pinned host memory and the
bounds read back to the host, copies inside the timed region; roofline = the dominant kernel's
achieved FP32 rate against the FP32 ALU peak; cpu_baseline = the CPU oracle on a bounded sample.
--impl reference times the CPU oracle as the reference arm.
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
SM_COUNT = 152
FP32_LANES_PER_SM = 128

AS_BIGM, AS_ITERS, SP_BIGM, SP_ITERS = 200, 800, 200, 1000


def workload_options(binding, profile=0):
    # autotune: each context times its passes' team sizes on its own net and batch at creation
    as_opt = binding.default_options(bigm_iters=AS_BIGM, as_iters=AS_ITERS, omega=round(0.3 * AS_ITERS),
                                     max_cuts=5, graph_chunk=25, profile=profile, autotune=1)
    sp_opt = binding.default_options(bigm_iters=SP_BIGM, as_iters=0, max_cuts=5, graph_chunk=25,
                                     profile=profile, autotune=1)
    return as_opt, sp_opt


def iterations_per_step():
    return AS_BIGM + AS_ITERS + SP_BIGM + SP_ITERS


def run_step(ctx_as, ctx_sp, batch, out_as, out_sp):
    """One step: the Active Set solve and the Saddle Point solve of the batch. The two contexts are
    independent; when they sit on different streams their launches overlap on the GPU (all work
    is enqueued before the first bound evaluation, which waits for its own stream)."""
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
    run(pc)
    kt = pc.kernel_times()
    top = max(kt, key=lambda k: kt[k][0])
    sched = slots_schedule(opt)
    # per-subdomain caps: the mean active-set size follows min(slots, cap)
    caps = prob["caps"].astype(float)
    mean_slots = [float(np.minimum(k, caps).mean()) for k in sched]
    flops = algorithmic_flops(prob["net"], S, top, mean_slots, kt[top][1])
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12
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


def precision_run(binding, torch, dev, stream, rank, S=1024, chunk=25):
    """The precision workload: the conv net 3x32x32 -> 4 conv 3x3 -> FC512 -> FC10 on S boxes of
    half-width 8/255, 100 Big-M + 400 Active Set iterations, once in float32 and once in the BF16
    form (tensor-core products, precision 16), same schedule, same GPU. Reports each form's
    subproblem-iterations/s (one timed run after a warm-up) and the time to bound: iteration time
    (CUDA events around each chunk of iterations; the bound evaluations between chunks are not
    counted) until a subproblem's bound, re-evaluated in float32, first reaches the float32
    form's final bound minus 1e-4 (absolute, and relative to 1 + |bound|); the BF16 form also on
    an 800-iteration schedule of its own."""
    from paper_2101_05844_gb300 import synth
    prob = synth.problem("conv4", S=S, seed=rank)
    iters = 500
    t = {k: torch.from_numpy(prob[k]).to(dev) for k in ("lo", "hi", "C")}
    out = {}
    finals = {}
    ctxs = {}
    for prec in (32, 16):
        opt = binding.default_options(bigm_iters=100, as_iters=400, omega=120, max_cuts=5, graph_chunk=25,
                                      precision=prec)
        ctxs[prec] = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=opt, stream=stream)
    bound = torch.zeros(S, dtype=torch.float64, device=dev)
    for prec, ctx in ctxs.items():
        ctx.reset(t["lo"], t["hi"], t["C"])
        ctx.as_step(iters)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.reset(t["lo"], t["hi"], t["C"])
        e0.record()
        ctx.as_step(iters)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        ctx.bound_into(64, bound)
        finals[prec] = bound.cpu().numpy().copy()
        out[f"fp{prec}" if prec == 32 else "bf16"] = {"value": S * iters / (ms / 1e3), "unit": UNIT, "ms": ms,
                                                       "mean_final_bound": float(finals[prec].mean())}
    # the bound a form must reach: the float32 form's final bound less 1e-4, absolute, and less
    # 1e-4 (1 + |bound|) (bounds here reach 1e4-1e5, where 1e-4 is below a float32 ulp)
    targets = {"abs_1e-4": finals[32] - 1e-4, "rel_1e-4": finals[32] - 1e-4 * (1 + np.abs(finals[32]))}
    for prec, ctx in ctxs.items():
        ctx.reset(t["lo"], t["hi"], t["C"])
        reach = {k: np.full(S, np.nan) for k in targets}
        elapsed = 0.0
        for c0 in range(0, iters, chunk):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.as_step(min(chunk, iters - c0))
            e1.record()
            e1.synchronize()
            elapsed += e0.elapsed_time(e1)
            ctx.bound_into(64, bound)
            b = bound.cpu().numpy()
            for k, tg in targets.items():
                new = np.isnan(reach[k]) & (b >= tg)
                reach[k][new] = elapsed
        key = "fp32" if prec == 32 else "bf16"
        out[key]["time_to_bound_ms"] = {}
        for k, r in reach.items():
            done = ~np.isnan(r)
            out[key]["time_to_bound_ms"][k] = {"reached": int(done.sum()), "of": S,
                                               "median": float(np.median(r[done])) if done.any() else None,
                                               "max": float(np.max(r[done])) if done.any() else None}
    gap = finals[16] - finals[32]
    out["bf16_minus_fp32_final_bound"] = {"mean": float(gap.mean()), "min": float(gap.min()), "max": float(gap.max())}
    # the BF16 form on a schedule of its own: 800 iterations (160 Big-M + 640 Active Set, the
    # learning rates stretched over them), about the float32 form's 500 iterations in wall time
    long_opt = binding.default_options(bigm_iters=160, as_iters=640, omega=192, max_cuts=5, graph_chunk=25,
                                       precision=16)
    lc = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=long_opt, stream=stream)
    lc.reset(t["lo"], t["hi"], t["C"])
    reach = {k: np.full(S, np.nan) for k in targets}
    elapsed = 0.0
    for c0 in range(0, 800, chunk):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lc.as_step(chunk)
        e1.record()
        e1.synchronize()
        elapsed += e0.elapsed_time(e1)
        lc.bound_into(64, bound)
        b = bound.cpu().numpy()
        for k, tg in targets.items():
            new = np.isnan(reach[k]) & (b >= tg)
            reach[k][new] = elapsed
    fin = bound.cpu().numpy().copy()
    out["bf16_800"] = {"ms": elapsed, "mean_final_bound": float(fin.mean()),
                       "minus_fp32_final_bound_mean": float((fin - finals[32]).mean()), "time_to_bound_ms": {}}
    for k, r in reach.items():
        done = ~np.isnan(r)
        out["bf16_800"]["time_to_bound_ms"][k] = {"reached": int(done.sum()), "of": S,
                                                  "median": float(np.median(r[done])) if done.any() else None,
                                                  "max": float(np.max(r[done])) if done.any() else None}
    lc.close()
    # per-kernel device time of 60 iterations (20 Big-M + 40 Active Set, 5 slots), each form
    out["kernel_ms_60_iterations"] = {}
    for prec in (32, 16):
        popt = binding.default_options(bigm_iters=20, as_iters=40, omega=12, max_cuts=5, graph_chunk=0, profile=1,
                                       precision=prec)
        pc = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=popt, stream=stream)
        pc.as_step(60)
        out["kernel_ms_60_iterations"]["fp32" if prec == 32 else "bf16"] = {
            k: v[0] for k, v in pc.kernel_times().items() if v[1]}
        pc.close()
    out["workload"] = {"net": "conv4", "subproblems": S, "iterations": iters, "eps": "8/255"}
    for ctx in ctxs.values():
        ctx.close()
    return out


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


def hbm_rooflines(workload, kt):
    """The HBM side of the roofline for every kernel with a committed DRAM capture: measured DRAM
    bytes per launch (ncu, the captured build) over this run's mean launch duration (CUDA events),
    against the measured copy bandwidth of MEASURED_PEAKS.json."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, src = float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        peak, src = 6800.0, "fallback 6.8 TB/s"
    out = {}
    for k, (tms, n) in kt.items():
        t = captured_traffic(workload, k)
        if t is None or not n or tms <= 0:
            continue
        us = tms / n * 1e3
        gbs = t / (us * 1e-6) / 1e9
        out[k] = {"dram_bytes_per_launch": t, "launch_us": us, "achieved": gbs, "peak": peak, "unit": "GB/s",
                  "frac": gbs / peak, "peak_source": src}
    return out


def captured_traffic(workload, kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu capture of this workload, or None
    when there is none or the kernel source has changed since it was taken."""
    import hashlib
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", f"dram_traffic_{workload}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        src = os.path.join(os.path.dirname(os.path.abspath(__file__)), rec["source"])
        with open(src, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != rec["source_sha256"]:
                return None
        return rec["dram_bytes_per_launch"].get(kernel)
    except (OSError, KeyError, ValueError):
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


def job_throughput(S_per_rank, world, ms_per_step):
    """Whole-job subproblem-iterations per second: every rank bounds its own batch of S_per_rank
    subproblems for iterations_per_step() iterations in ms_per_step (the slowest rank's)."""
    return S_per_rank * iterations_per_step() * world / (ms_per_step / 1e3)


def _oracle_sample_code(prob_name, s, seconds_budget, variant=""):
    """A bounded oracle run on subproblem s: variant "" the workload itself, "l2" over the l2 ball
    inscribed in its box, "layer2" the intermediate-bounds subproblem of layer 2's first neuron
    (the sub-network up to the second layer, property row +e_0)."""
    return f"""
import os, sys, time, json
import numpy as np
sys.path.insert(0, {ROOT!r})
from oracle import active_set as AS, network as nw
from paper_2101_05844_gb300 import synth
prob = synth.problem({prob_name!r}, seed=0)
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
opt = AS.Options(bigm_iters=4, as_iters=200, omega=15, max_cuts=5)
st = AS.ActiveSet(P, opt)
t0 = time.time(); n = 0
while n < 40 and (time.time() - t0) < {seconds_budget}:
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


def cpu_baseline(prob_name, seconds_budget=20.0):
    """Times the CPU oracle, single-threaded, on a bounded sample of the workload: one subproblem,
    a few Big-M then Active Set iterations (with the two first mask additions). As context, the
    same sample on every subproblem at once, one single-threaded process each on the host's cores
    (fresh interpreters, started after the GPU work: nothing is forked from a CUDA process)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", _oracle_sample_code(prob_name, 0, seconds_budget)],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    out = {"value": d["iters"] / d["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"1 of the 9 subproblems, {d['iters']} iterations (4 Big-M, then Active Set, masks "
                     f"added at Active Set iterations 0, 1, 15, 16, 30), FP64 numpy, dense conv "
                     f"operators, single thread; {d['seconds']:.1f} s"}
    from paper_2101_05844_gb300 import synth
    S = synth.problem(prob_name, seed=0)["lo"].shape[0]
    k = max(1, min(os.cpu_count() or 1, S))
    procs = [subprocess.Popen([sys.executable, "-c", _oracle_sample_code(prob_name, q, seconds_budget / 2)],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for q in range(k)]
    rates = []
    for p in procs:
        so, _ = p.communicate(timeout=600)
        if p.returncode == 0:
            e = json.loads(so.strip().splitlines()[-1])
            rates.append(e["iters"] / e["seconds"])
    if len(rates) == k:
        out["all_cores"] = {"value": sum(rates), "unit": UNIT, "cores": k, "host_cores": os.cpu_count(),
                            "sample": f"the same sample on {k} subproblems at once, one single-threaded "
                                      f"process each; the sum of their rates"}
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = cpu_baseline(args.workload, seconds_budget=max(10.0, 20.0 / max(1, args.steps)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "subproblems": 9, "note": "CPU oracle, bounded sample"},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="wide_conv")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", action="store_true",
                    help="also time the precision workload: conv4 on 1024 boxes, float32 against the "
                         "BF16 form, subproblem-iterations/s and time to the float32 bound")
    ap.add_argument("--precision-subproblems", type=int, default=1024,
                    help="boxes of the precision form (1024 by default; fewer for a profiler capture)")
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
                    help="also time the headline Active Set schedule over the l2 ball inscribed in each box")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return

    import numpy as np
    import torch

    from paper_2101_05844_gb300 import binding, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    binding.lib()

    prob = synth.problem(args.workload, seed=rank)   # each rank bounds its own batch (weak scaling)
    S = prob["lo"].shape[0]
    dev = torch.device("cuda", local)
    lo_d = torch.from_numpy(prob["lo"]).to(dev)
    hi_d = torch.from_numpy(prob["hi"]).to(dev)
    C_d = torch.from_numpy(prob["C"]).to(dev)
    lo_h = torch.from_numpy(prob["lo"]).pin_memory()
    hi_h = torch.from_numpy(prob["hi"]).pin_memory()
    C_h = torch.from_numpy(prob["C"]).pin_memory()
    out_d = [torch.zeros(S, dtype=torch.float64, device=dev) for _ in range(2)]
    out_h = [torch.zeros(S, dtype=torch.float64).pin_memory() for _ in range(2)]
    as_opt, sp_opt = workload_options(binding)
    stream = torch.cuda.current_stream().cuda_stream
    # the step's two solves on streams of their own (joined to the timing stream by events)
    s_as, s_sp = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ctx_as = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=as_opt,
                             stream=s_as.cuda_stream)
    ctx_sp = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=sp_opt,
                             stream=s_sp.cuda_stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(batch, outs, k):
        times = []
        main = torch.cuda.current_stream(dev)
        for _ in range(k):
            flush.fill_(1.0)                      # evict L2 between steps
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            s_as.wait_event(e0)
            s_sp.wait_event(e0)
            run_step(ctx_as, ctx_sp, batch, outs[0], outs[1])
            main.wait_stream(s_as)
            main.wait_stream(s_sp)
            e1.record(main)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    torch.cuda.synchronize()
    for _ in range(args.warmup):
        run_step(ctx_as, ctx_sp, (lo_d, hi_d, C_d), out_d[0], out_d[1])
    barrier()
    l0 = ctx_as.launch_count() + ctx_sp.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        times = timed((lo_d, hi_d, C_d), out_d, args.steps)
        barrier()
    launches = ctx_as.launch_count() + ctx_sp.launch_count() - l0
    # end to end through the API with host buffers
    for _ in range(max(1, args.warmup // 2)):
        run_step(ctx_as, ctx_sp, (lo_h, hi_h, C_h), out_h[0], out_h[1])
    barrier()
    e2e_times = timed((lo_h, hi_h, C_h), out_h, args.steps)
    barrier()
    bounds_as = out_h[0].numpy().copy()
    bounds_sp = out_h[1].numpy().copy()

    ms, ms_e2e = slowest_rank([sum(times) / len(times), sum(e2e_times) / len(e2e_times)], dist, dev)
    value = job_throughput(S, world, ms)
    e2e_value = job_throughput(S, world, ms_e2e)

    # per-kernel device time for the roofline: one profiled step (CUDA events around each launch)
    as_p, sp_p = workload_options(binding, profile=1)
    pa = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=as_p, stream=stream)
    ps = binding.Context(prob["net"], prob["lo"], prob["hi"], prob["C"], options=sp_p, stream=stream)
    run_step(pa, ps, (lo_d, hi_d, C_d), out_d[0], out_d[1])
    kt = {}
    for ctx in (pa, ps):
        for name, (tms, n) in ctx.kernel_times().items():
            a, b = kt.get(name, (0.0, 0))
            kt[name] = (a + tms, b + n)
    top = max(kt, key=lambda k: kt[k][0])
    sched = slots_schedule(as_opt)
    tms, n = kt[top]
    flops = algorithmic_flops(prob["net"], S, top, sched, n)
    peak_tflops = SM_COUNT * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12
    achieved = flops / (tms / 1e3) / 1e12 if tms > 0 else None
    step_kernel_ms = sum(v[0] for v in kt.values())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "subproblems_per_gpu": S,
                   "iterations_per_step": {"active_set": AS_BIGM + AS_ITERS, "big_m_before_sp": SP_BIGM,
                                           "saddle_point": SP_ITERS},
                   "l2": "flushed between timed steps (write of 2x L2)", "parallelism": f"replicas x{world}",
                   "team_targets": {"active_set": list(ctx_as.team_targets()),
                                    "saddle_point": list(ctx_sp.team_targets())}},
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": 2 * (lo_h.numel() * 4 + hi_h.numel() * 4 + C_h.numel() * 4),
                "d2h_bytes_per_step": 2 * S * 8},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": top, "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": (achieved / peak_tflops) if achieved else None,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (derived)",
                     "traffic": captured_traffic(args.workload, top), "launches": n, "kernel_ms": tms,
                     "share_of_kernel_time": tms / step_kernel_ms if step_kernel_ms else None},
        "roofline_hbm": hbm_rooflines(args.workload, kt),
        "kernel_ms_per_step": {k: v[0] for k, v in kt.items() if v[1]},
        "clocks": clk.summary(),
        "bounds": {"active_set": [float(v) for v in bounds_as], "saddle_point": [float(v) for v in bounds_sp]},
    }
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
    if args.precision:
        line["precision"] = precision_run(binding, torch, dev, stream, rank, S=args.precision_subproblems)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    if rank == 0:
        print(json.dumps(line))
    for c in (ctx_as, ctx_sp, pa, ps):
        c.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

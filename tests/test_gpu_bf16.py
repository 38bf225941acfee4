"""The BF16 form of the Active Set passes (as_options.precision = 16) against the FP64 oracle.

The BF16 form rounds the operands of every product to bf16 (W, x*, and the dual row sums) and
accumulates in float32 on the tensor cores. A bf16 rounding moves an operand by at most 2^-9 of
itself, so a product moves by at most (2^-9 + 2^-9 + 2^-18) of |w| |v|, and a sum of products by at
most 2^-8 of sum |w| |v| plus float32 accumulation. The tests use the bound
    e = 2^-7 sum |w| |v|
(twice that, which also covers float32 accumulation at these sizes) for every sum the form takes on
the tensor cores, and check:
  * one iteration from a drawn state (installed on both sides, nothing taken from the GPU): z* is
    exact (its coefficients need no products), x* equals the oracle's wherever the oracle's |f|
    clears e, and every dual lies in the range of the oracle's own Adam step over gradients
    within e of the oracle's (slack 1e-7 + 1e-5 relative: the Adam step itself runs in float32, as
    in the float32 form, whose lockstep tolerance this is);
    An input whose x* the GPU takes the other way (only possible within that bound) widens the
    bound of the rows it feeds by |W| (|l| + |u|); a row whose own x* differs is checked for
    validity only, and at least 90% of the rows must be checked in full;
  * free-running solves: every bound, which as_bound re-evaluates in float32 with float32 lambda,
    kappa, is valid (below the network's minimum over sampled inputs and box vertices, and, on a
    six-neuron net, below the exact LP over the tighter relaxation), and stays within the stated
    gap of the oracle's own FP64 run with the same schedule.
"""
import numpy as np
import pytest

from oracle import active_set as AS
from oracle import dual as du
from oracle import network as nw
from oracle import relaxation as rx
from paper_2101_05844_gb300 import binding, synth
from tests.helpers import netlp_for, sample_min_output
from tests.state_helpers import conv4_full_batch, draw_state, hidden_concat, oracle_bounds_f32, split_hidden

pytestmark = pytest.mark.gpu
E_REL = 2.0 ** -7
# stated gap of the BF16 form's final bound to the oracle's FP64 run with the same schedule, per
# unit of 1 + |bound| (measured on GB300: 0.9e-3 to 4.1e-3 on the three free-running nets)
GAP = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    binding.lib()


def _adam_range(theta, m, v, g, e, lr, step, opt):
    """Range of one oracle Adam step (AS.adam) over gradients in [g - e, g + e]. The step is not
    monotone in g: with a = b1 m, c = 1 - b1, d = b2 v, h = 1 - b2 the update is proportional to
    (a + c g) / sqrt(d + h g^2) (up to eps), whose one stationary point is g* = c d / (a h). The
    interval is sampled densely, and g* (with a fine grid around it, for eps) is added where it
    lies inside."""
    g = np.asarray(g, np.float64)
    e = np.broadcast_to(np.asarray(e, np.float64), g.shape)
    cands = [g + d * e for d in np.linspace(-1.0, 1.0, 129)]
    with np.errstate(divide="ignore", invalid="ignore"):
        gs = (1 - opt.adam_b1) * opt.adam_b2 * v / (opt.adam_b1 * (1 - opt.adam_b2) * m)
    gs = np.where(np.isfinite(gs), gs, g)
    for r in np.linspace(-1e-3, 1e-3, 21):
        cands.append(np.clip(gs * (1 + r), g - e, g + e))
    outs = []
    for gg in cands:
        th, mm, vv = theta.copy(), m.copy(), v.copy()
        AS.adam(th, mm, vv, gg, lr, step, opt)
        outs.append(th)
    return np.min(outs, 0), np.max(outs, 0)


CASES = [
    ("mlp_tiny", 1, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 3, 0),     # Big-M
    ("mlp_tiny", 1, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 7, 2),     # AS, no addition
    ("mlp_tiny", 1, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 8, 2),     # AS, adds slot 2
    ("small_conv", 3, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 12, 4),  # stride 2 + 1, adds 4
    ("small_conv", 3, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=7), 10, 3),
    ("mlp_5_7_6_3", 4, dict(bigm_iters=2, as_iters=30, omega=4, max_cuts=8), 16, 6),  # adds slot 6
    ("wide_conv", 9, dict(bigm_iters=5, as_iters=40, omega=3, max_cuts=5), 12, 4),   # 4x4 stride 2
]


def pre_step(solvers):
    """The oracle solvers' values before the step (the range check needs them after the oracle's own
    step)."""
    return {s: dict(alpha=[None if a is None else a.copy() for a in sv.st.alpha],
                    beta0=[None if a is None else a.copy() for a in sv.st.beta0],
                    beta1=[None if a is None else a.copy() for a in sv.st.beta1],
                    m={q: [None if a is None else a.copy() for a in sv.m[q]] for q in sv.m},
                    v={q: [None if a is None else a.copy() for a in sv.v[q]] for q in sv.v},
                    slots=[[(sl.beta.copy(), sl.m.copy(), sl.v.copy(), sl.added_at) for sl in sv.st.slots[k]]
                           for k in range(sv.P.n)]) for s, sv in solvers.items()}


def check_bf16_step(ctx, solvers, pre, it, t, lr, opt):
    """After one GPU iteration of the BF16 form from the drawn state: z* exact, x* equal wherever
    the oracle's |f| clears the bf16 bound, every dual in the range of the oracle's Adam step over
    gradients within the bound (solvers, pre: dicts over the checked subproblems; the oracle
    solvers take their own step here). Returns (rows checked in full, rows)."""
    S = ctx.S
    xstar = ctx.get_state(binding.ST_XSTAR).reshape(S, -1)
    zstar = ctx.get_state(binding.ST_ZSTAR, np.uint8).reshape(S, -1)
    al = ctx.get_state(binding.ST_ALPHA).reshape(S, -1)
    b0 = ctx.get_state(binding.ST_BETA0).reshape(S, -1)
    b1 = ctx.get_state(binding.ST_BETA1).reshape(S, -1)
    sb = ctx.get_state(binding.ST_SLOT_BETA).reshape(S, ctx.cap, -1)
    rows_checked = rows_total = 0
    for s, sv in solvers.items():
        P = sv.P
        _, f, g, x, z = du.evaluate(P, sv.st)
        grads = du.supergradient(P, sv.st, x, z)
        offs_t = np.cumsum([0] + P.widths)
        np.testing.assert_array_equal(zstar[s], hidden_concat(z).astype(np.uint8))
        xo = np.concatenate([x[k] for k in range(P.n)]).astype(np.float32)
        # bf16 error bound of f: col sums over |W| |dual row sums|
        ef = [None] * P.n
        for k in range(1, P.n):
            rows = np.abs(sv.st.alpha[k]) + np.abs(sv.st.beta1[k]) + sum(np.abs(sl.beta) for sl in sv.st.slots[k])
            ef[k - 1] = E_REL * (np.abs(P.W[k]).T @ rows) + 1e-6
        ef[P.n - 1] = np.full(P.widths[P.n - 1], 1e-6)   # f of the last hidden layer: no product
        decided = np.concatenate([np.abs(f[k]) > ef[k] for k in range(P.n)])
        np.testing.assert_array_equal(xstar[s][decided], xo[decided])
        mism = [xstar[s][offs_t[k]:offs_t[k + 1]] != xo[offs_t[k]:offs_t[k + 1]] for k in range(P.n)]
        # bf16 error bound of the row sums (W x*, masked products) over |W| |x*|, widened by every
        # input whose x* the GPU took the other way (within the bound above): |W| (|l| + |u|)
        ex = [None] * P.n
        for k in range(1, P.n):
            far = mism[k - 1] * (np.abs(P.lo[k - 1]) + np.abs(P.hi[k - 1]))
            ex[k] = E_REL * (np.abs(P.W[k]) @ np.abs(x[k - 1])) + np.abs(P.W[k]) @ far + 1e-6
        slots_before = len(sv.st.slots[1])
        sv.step(1)
        pr = pre[s]

        def in_range(gpu, theta, m, v, gr, e, step, own):
            """gpu within the oracle's Adam step range; rows whose own x* differs: validity only."""
            lo, hi = _adam_range(theta, m, v, gr, e, lr, step, opt)
            slack = 1e-7 + 1e-5 * np.abs(hi)   # the float32 Adam step: the float32 lockstep's tolerance
            ok = (gpu >= lo - slack) & (gpu <= hi + slack)
            if not (ok | own).all():
                q = int(np.argmax(np.where(own, -np.inf, np.maximum(lo - gpu, gpu - hi))))
                # the gradient that gives the GPU's value, by a scan of the oracle's Adam step
                gs = gr[q] + np.linspace(-20, 20, 4001) * e[q] if np.ndim(e) else gr[q] + np.linspace(-20, 20, 4001) * e
                tq = np.full(gs.size, theta[q]); mq = np.full(gs.size, m[q]); vq = np.full(gs.size, v[q])
                AS.adam(tq, mq, vq, gs, lr, step, opt)
                gimp = float(gs[np.argmin(np.abs(tq - gpu[q]))])
                eq = float(e[q]) if np.ndim(e) else float(e)
                raise AssertionError(f"entry {q}: gpu {gpu[q]:.9g} not in [{lo[q]:.9g}, {hi[q]:.9g}]; theta {theta[q]:.6g}"
                                     f" m {m[q]:.6g} v {v[q]:.6g}; oracle g {gr[q]:.6g} e {eq:.3g}; implied g {gimp:.6g};"
                                     f" lr {lr:.6g} step {step}")
            assert (gpu >= 0).all()

        offs = offs_t - P.widths[0]
        for k in range(1, P.n):
            h = slice(offs[k], offs[k + 1])
            own = mism[k]
            rows_checked += int((~own).sum())
            rows_total += own.size
            in_range(al[s, h], pr["alpha"][k], pr["m"]["a"][k], pr["v"]["a"][k], grads["galpha"][k], ex[k], it + 1,
                     own)
            in_range(b0[s, h], pr["beta0"][k], pr["m"]["0"][k], pr["v"]["0"][k], grads["gbeta0"][k], 1e-6, it + 1,
                     own)
            in_range(b1[s, h], pr["beta1"][k], pr["m"]["1"][k], pr["v"]["1"][k], grads["gbeta1"][k], ex[k], it + 1,
                     own)
            for b, (beta, m, v, added) in enumerate(pr["slots"][k]):
                in_range(sb[s, b, h], beta, m, v, grads["gslots"][k][b], 2 * ex[k], t - added + 1, own)
            if len(sv.st.slots[k]) > slots_before:   # the slot this iteration added: zero start
                I = rx.mask(P.W[k], P.lo[k - 1], P.hi[k - 1], x[k - 1], z[k])
                lam_n, mu_n = rx.row_sums(P.W[k], P.lo[k - 1], P.hi[k - 1], I)
                gnew = x[k] - (P.W[k] * I) @ x[k - 1] + lam_n * (1 - z[k]) - z[k] * (P.b[k] + mu_n)
                zero = np.zeros_like(gnew)
                in_range(sb[s, slots_before, h], zero, zero, zero, gnew, 2 * ex[k], 1, own)
    return rows_checked, rows_total


@pytest.mark.parametrize("name,S,kw,it,nslots", CASES)
def test_bf16_one_iteration_within_rounding_bound(name, S, kw, it, nslots):
    prob = synth.problem(name, S=S, seed=0)
    dense = nw.dense_layers(prob["net"])   # conv operators built once for all subproblems
    Ps0 = nw.problems(prob, dense=dense)
    lh, uh = oracle_bounds_f32(Ps0)
    widths = Ps0[0].widths
    Ps = nw.problems(prob, bounds=[(split_hidden(lh[s].astype(np.float64), widths)[1:],
                                    split_hidden(uh[s].astype(np.float64), widths)[1:]) for s in range(S)],
                     dense=dense)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, precision=16, **kw), bounds=(lh, uh))
    solvers = draw_state(Ps, ctx, kw, it, nslots, seed=100 + it)
    opt = AS.Options(**{k: v for k, v in kw.items() if hasattr(AS.Options, k)})
    # the oracle's pre-step values and the step's schedule
    solvers = dict(enumerate(solvers))
    pre = pre_step(solvers)
    if it < opt.bigm_iters:
        lr, t = AS.linear_lr(opt.bigm_lr0, opt.bigm_lr1, it, opt.bigm_iters), -1
    else:
        t = it - opt.bigm_iters
        lr = AS.linear_lr(opt.as_lr0, opt.as_lr1, t, opt.as_iters)
    ctx.as_step(1)
    rows_checked, rows_total = check_bf16_step(ctx, solvers, pre, it, t, lr, opt)
    assert rows_checked >= 0.9 * rows_total, (rows_checked, rows_total)


@pytest.mark.parametrize("it,nslots", [(300, 4), (340, 4)])
def test_bf16_conv4_full_size_one_iteration_on_a_sampled_box(it, nslots):
    """The default bench workload at full size (conv4 net, 1024 boxes, BF16 form) in the bench's
    launch configuration: one iteration from a drawn state with 4 filled slots (omega 120:
    iteration 300 is ordinary, 340 adds slot 4), one sampled box against the oracle within the
    bf16 bound (its stride-1 conv products and every col-pass product take window operands)."""
    kw = dict(bigm_iters=100, as_iters=400, omega=120, max_cuts=5)
    sample = {613}
    ctx, Ps = conv4_full_batch(16, kw, sample)
    solvers = draw_state(Ps, ctx, kw, it, nslots, seed=700 + it, subset=sample)
    opt = AS.Options(**kw)
    pre = pre_step(solvers)
    t = it - opt.bigm_iters
    lr = AS.linear_lr(opt.as_lr0, opt.as_lr1, t, opt.as_iters)
    ctx.as_step(1)
    rows_checked, rows_total = check_bf16_step(ctx, solvers, pre, it, t, lr, opt)
    assert rows_checked >= 0.9 * rows_total, (rows_checked, rows_total)


FREE = [
    ("mlp_tiny", 1, dict(bigm_iters=20, as_iters=80, omega=24, max_cuts=5)),
    ("mlp_5_7_6_3", 4, dict(bigm_iters=30, as_iters=60, omega=20, max_cuts=4)),
    ("small_conv", 3, dict(bigm_iters=20, as_iters=40, omega=12, max_cuts=5)),
]


@pytest.mark.parametrize("name,S,kw", FREE)
def test_bf16_free_running_bound_is_valid_and_close_to_oracle(name, S, kw):
    prob = synth.problem(name, S=S, seed=0)
    Ps = nw.problems(prob)
    iters = kw["bigm_iters"] + kw["as_iters"]
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, precision=16, **kw))
    ctx.as_step(iters)
    b = ctx.bound()
    gaps = []
    for s, P in enumerate(Ps):
        ref = AS.ActiveSet(P, AS.Options(**kw)).step(iters).bound()
        assert b[s] <= sample_min_output(P, 5000) + 1e-6
        gaps.append(abs(b[s] - ref) / (1 + abs(ref)))
    print(f"BF16 form vs oracle, {name}: max gap {max(gaps):.2e} (per unit of 1 + |bound|)")
    assert max(gaps) <= GAP


def test_bf16_bound_below_the_exact_lp_of_the_tighter_relaxation():
    """On a net small enough for the exact rational LP over every constraint of problem (4)
    (4-3-3-1, six hidden neurons): the BF16 form's bound stays below the LP optimum."""
    prob = synth.problem("mlp_4_3_3_1", seed=4)
    P = nw.problems(prob)[0]
    kw = dict(bigm_iters=20, as_iters=80, omega=24, max_cuts=5)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, precision=16, **kw))
    ctx.as_step(100)
    lp_a = float(netlp_for(P).solve("A", P.W[P.n][0], P.b[P.n][0]))
    assert ctx.bound()[0] <= lp_a + 1e-6


def test_bf16_graph_replay_equals_plain_launches():
    """The captured graph (grouped GEMMs sizing their rows from the device counter) gives the
    same iterates as plain launches."""
    prob = synth.problem("small_conv", S=3, seed=1)
    kw = dict(bigm_iters=10, as_iters=40, omega=8, max_cuts=5, precision=16)
    a = binding.context_for(prob, binding.default_options(graph_chunk=0, **kw))
    g = binding.context_for(prob, binding.default_options(graph_chunk=10, **kw))
    a.as_step(50)
    g.as_step(50)
    np.testing.assert_array_equal(a.get_state(binding.ST_SLOT_BETA), g.get_state(binding.ST_SLOT_BETA))
    np.testing.assert_array_equal(a.bound(), g.bound())


def test_window_and_gathered_products_agree(monkeypatch):
    """The conv products by window operands (each CTA loads its rows' input window once; a kernel
    tap is a shift of the operand descriptor) and by gathered operands (environment CB_TC_WINDOWS =
    0) sum the same bf16 terms in another order: one iteration from the same drawn state on 8 boxes
    of the conv4 batch gives duals equal up to float32 summation order (a decision near a tie may
    flip: at least 99.9% of the entries agree)."""
    kw = dict(bigm_iters=100, as_iters=400, omega=120, max_cuts=5)
    prob = synth.problem("conv4", S=1024, seed=0, part=(0, 8))
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("CB_TC_WINDOWS", flag)
        ctx = binding.context_for(prob, binding.default_options(graph_chunk=25, precision=16, **kw))
        draw_state([None] * ctx.S, ctx, kw, 340, 4, seed=9, subset=set())
        ctx.as_step(1)
        out[flag] = [ctx.get_state(code).ravel() for code in
                     (binding.ST_ALPHA, binding.ST_BETA0, binding.ST_BETA1, binding.ST_SLOT_BETA, binding.ST_XSTAR)]
    for a, b in zip(out["1"], out["0"]):
        close = np.abs(a - b) <= 1e-5 * (1 + np.abs(b))
        assert close.mean() >= 0.999, close.mean()


def test_autotuned_products_keep_the_bound():
    """as_options.autotune in the BF16 form times each product's plans (window operands, gathered
    operands at N tiles of 32-256 columns) and keeps the fastest: the bound stays within the bf16
    gap of the oracle on the small conv net, and on 8 boxes of the conv4 batch it equals the untuned
    context's up to the summation order of the products."""
    prob = synth.problem("small_conv", S=3, seed=0)
    kw = dict(bigm_iters=20, as_iters=40, omega=12, max_cuts=5)
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=0, precision=16, autotune=1, **kw))
    ctx.as_step(60)
    b = ctx.bound()
    for s, P in enumerate(nw.problems(prob)):
        ref = AS.ActiveSet(P, AS.Options(**kw)).step(60).bound()
        assert abs(b[s] - ref) <= GAP * (1 + abs(ref))
    kw = dict(bigm_iters=20, as_iters=40, omega=12, max_cuts=5)
    prob = synth.problem("conv4", S=1024, seed=0, part=(0, 8))
    out = []
    for tune in (1, 0):
        ctx = binding.context_for(prob, binding.default_options(graph_chunk=25, precision=16, autotune=tune, **kw))
        ctx.as_step(60)
        out.append(ctx.bound())
    np.testing.assert_allclose(out[0], out[1], rtol=1e-3, atol=1e-3)

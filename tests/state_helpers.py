"""Matching dual states for the CUDA context and the oracle, drawn from the seeded generator.

A state is drawn once (duals, active-set snapshot bits, Adam moments) and written to both sides:
to the context through as_set_state, and to the oracle as a DualState whose masks the oracle
computes itself with eq. (3) at the snapshot points. Nothing flows from the CUDA path to the
oracle.
"""
import numpy as np

from oracle import active_set as AS
from oracle import dual as du
from oracle import relaxation as rx
from paper_2101_05844_gb300 import binding
from paper_2101_05844_gb300.synth import SplitMix64


def oracle_bounds_f32(Ps):
    """Interval bounds by the oracle (FP64), rounded outward to float32, as hidden vectors."""
    lh = np.stack([np.concatenate([np.asarray(P.lhat[k]) for k in range(1, P.n)]) for P in Ps])
    uh = np.stack([np.concatenate([np.asarray(P.uhat[k]) for k in range(1, P.n)]) for P in Ps])
    lo32 = lh.astype(np.float32)
    lo32 = np.where(lo32.astype(np.float64) > lh, np.nextafter(lo32, np.float32(-np.inf)), lo32)
    hi32 = uh.astype(np.float32)
    hi32 = np.where(hi32.astype(np.float64) < uh, np.nextafter(hi32, np.float32(np.inf)), hi32)
    return lo32.astype(np.float32), hi32.astype(np.float32)


def split_hidden(vec, widths):
    out, o = [None], 0
    for w in widths[1:]:
        out.append(vec[o:o + w])
        o += w
    return out


def draw_state(Ps, ctx, opt_kw, it, nslots, seed, scale=0.3, adam=True, subset=None, interior0=False):
    """Draw a state at global iteration `it` with `nslots` filled slots; install it on both sides.

    Returns the oracle ActiveSet solvers: a list over all subproblems, or a dict over `subset`
    (the oracle side is then built for those subproblems only). interior0: the inputs (layer 0)
    were strictly inside their box when each slot was added (an ellipsoid input set), so layer 1's
    masks are the oracle's eq. (3) at an interior point, whatever the drawn snapshot bits."""
    rng = SplitMix64(seed)
    S, NH, NT, cap = ctx.S, ctx.NH, ctx.NT, ctx.cap
    widths = ctx.widths

    def dual(n):
        v = rng.uniform(n) * scale
        v[rng.uniform(n) < 0.3] = 0.0
        return v.astype(np.float32)

    alpha, beta0, beta1 = dual(S * NH).reshape(S, NH), dual(S * NH).reshape(S, NH), dual(S * NH).reshape(S, NH)
    sb = np.zeros((S, cap, NH), np.float32)
    sb[:, :nslots] = dual(S * nslots * NH).reshape(S, nslots, NH)
    xs_bits = (rng.uniform(S * NT * 8) < 0.5).reshape(S, NT, 8)
    zs_bits = (rng.uniform(S * NH * 8) < 0.5).reshape(S, NH, 8)
    xs_bits[:, :, nslots:] = False
    zs_bits[:, :, nslots:] = False
    w8 = (1 << np.arange(8)).astype(np.uint8)
    xsnap = (xs_bits * w8).sum(-1).astype(np.uint8)
    zsnap = (zs_bits * w8).sum(-1).astype(np.uint8)
    m3 = (rng.uniform(6 * S * NH).reshape(6, S, NH) * 0.05).astype(np.float32) if adam else \
        np.zeros((6, S, NH), np.float32)
    m3[1::2] = m3[1::2] ** 2 + 1e-6 if adam else 0.0
    ms = np.zeros((2, S, cap, NH), np.float32)
    if adam:
        ms[0, :, :nslots] = (rng.uniform(S * nslots * NH).reshape(S, nslots, NH) * 0.05)
        ms[1, :, :nslots] = ms[0, :, :nslots] ** 2 + 1e-6
    ctx.set_state(binding.ST_ITER, np.array([it, 0, 0], np.int32))
    ctx.set_state(binding.ST_ALPHA, alpha)
    ctx.set_state(binding.ST_BETA0, beta0)
    ctx.set_state(binding.ST_BETA1, beta1)
    ctx.set_state(binding.ST_ADAM, m3)
    ctx.set_state(binding.ST_SLOT_ADAM, ms)
    ctx.set_state(binding.ST_XSNAP, xsnap)
    ctx.set_state(binding.ST_ZSNAP, zsnap)
    ctx.set_state(binding.ST_SLOT_BETA, sb)
    opt = AS.Options(**{k: v for k, v in opt_kw.items() if hasattr(AS.Options, k)})
    solvers = {} if subset is not None else []
    for s, P in enumerate(Ps):
        if subset is not None and s not in subset:
            continue
        st = du.DualState.zeros(P)
        st.alpha = [None] + split_hidden(alpha[s].astype(np.float64), widths)[1:]
        st.beta0 = [None] + split_hidden(beta0[s].astype(np.float64), widths)[1:]
        st.beta1 = [None] + split_hidden(beta1[s].astype(np.float64), widths)[1:]
        offs = np.cumsum([0] + widths)
        for b in range(nslots):
            added = opt.omega * (b // opt.vars_per_add) + (b % opt.vars_per_add) if opt.omega > 0 else b
            for k in range(1, P.n):
                xprev_bits = xs_bits[s, offs[k - 1]:offs[k], b]
                xprev = np.where(xprev_bits, P.hi[k - 1], P.lo[k - 1])
                if interior0 and k == 1:
                    xprev = 0.5 * (P.lo[0] + P.hi[0])
                zk = zs_bits[s, offs[k] - widths[0]:offs[k + 1] - widths[0], b].astype(np.float64)
                I = rx.mask(P.W[k], P.lo[k - 1], P.hi[k - 1], xprev, zk)
                hk = slice(offs[k] - widths[0], offs[k + 1] - widths[0])
                du.add_slot(P, st, k, I, added_at=added, beta=sb[s, b, hk].astype(np.float64))
                st.slots[k][-1].m = ms[0, s, b, hk].astype(np.float64)
                st.slots[k][-1].v = ms[1, s, b, hk].astype(np.float64)
        solver = AS.ActiveSet(P, opt, cap=None, state=st)
        solver.it = it
        for q, key in enumerate(["a", "0", "1"]):
            solver.m[key] = [None] + [v.astype(np.float64) for v in split_hidden(m3[2 * q, s], widths)[1:]]
            solver.v[key] = [None] + [v.astype(np.float64) for v in split_hidden(m3[2 * q + 1, s], widths)[1:]]
        if subset is not None:
            solvers[s] = solver
        else:
            solvers.append(solver)
    return solvers


def hidden_concat(lists):
    return np.concatenate([np.asarray(v) for v in lists[1:]])


def conv4_full_batch(precision, opt_kw, sample):
    """The conv4 workload at full size (1024 boxes) in the bench's launch configuration (CUDA
    graphs of 25 iterations), and the oracle's problems for the sampled boxes only, over the
    context's own interval bounds (the oracle's dense conv operators are large; interval bounds
    have tests of their own). Returns (ctx, Ps): Ps a list over all boxes, None where not sampled."""
    from oracle import network as nw
    from paper_2101_05844_gb300 import synth
    prob = synth.problem("conv4", seed=0)
    S = prob["lo"].shape[0]
    ctx = binding.context_for(prob, binding.default_options(graph_chunk=25, precision=precision, **opt_kw))
    lh = ctx.get_state(binding.ST_LHAT).reshape(S, -1).astype(np.float64)
    uh = ctx.get_state(binding.ST_UHAT).reshape(S, -1).astype(np.float64)
    dense = nw.dense_layers(prob["net"])
    Ps = [None] * S
    for s in sample:
        one = dict(prob, lo=prob["lo"][s:s + 1], hi=prob["hi"][s:s + 1], C=prob["C"][s:s + 1])
        bd = (split_hidden(lh[s], ctx.widths)[1:], split_hidden(uh[s], ctx.widths)[1:])
        Ps[s] = nw.problems(one, bounds=[bd], dense=dense)[0]
    return ctx, Ps

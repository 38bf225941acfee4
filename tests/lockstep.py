"""One-iteration comparison of the CUDA Active Set step with the oracle's, with tolerances derived
from float32 arithmetic instead of blanket exemptions.

The GPU sums in float32; the oracle in float64. A supergradient entry of hidden neuron i of layer k
is a sum of terms whose magnitudes add up to at most
    T_i = (|W_k| |x_{k-1}|)_i + (|W_k| max(|l_{k-1}|, |u_{k-1}|))_i + |b_i| + |x_i| + |lhat_i| + |uhat_i|
(the products of W x*, of the masked products and of the slots' lambda, kappa, and the vector terms
of eq. 9), so its float32 value is within
    delta_i = 2^-24 (2 sqrt(n) + 8) T_i,     n the layer's fan-in,
of the exact one (recursive and tree summation, the square root for rounding errors of random
sign). Every updated dual is then checked against the oracle's projected Adam step within the
rounding tolerance (1e-5 relative, 1e-7 absolute) plus the spread of the oracle's own step over
gradients in [g - delta, g + delta]: where the step is insensitive (the usual case) that spread is
zero, and where it is not (a gradient next to zero and no moment to damp it) the spread is the
step's own range; an exactly zero gradient is a structural zero (say x* = 0 and z* = 0), which
float32 evaluates exactly too. The primal minimiser x*, z* (eqs. 7-8) is compared exactly wherever its deciding
sum f (resp. g) clears the same kind of bound; rows that read an undecided x* or z* are reported
and left out, and the fraction left out must stay small.
"""
import numpy as np

from oracle import active_set as AS
from oracle import dual as du
from oracle import relaxation as rx

U32 = 2.0 ** -24


def _hc(lists):
    return np.concatenate([np.asarray(v, np.float64) for v in lists[1:]])


def _adam_spread(theta, m, v, g, delta, lr, step, opt):
    # a gradient that is exactly zero is a structural zero (x* = 0 with z* = 0, say), which float32
    # evaluates exactly as well
    delta = np.where(g == 0, 0.0, delta)
    out = []
    for gg in (g - delta, g, g + delta):
        th, mm, vv = theta.copy(), m.copy(), v.copy()
        AS.adam(th, mm, vv, gg, lr, step, opt)
        out.append(th)
    return np.max(out, axis=0) - np.min(out, axis=0)


def _sum_bound(n, T):
    return U32 * (2.0 * np.sqrt(n) + 8.0) * T


def check_active_set_step(sv, gpu, rtol=1e-5, atol=1e-7, min_tight=0.9, max_exempt=0.1):
    """Steps the oracle solver sv once and compares it with the GPU's state after its step.

    gpu: dict with float32 arrays alpha, beta0, beta1 (hidden vectors), slots [cap][NH] and xstar
    [NT] of one subproblem. Returns a dict of counts (checked entries, exempt rows)."""
    P, opt, it = sv.P, sv.opt, sv.it
    n = P.n
    _, f, g, x, z = du.evaluate(P, sv.st)
    grads = du.supergradient(P, sv.st, x, z)
    if it < opt.bigm_iters:
        lr, t = AS.linear_lr(opt.bigm_lr0, opt.bigm_lr1, it, opt.bigm_iters), -1
    else:
        t = it - opt.bigm_iters
        lr = AS.linear_lr(opt.as_lr0, opt.as_lr1, t, opt.as_iters)
    new_b = AS.addition_slot(t, opt, sv.cap) if t >= 0 else -1
    nold = len(sv.st.slots[1])
    # the gradient of the slot this iteration adds: eq. (9) at the oracle's mask at (x*, z*)
    gnew = [None]
    if new_b >= 0:
        for k in range(1, n):
            I = rx.mask(P.W[k], P.lo[k - 1], P.hi[k - 1], x[k - 1], z[k])
            lam, mu = rx.row_sums(P.W[k], P.lo[k - 1], P.hi[k - 1], I)
            gnew.append(x[k] - (P.W[k] * I) @ x[k - 1] + lam * (1 - z[k]) - z[k] * (P.b[k] + mu))
    # bounds on the float32 error of every sum the step decides on
    delta, affected = [None], [None]
    und_f = []
    for m in range(n):
        Tf = np.zeros(P.widths[m])
        if m >= 1:
            Tf += np.abs(sv.st.alpha[m]) + np.abs(sv.st.beta0[m]) + np.abs(sv.st.beta1[m])
            for sl in sv.st.slots[m]:
                Tf += np.abs(sl.beta)
        if m + 1 <= n - 1:
            up = np.abs(sv.st.alpha[m + 1]) + np.abs(sv.st.beta1[m + 1])
            for sl in sv.st.slots[m + 1]:
                up = up + np.abs(sl.beta)
            Tf += np.abs(P.W[m + 1]).T @ up
        else:
            Tf += np.abs(P.W[n][0])
        fan = P.W[m + 1].shape[0]
        und_f.append(np.abs(f[m]) <= _sum_bound(fan, Tf))
    for k in range(1, n):
        fan = P.W[k].shape[1]
        mag = np.maximum(np.abs(P.lo[k - 1]), np.abs(P.hi[k - 1]))
        T = (np.abs(P.W[k]) @ np.abs(x[k - 1]) + np.abs(P.W[k]) @ mag + np.abs(P.b[k]) + np.abs(x[k])
             + np.abs(P.lhat[k]) + np.abs(P.uhat[k]))
        delta.append(_sum_bound(fan, T))
        Tg = np.abs(sv.st.beta0[k] * P.uhat[k]) + np.abs(sv.st.beta1[k] * P.lhat[k])
        for sl in sv.st.slots[k]:
            Tg = Tg + np.abs(sl.beta) * (np.abs(sl.lam) + np.abs(sl.mu) + np.abs(P.b[k]))
        und_g = (g[k] != 0) & (np.abs(g[k]) <= _sum_bound(fan, Tg))
        affected.append(und_g | und_f[k] | ((np.abs(P.W[k]) @ und_f[k - 1].astype(float)) > 0))
    # the pre-step state, then the oracle's step
    pre = {key: [None] + [np.array(a[k]) for k in range(1, n)]
           for key, a in (("alpha", sv.st.alpha), ("beta0", sv.st.beta0), ("beta1", sv.st.beta1))}
    mom = {key: ([None] + [sv.m[c][k].copy() for k in range(1, n)], [None] + [sv.v[c][k].copy() for k in range(1, n)])
           for key, c in (("alpha", "a"), ("beta0", "0"), ("beta1", "1"))}
    spre = [[(sl.beta.copy(), sl.m.copy(), sl.v.copy(), sl.added_at) for sl in sv.st.slots[k]] for k in range(n)]
    sv.step(1)
    offs = np.cumsum([0] + P.widths)
    und_x = np.concatenate(und_f)
    xg = np.asarray(gpu["xstar"], np.float32)
    np.testing.assert_array_equal(xg[~und_x], np.concatenate(x).astype(np.float32)[~und_x])
    skip = np.concatenate(affected[1:]).astype(bool)
    assert skip.mean() <= max_exempt, f"{skip.mean():.3f} of the rows read an undecided x* or z*"
    dl = _hc(delta)
    checked, tight = 0, 0

    def compare(got, ref, spread):
        nonlocal checked, tight
        ok = ~skip
        allowed = rtol * np.abs(ref) + atol + spread
        bad = ok & (np.abs(got - ref) > allowed)
        assert not bad.any(), (f"{bad.sum()} entries off: gpu {got[bad][:4]}, oracle {ref[bad][:4]}, "
                               f"spread {spread[bad][:4]}")
        assert (got >= 0).all()
        checked += int(ok.sum())
        tight += int((ok & (spread <= rtol * np.abs(ref) + atol)).sum())

    gk = {"alpha": grads["galpha"], "beta0": grads["gbeta0"], "beta1": grads["gbeta1"]}
    for key, ref in (("alpha", sv.st.alpha), ("beta0", sv.st.beta0), ("beta1", sv.st.beta1)):
        spread = _adam_spread(_hc(pre[key]), _hc(mom[key][0]), _hc(mom[key][1]), _hc(gk[key]), dl, lr, it + 1, opt)
        compare(np.asarray(gpu[key], np.float64), _hc(ref), spread)
    for b in range(len(sv.st.slots[1])):
        ref = _hc([None] + [sv.st.slots[k][b].beta for k in range(1, n)])
        if b < nold:
            th0 = _hc([None] + [spre[k][b][0] for k in range(1, n)])
            m0 = _hc([None] + [spre[k][b][1] for k in range(1, n)])
            v0 = _hc([None] + [spre[k][b][2] for k in range(1, n)])
            gref = _hc([None] + [grads["gslots"][k][b] for k in range(1, n)])
            step = t - spre[1][b][3] + 1
        else:
            th0 = m0 = v0 = np.zeros_like(ref)
            gref = _hc(gnew)
            step = 1
        spread = _adam_spread(th0, m0, v0, gref, dl, lr, step, opt)
        compare(np.asarray(gpu["slots"][b], np.float64), ref, spread)
    assert checked > 0 and tight >= min_tight * checked, f"{tight} of {checked} entries at the rounding tolerance"
    return {"checked": checked, "tight": tight, "exempt_rows": int(skip.sum()), "rows": int(skip.size),
            "undecided_x": int(und_x.sum())}

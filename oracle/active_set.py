"""Big-M solver (Alg. 3, App. B) and Active Set (Alg. 1, Sec. 4) (oracle; test infrastructure only).

Iteration it = 0 .. T_M - 1 is a Big-M iteration (B empty), it = T_M .. T_M + T_A - 1 is Active Set
iteration t = it - T_M. Each iteration: closed-form inner minimisation (eqs. 7-8); on addition
iterations, the oracle eq. (3) at (x*, z*) for every hidden layer appended to B_k (Alg. 1); the
supergradient (eq. 9); an Adam ascent step (Kingma and Ba, as Sec. 8.1 states) and clipping at zero.

Schedule readings (the paper fixes the pattern, not every constant; Sec. 8.1):
  * step sizes fall linearly, lr_t = lr_0 + (lr_1 - lr_0) t / max(1, T - 1): Big-M 1e-2 -> 1e-4,
    then reset for Active Set, 1e-3 -> 1e-6;
  * masks are added at Active Set iterations t with t mod omega < vars_per_add (2 in the paper:
    "every addition consists of 2 new variables", one per iteration as Alg. 1 calls the oracle once
    per iteration), slot index b = (t div omega) * vars_per_add + (t mod omega), while b < cap;
  * Adam uses beta1 = 0.9, beta2 = 0.999, eps = 1e-8 with bias correction (Kingma and Ba's
    defaults; the paper names Adam only). alpha, beta_0, beta_1 keep their moments and step count
    across the Big-M -> Active Set switch; a new beta_{k,I} starts at zero with zero moments and
    its own step count, and takes its first step in the iteration that adds it;
  * the best bound over all evaluated iterates is kept beside the final one.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import dual as du
from . import relaxation as rx


@dataclass
class Options:
    bigm_iters: int = 0
    as_iters: int = 0
    bigm_lr0: float = 1e-2
    bigm_lr1: float = 1e-4
    as_lr0: float = 1e-3
    as_lr1: float = 1e-6
    omega: int = 450
    vars_per_add: int = 2
    max_cuts: int = 7
    adam_b1: float = 0.9
    adam_b2: float = 0.999
    adam_eps: float = 1e-8
    # Saddle Point (Alg. 2, App. C)
    sp_gamma0: float = 10.0
    sp_c_alpha: float = 1e-3
    sp_c_beta: float = 1e-3
    sp_init_steps: int = 100
    sp_init_lr0: float = 1e-2
    sp_init_lr1: float = 1e-5


def linear_lr(a: float, b: float, t: int, T: int) -> float:
    return a + (b - a) * t / max(1, T - 1)


def addition_slot(t: int, opt: Options, cap: int) -> int:
    """Slot index added at Active Set iteration t, or -1."""
    if opt.omega > 0:
        q, r = divmod(t, opt.omega)
    else:
        q, r = (0, t) if t < opt.vars_per_add else (1, opt.vars_per_add)
    if r >= opt.vars_per_add:
        return -1
    b = q * opt.vars_per_add + r
    return b if b < cap else -1


def adam(theta, m, v, g, lr, step, opt: Options):
    m[:] = opt.adam_b1 * m + (1 - opt.adam_b1) * g
    v[:] = opt.adam_b2 * v + (1 - opt.adam_b2) * g * g
    mh = m / (1 - opt.adam_b1 ** step)
    vh = v / (1 - opt.adam_b2 ** step)
    theta[:] = np.maximum(theta + lr * mh / (np.sqrt(vh) + opt.adam_eps), 0.0)


class ActiveSet:
    """Stateful Big-M + Active Set solver for one subproblem."""

    def __init__(self, P, opt: Options, cap: int | None = None, state: du.DualState | None = None):
        self.P = P
        self.opt = opt
        self.cap = opt.max_cuts if cap is None else cap
        self.st = state if state is not None else du.DualState.zeros(P)
        z = lambda: [None] + [np.zeros(P.widths[k]) for k in range(1, P.n)]
        self.m = {"a": z(), "0": z(), "1": z()}
        self.v = {"a": z(), "0": z(), "1": z()}
        self.it = 0
        self.best = -np.inf
        self.trace = []

    def step(self, n_iters: int):
        P, opt, st = self.P, self.opt, self.st
        for _ in range(n_iters):
            it = self.it
            if it < opt.bigm_iters:
                lr = linear_lr(opt.bigm_lr0, opt.bigm_lr1, it, opt.bigm_iters)
                t = -1
            else:
                t = it - opt.bigm_iters
                lr = linear_lr(opt.as_lr0, opt.as_lr1, t, opt.as_iters)
            val, f, g, x, z = du.evaluate(P, st)
            self.best = max(self.best, val)
            self.trace.append(val)
            if t >= 0:
                b = addition_slot(t, opt, self.cap)
                if b >= 0:
                    for k in range(1, P.n):
                        I = rx.mask(P.W[k], P.lo[k - 1], P.hi[k - 1], x[k - 1], z[k])
                        du.add_slot(P, st, k, I, added_at=t)
            gr = du.supergradient(P, st, x, z)
            step = it + 1
            for k in range(1, P.n):
                adam(st.alpha[k], self.m["a"][k], self.v["a"][k], gr["galpha"][k], lr, step, opt)
                adam(st.beta0[k], self.m["0"][k], self.v["0"][k], gr["gbeta0"][k], lr, step, opt)
                adam(st.beta1[k], self.m["1"][k], self.v["1"][k], gr["gbeta1"][k], lr, step, opt)
                for sl, gs in zip(st.slots[k], gr["gslots"][k]):
                    adam(sl.beta, sl.m, sl.v, gs, lr, t - sl.added_at + 1, opt)
            self.it += 1
        return self

    def bound(self) -> float:
        val = du.evaluate(self.P, self.st)[0]
        self.best = max(self.best, val)
        return val


def solve(P, opt: Options, cap: int | None = None):
    """Run T_M + T_A iterations; return (final bound, best bound, solver)."""
    s = ActiveSet(P, opt, cap).step(opt.bigm_iters + opt.as_iters)
    final = s.bound()
    return final, s.best, s

"""Branch and bound with stratified bounding (Sec. 6.2) (oracle; test infrastructure only).

Sec. 6.2: branch and bound splits the problem domain into subproblems and bounds the minimum of
the property over each; a subproblem whose lower bound is positive cannot hold a counterexample
and is pruned (the canonical form of Bunel et al.: the property holds when min > 0); the network
evaluated at the input point x_0* of the bounding solver's final iterate gives an upper bound
(footnote of Sec. 6.2, for Active Set). Two bounding algorithms are stratified: a_l (inexpensive
and loose) and a_t (tighter and costly). At the root, l_{a_t-a_l} = l_{a_t}(r) - l_{a_l}(r); an
exponential moving average i(s) tracks the parent-to-child increase of the lower bound; for a
child s of p the enumeration subtrees each algorithm would grow are estimated as
    |s|_{a_l} = 2^(-l_{a_l}(p) / i(s) + 1) - 1,   |s|_{a_t} = 2^(-(l_{a_l}(p) + l_{a_t-a_l}) / i(s) + 1) - 1,
and s and its whole subtree are bounded by a_t once |s|_{a_l} / |s|_{a_t} > c_{a_t/a_l}.

Readings where Sec. 6.2 and Sec. 8.2 leave the procedure open:
  * domains are (input box, ReLU splits); a branch splits one unsplit ambiguous neuron into its
    passing (+1) and blocking (-1) phase, the +1 child first. BaBSR's branching score (built on
    the Wong and Kolter bounds) is out of scope: the neuron taken is the ambiguous one with the
    largest -lhat * uhat / (uhat - lhat), the largest gap between the ReLU and the upper line of
    its triangle relaxation, the lowest index on ties;
  * each batch takes the B/2 unpruned domains with the lowest lower bounds (creation order on
    ties) and bounds their B children together; a child's lower bound is the larger of its own
    and its parent's (the child's domain lies inside the parent's);
  * intermediate bounds of a domain: interval propagation with the domain's split clamps,
    intersected with the root's intermediate bounds (App. E, computed once) when those are given;
  * the moving average starts at the first parent-to-child increase, i <- (1 - w) i + w d over
    the children of a batch in order, counting only children bounded by their parent's algorithm
    (a switch of algorithm is not a tightening by splitting); before its first sample, and the
    root's children, use a_l; with i <= 0 a child is hard when l_{a_t-a_l} > 0; a non-positive
    |s|_{a_t} (a_t would prune s at once) marks s hard when |s|_{a_l} > 0;
  * a domain with no ambiguous unsplit neuron left and a non-positive lower bound cannot be split
    (its relaxation is exact: its dual solve has not converged yet); it is bounded again from its
    own final duals, as a single child with the same splits, up to leaf_rebounds times, and then
    set aside, which makes the result "unknown" unless a counterexample turns up; these re-solves
    do not enter the moving average (they tighten by iterations, not by splitting);
  * the search stops with "falsified" as soon as an evaluated point has a negative property value,
    with "verified" when no domain is left, and with "unknown" when max_domains bounds are done;
  * warm start (Sec. 8.2 starts each child's duals from its parent's solve): a child's
    solve starts from its parent's final alpha, beta_0, beta_1, with zero Adam moments, an empty
    active set and its algorithm's full schedule (its Big-M phase, then Active Set); the root
    starts from zero duals.
"""
from __future__ import annotations

import heapq
import math
from dataclasses import dataclass, field

import numpy as np

from . import active_set as AS
from . import dual as du
from . import network as nw

VERIFIED, FALSIFIED, UNKNOWN = "verified", "falsified", "unknown"


@dataclass
class BabOptions:
    loose: AS.Options
    tight: AS.Options
    stratify: bool = True
    cost_ratio: float = 4.0     # c_{a_t/a_l}
    ema_weight: float = 0.3     # w
    batch: int = 8              # children bounded per batch (even)
    max_domains: int = 400
    warm_start: bool = True
    leaf_rebounds: int = 8


@dataclass
class Domain:
    splits: np.ndarray
    lb: float
    v: float                    # the raw bound of its own solve
    hard: bool
    branch: int
    seq: int
    alg: str = field(default="l")
    duals: tuple = None          # (alpha, beta0, beta1) of its own solve, 1-based lists
    rebounds: int = 0
    again: bool = False          # a re-solve of its parent's domain


def subtree_ratio(lp: float, delta: float, i: float) -> float:
    """|s|_{a_l} / |s|_{a_t} of Sec. 6.2 (inf when a_t would prune s at once)."""
    a = -lp / i + 1.0
    b = -(lp + delta) / i + 1.0
    if a > 60.0 and b > 60.0:
        return 2.0 ** (a - b)
    sl, st = 2.0 ** a - 1.0, 2.0 ** b - 1.0
    if st <= 0.0:
        return math.inf if sl > 0.0 else 0.0
    return sl / st


def is_hard(lp: float, delta: float, i, c: float) -> bool:
    if i is None:
        return False
    if i <= 0.0:
        return delta > 0.0
    return subtree_ratio(lp, delta, i) > c


def branch_neuron(lhat, uhat, splits) -> int:
    """The ambiguous unsplit neuron with the largest -l u / (u - l), or -1."""
    l, u = np.concatenate(lhat[1:]), np.concatenate(uhat[1:])
    amb = (l < 0) & (u > 0) & (splits == 0)
    if not amb.any():
        return -1
    score = np.where(amb, -l * u / np.where(amb, u - l, 1.0), -np.inf)
    return int(np.argmax(score))


def forward(dense, x):
    h = np.asarray(x, np.float64)
    for W, b, _ in dense[:-1]:
        h = np.maximum(W @ h + b, 0.0)
    W, b, _ = dense[-1]
    return W @ h + b


class BaB:
    def __init__(self, net, lo0, hi0, crow, opt: BabOptions, root_bounds=None, ball=False):
        self.net, self.opt = net, opt
        self.lo0, self.hi0 = np.asarray(lo0, np.float64), np.asarray(hi0, np.float64)
        self.crow = np.asarray(crow, np.float64)
        self.dense = nw.dense_layers(net)
        self.Ws = [d[0] for d in self.dense[:-1]]
        self.bs = [d[1] for d in self.dense[:-1]]
        self.NH = sum(W.shape[0] for W in self.Ws)
        self.root_bounds = root_bounds
        self.ball = ball   # the input set is the ellipsoid inscribed in the box
        self.ub, self.x_ub = math.inf, None
        self.bounded = 0
        self.seq = 0
        self.ema = None
        self.hard_bounded = 0

    def _bounds(self, splits):
        lh, uh, _, _ = nw.ibp(self.Ws, self.bs, self.lo0, self.hi0, splits, self.ball)
        lh, uh = [None] + list(lh[1:]), [None] + list(uh[1:])
        if self.root_bounds is not None:
            rl, ru = self.root_bounds
            lh = [None] + [np.maximum(a, b) for a, b in zip(lh[1:], rl[1:])]
            uh = [None] + [np.minimum(a, b) for a, b in zip(uh[1:], ru[1:])]
        return lh, uh

    def _solve(self, splits, alg, warm=None):
        lh, uh = self._bounds(splits)
        P = nw.Problem(self.net, self.lo0, self.hi0, self.crow, bounds=(lh[1:], uh[1:]), dense=self.dense,
                       ball=self.ball)
        opt = self.opt.loose if alg == "l" else self.opt.tight
        st = None
        if warm is not None and self.opt.warm_start:
            cp = lambda v: [None] + [a.copy() for a in v[1:]]
            st = du.DualState(cp(warm[0]), cp(warm[1]), cp(warm[2]), [[] for _ in range(P.n)])
        s = AS.ActiveSet(P, opt, state=st).step(opt.bigm_iters + opt.as_iters)
        final = s.bound()
        cp = lambda v: [None] + [a.copy() for a in v[1:]]
        self._last_duals = (cp(s.st.alpha), cp(s.st.beta0), cp(s.st.beta1))
        x0 = du.evaluate(P, s.st)[3][0]
        val = float(self.crow @ forward(self.dense, x0))
        if val < self.ub:
            self.ub, self.x_ub = val, np.array(x0)
        self.bounded += 1
        if alg == "t":
            self.hard_bounded += 1
        return final, branch_neuron(lh, uh, splits)

    def run(self):
        o = self.opt
        root = np.zeros(self.NH, np.int8)
        vt, br = self._solve(root, "t")
        duals = self._last_duals
        if o.stratify:
            vl, _ = self._solve(root, "l")
            duals = self._last_duals
            self.delta = vt - vl
        else:
            vl, self.delta = vt, 0.0
        r = Domain(root, max(vl, vt), vl, False, br, 0, "l" if o.stratify else "t", duals)
        self.seq = 1
        self.lower_pruned = math.inf
        pool, leaves = [], []
        if r.lb > 0:
            self.lower_pruned = r.lb
        else:
            heapq.heappush(pool, (r.lb, r.seq, r))
        while True:
            if self.ub < 0:
                return self._result(FALSIFIED, pool, leaves)
            if not pool:
                return self._result(UNKNOWN if leaves else VERIFIED, pool, leaves)
            if self.bounded >= o.max_domains:
                return self._result(UNKNOWN, pool, leaves)
            parents = []
            while pool and len(parents) < o.batch // 2:
                parents.append(heapq.heappop(pool)[2])
            kids = []
            for p in parents:
                if p.branch < 0:
                    if p.rebounds < o.leaf_rebounds:
                        kids.append((p, Domain(p.splits.copy(), 0.0, 0.0, p.hard, -1, self.seq, p.alg,
                                               rebounds=p.rebounds + 1, again=True)))
                        self.seq += 1
                    else:
                        leaves.append(p)
                    continue
                for sgn in (1, -1):
                    sp = p.splits.copy()
                    sp[p.branch] = sgn
                    if not o.stratify:
                        hard = True
                    else:
                        hard = p.hard or is_hard(p.v, self.delta, self.ema, o.cost_ratio)
                    kids.append((p, Domain(sp, 0.0, 0.0, hard, -1, self.seq, "t" if hard else "l")))
                    self.seq += 1
            for alg in ("l", "t"):   # the easy batch, then the hard one
                for p, c in kids:
                    if c.alg == alg:
                        c.v, c.branch = self._solve(c.splits, alg, p.duals)
                        c.duals = self._last_duals
                        c.lb = max(c.v, p.lb)
            for p, c in kids:
                if c.alg == p.alg and not c.again:
                    d = c.v - p.v
                    self.ema = d if self.ema is None else (1 - o.ema_weight) * self.ema + o.ema_weight * d
                if c.lb > 0:
                    self.lower_pruned = min(self.lower_pruned, c.lb)
                else:
                    heapq.heappush(pool, (c.lb, c.seq, c))

    def _result(self, status, pool, leaves):
        front = [d.lb for _, _, d in pool] + [d.lb for d in leaves]
        lower = min(front) if front else self.lower_pruned
        return {"status": status, "lower": lower, "upper": self.ub, "x": self.x_ub,
                "bounded": self.bounded, "hard_bounded": self.hard_bounded}

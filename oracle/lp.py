"""Exact linear programs for tiny networks (oracle; test infrastructure only).

An exact two-phase simplex over Python Fractions (Bland's rule, so it terminates), and builders for
the LP relaxations the paper compares:
  "M"       problem (2): the Big-M / Planet relaxation M_k (Sec. 2.1);
  "A"       problem (4): M_k plus every exponential-family constraint I in E_k (Sec. 2.2);
  "Aprime"  the original set A'_k of Anderson et al., eq. (17) in App. F: x >= xhat, the box on
            xhat, and the exponential-family constraint for every I in 2^{W_k}, 0 and 1 included.
Variables are x_0, then (x_k, z_k) for each hidden layer; xhat_k = W_k x_{k-1} + b_k is substituted.
Every constraint is kept as (coefficient dict, right-hand side) meaning a . v <= rhs, labelled
with the dual variable the paper attaches to it (App. D), so the same rows also give the
constraint-form Lagrangian.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product

import numpy as np


def _F(v) -> Fraction:
    return v if isinstance(v, Fraction) else Fraction(float(v))


def simplex_min(c, rows, rhs, lb, ub):
    """min c.v  s.t.  rows[i] . v <= rhs[i],  lb <= v <= ub  (exact). Returns (value, v) or
    (None, None) when infeasible. Unbounded problems cannot arise: every variable is boxed."""
    n = len(c)
    A = [list(map(_F, r)) for r in rows]
    r = [_F(v) - sum(a * _F(l) for a, l in zip(rw, lb)) for rw, v in zip(A, rhs)]
    for j in range(n):  # y_j = v_j - lb_j <= ub_j - lb_j
        e = [Fraction(0)] * n
        e[j] = Fraction(1)
        A.append(e)
        r.append(_F(ub[j]) - _F(lb[j]))
    m = len(A)
    ncol = n + m
    T, basis, arts = [], [], []
    for i in range(m):
        sgn = 1 if r[i] >= 0 else -1
        row = [sgn * a for a in A[i]] + [Fraction(0)] * m
        row[n + i] = Fraction(sgn)
        T.append(row)
        if sgn > 0:
            basis.append(n + i)
        else:
            arts.append(i)
            basis.append(None)
    # artificial columns
    na = len(arts)
    for i, row in enumerate(T):
        row.extend([Fraction(0)] * na)
    for a_idx, i in enumerate(arts):
        T[i][ncol + a_idx] = Fraction(1)
        basis[i] = ncol + a_idx
    b = [abs(v) for v in r]
    total = ncol + na

    def run(cost):
        while True:
            # reduced costs
            cb = [cost[basis[i]] for i in range(m)]
            enter = None
            for j in range(total):
                if j in basis_set:
                    continue
                rc = cost[j] - sum(cb[i] * T[i][j] for i in range(m) if T[i][j] != 0)
                if rc < 0:
                    enter = j
                    break
            if enter is None:
                return
            best, leave = None, None
            for i in range(m):
                a = T[i][enter]
                if a > 0:
                    ratio = b[i] / a
                    if best is None or ratio < best or (ratio == best and basis[i] < basis[leave]):
                        best, leave = ratio, i
            if leave is None:
                raise RuntimeError("unbounded LP")
            piv = T[leave][enter]
            T[leave] = [v / piv for v in T[leave]]
            b[leave] /= piv
            for i in range(m):
                if i != leave and T[i][enter] != 0:
                    f = T[i][enter]
                    T[i] = [vi - f * vl for vi, vl in zip(T[i], T[leave])]
                    b[i] -= f * b[leave]
            basis_set.discard(basis[leave])
            basis[leave] = enter
            basis_set.add(enter)

    basis_set = set(basis)
    if na:
        cost1 = [Fraction(0)] * ncol + [Fraction(1)] * na
        run(cost1)
        if sum(b[i] for i in range(m) if basis[i] >= ncol) > 0:
            return None, None
        # drive remaining artificials out of the basis where possible
        for i in range(m):
            if basis[i] >= ncol:
                for j in range(ncol):
                    if T[i][j] != 0 and j not in basis_set:
                        piv = T[i][j]
                        T[i] = [v / piv for v in T[i]]
                        b[i] /= piv
                        for i2 in range(m):
                            if i2 != i and T[i2][j] != 0:
                                f = T[i2][j]
                                T[i2] = [v2 - f * v1 for v2, v1 in zip(T[i2], T[i])]
                                b[i2] -= f * b[i]
                        basis_set.discard(basis[i])
                        basis[i] = j
                        basis_set.add(j)
                        break
    cost2 = [_F(v) for v in c] + [Fraction(0)] * m + [Fraction(10 ** 30)] * na
    run(cost2)
    y = [Fraction(0)] * total
    for i in range(m):
        y[basis[i]] = b[i]
    v = [y[j] + _F(lb[j]) for j in range(n)]
    return sum(_F(cj) * vj for cj, vj in zip(c, v)), v


class NetLP:
    """Constraint rows of the LP relaxations of a small network with given bounds.

    Ws, bs: hidden layers' dense (W_k, b_k), k = 1..L; lhat/uhat/lo/hi: 1-based bound lists as in
    oracle.network (lo[0], hi[0] the input box).
    """

    def __init__(self, Ws, bs, lhat, uhat, lo, hi):
        self.Ws, self.bs = Ws, bs
        self.lhat, self.uhat, self.lo, self.hi = lhat, uhat, lo, hi
        self.L = len(Ws)
        widths = [len(lo[0])] + [W.shape[0] for W in Ws]
        self.widths = widths
        self.xoff, self.zoff = [0], [None]
        off = widths[0]
        for k in range(1, self.L + 1):
            self.xoff.append(off)
            off += widths[k]
            self.zoff.append(off)
            off += widths[k]
        self.nvar = off
        lb = [Fraction(0)] * off
        ub = [Fraction(0)] * off
        for j in range(widths[0]):
            lb[j], ub[j] = _F(lo[0][j]), _F(hi[0][j])
        for k in range(1, self.L + 1):
            for i in range(widths[k]):
                lb[self.xoff[k] + i], ub[self.xoff[k] + i] = _F(lo[k][i]), _F(hi[k][i])
                lb[self.zoff[k] + i], ub[self.zoff[k] + i] = Fraction(0), Fraction(1)
        self.lb, self.ub = lb, ub

    def _xhat(self, k, i):
        """(coefficient dict, constant) of xhat_k[i] = W_k[i] x_{k-1} + b_k[i]."""
        W, b = self.Ws[k - 1], self.bs[k - 1]
        d = {self.xoff[k - 1] + j: _F(W[i, j]) for j in range(W.shape[1]) if W[i, j] != 0}
        return d, _F(b[i])

    def mask_row(self, k, i, I):
        """Exponential-family constraint of neuron i, mask row I (eq. 4), as (dict, rhs)."""
        W = self.Ws[k - 1]
        l, u = self.lo[k - 1], self.hi[k - 1]
        lam, mu = Fraction(0), Fraction(0)
        d = {self.xoff[k] + i: Fraction(1)}
        for j in range(W.shape[1]):
            w = _F(W[i, j])
            Lc, Uc = (_F(l[j]), _F(u[j])) if w >= 0 else (_F(u[j]), _F(l[j]))
            if I[j]:
                lam += w * Lc
                if w != 0:
                    d[self.xoff[k - 1] + j] = d.get(self.xoff[k - 1] + j, Fraction(0)) - w
            else:
                mu += w * Uc
        d[self.zoff[k] + i] = -(_F(self.bs[k - 1][i]) + lam + mu)
        return d, -lam

    def rows(self, kind: str, masks=None):
        """[(label, dict, rhs)] for relaxation kind "M", "A", "Aprime", or "M+" with explicit
        masks = {(k, i): [mask rows]} added to M (an active set)."""
        out = []
        for k in range(1, self.L + 1):
            fan_in = self.widths[k - 1]
            for i in range(self.widths[k]):
                xh, c = self._xhat(k, i)
                xi, zi = self.xoff[k] + i, self.zoff[k] + i
                # alpha: xhat - x <= 0
                d = dict(xh)
                d[xi] = d.get(xi, Fraction(0)) - 1
                out.append((("alpha", k, i), d, -c))
                if kind in ("M", "A", "M+"):
                    uh, lh = _F(self.uhat[k][i]), _F(self.lhat[k][i])
                    out.append((("beta0", k, i), {xi: Fraction(1), zi: -uh}, Fraction(0)))
                    d = {j: -v for j, v in xh.items()}
                    d[xi] = d.get(xi, Fraction(0)) + 1
                    d[zi] = -lh
                    out.append((("beta1", k, i), d, c - lh))
                if kind == "Aprime":
                    uh, lh = _F(self.uhat[k][i]), _F(self.lhat[k][i])
                    out.append((("xhat_hi", k, i), dict(xh), uh - c))
                    out.append((("xhat_lo", k, i), {j: -v for j, v in xh.items()}, c - lh))
                if kind in ("A", "Aprime"):
                    for I in product((0, 1), repeat=fan_in):
                        if kind == "A" and (sum(I) == 0 or sum(I) == fan_in):
                            continue
                        d, r = self.mask_row(k, i, I)
                        out.append((("beta", k, i, I), d, r))
                if kind == "M+" and masks is not None:
                    for I in masks.get((k, i), []):
                        d, r = self.mask_row(k, i, tuple(int(v) for v in I))
                        out.append((("beta", k, i, tuple(int(v) for v in I)), d, r))
        return out

    def solve(self, kind, obj_row, obj_const=0.0, masks=None, sense=1):
        """min (sense * (obj_row . x_L + obj_const)) over the relaxation; returns the value of
        obj_row . x_L + obj_const at the optimum (exact Fraction)."""
        c = [Fraction(0)] * self.nvar
        for j, w in enumerate(obj_row):
            c[self.xoff[self.L] + j] = sense * _F(w)
        R = self.rows(kind, masks)
        rows = []
        for _, d, _ in R:
            r = [Fraction(0)] * self.nvar
            for j, v in d.items():
                r[j] = v
            rows.append(r)
        val, v = simplex_min(c, rows, [r for _, _, r in R], self.lb, self.ub)
        if val is None:
            return None
        return sense * val + _F(obj_const)


def layer_bounds_lp(Ws, bs, lo0, hi0, kind="M"):
    """Pre-activation bounds of every hidden layer by LPs over the relaxation of the layers
    before it (problem 20 of App. E with C_k = kind). Returns 1-based (lhat, uhat, lo, hi)."""
    lhat, uhat = [None], [None]
    lo, hi = [np.asarray(lo0, np.float64)], [np.asarray(hi0, np.float64)]
    for k in range(1, len(Ws) + 1):
        W, b = Ws[k - 1], bs[k - 1]
        if k == 1:
            Wp, Wn = np.maximum(W, 0), np.minimum(W, 0)
            lh = Wp @ lo[0] + Wn @ hi[0] + b
            uh = Wp @ hi[0] + Wn @ lo[0] + b
        else:
            sub = NetLP(Ws[:k - 1], bs[:k - 1], lhat, uhat, lo, hi)
            lh = np.array([float(sub.solve(kind, W[i], b[i], sense=1)) for i in range(W.shape[0])])
            uh = np.array([float(sub.solve(kind, W[i], b[i], sense=-1)) for i in range(W.shape[0])])
        lhat.append(lh)
        uhat.append(uh)
        lo.append(np.maximum(lh, 0))
        hi.append(np.maximum(uh, 0))
    return lhat, uhat, lo, hi


def fig4_network():
    """The example network of Fig. 4 / App. F.1: two hidden layers of two ReLUs, output
    [2, -1] x_2, input box [-1, 1]^2."""
    W1 = np.array([[1.0, -1.0], [1.0, -1.0]])
    b1 = np.array([-1.0, 1.0])
    W2 = np.array([[-1.0, 2.0], [-2.0, 1.0]])
    b2 = np.array([-2.0, 0.0])
    w3 = np.array([2.0, -1.0])
    return [W1, W2], [b1, b2], w3, 0.0, -np.ones(2), np.ones(2)

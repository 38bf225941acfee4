"""The dual of the tighter relaxation restricted to an active set (oracle; test infrastructure only).

Notation follows Sec. 3-4 of the paper, layers k = 0..n, 1-based lists. Dual variables of hidden
layer k = 1..n-1: alpha_k (x_k >= xhat_k), beta_{k,0} (x_k <= uhat_k z_k),
beta_{k,1} (x_k <= xhat_k - lhat_k (1 - z_k)), and one beta_{k,I} per mask I in the active set B_k
(the exponential-family constraint of eq. 4). Dummies alpha_0 = beta_0 = 0, alpha_n = 1, beta_n = 0.

Readings of the paper taken here (each is justified where it is used):
  * the box for x_k in eqs. (7) and (13) is the post-activation box [l_k, u_k] (the dual's domain,
    eq. 5), not [lhat_k, uhat_k];
  * eq. (8) minimises the Lagrangian, whose x_0 term is -f_0^T x_0, so x_0* = u_0 where f_0 >= 0;
  * the last term of eq. (9) enters with a minus sign, -(W o (1-I) o Ucheck)<>z, as it does in the
    Lagrangian of App. D and in the proof of Proposition 1;
  * the constant term includes b_n (alpha_n = 1), as the Lagrangian of App. D does.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import relaxation as rx


@dataclass
class Slot:
    """One active-set variable beta_{k,I}: its mask, values and the mask's row sums."""
    I: np.ndarray            # bool [n_k, n_{k-1}]
    beta: np.ndarray         # [n_k]
    lam: np.ndarray          # sum_j W I Lcheck
    mu: np.ndarray           # sum_j W (1-I) Ucheck
    m: np.ndarray = None     # Adam first moment
    v: np.ndarray = None     # Adam second moment
    added_at: int = 0        # Active Set iteration at which the mask was added


@dataclass
class DualState:
    alpha: list
    beta0: list
    beta1: list
    slots: list = field(default_factory=list)   # slots[k] = list[Slot]

    @staticmethod
    def zeros(P) -> "DualState":
        z = [None] + [np.zeros(P.widths[k]) for k in range(1, P.n)]
        return DualState([None if a is None else a.copy() for a in z],
                         [None if a is None else a.copy() for a in z],
                         [None if a is None else a.copy() for a in z],
                         [[] for _ in range(P.n)])


def add_slot(P, st: DualState, k: int, I: np.ndarray, added_at: int = 0, beta=None):
    lam, mu = rx.row_sums(P.W[k], P.lo[k - 1], P.hi[k - 1], I)
    nk = P.widths[k]
    b = np.zeros(nk) if beta is None else np.asarray(beta, np.float64).copy()
    st.slots[k].append(Slot(I, b, lam, mu, np.zeros(nk), np.zeros(nk), added_at))


def coefficients(P, st: DualState):
    """f_k for k = 0..n-1 and g_k for k = 1..n-1 (Sec. 4.1, f_B and g_B)."""
    n = P.n
    f = [None] * n
    g = [None] * n
    for k in range(n):
        if k == n - 1:
            up = P.W[n].T @ np.ones(1)                 # W_n^T alpha_n with alpha_n = 1
        else:
            up = P.W[k + 1].T @ st.alpha[k + 1]
        fk = -up
        if k >= 1:
            fk = fk + st.alpha[k] - st.beta0[k] - st.beta1[k]
            for sl in st.slots[k]:
                fk = fk - sl.beta
        if k + 1 <= n - 1:
            fk = fk + P.W[k + 1].T @ st.beta1[k + 1]   # mask I = 1 term
            for sl in st.slots[k + 1]:
                fk = fk + (P.W[k + 1] * sl.I).T @ sl.beta
        f[k] = fk
        if k >= 1:
            gk = st.beta0[k] * P.uhat[k] + st.beta1[k] * P.lhat[k]
            for sl in st.slots[k]:
                gk = gk + sl.beta * (sl.lam + sl.mu + P.b[k])
            g[k] = gk
    return f, g


def x0_vertex(P, f0):
    """argmin of -f0^T x_0 over the input set: the box vertex (u_0 where f0 >= 0), or over the
    ellipsoid inscribed in the box (P.ball) c + e^2 f0 / |e f0|_2 (c where f0 = 0)."""
    if not getattr(P, "ball", False):
        return np.where(f0 >= 0, P.hi[0], P.lo[0])
    c = 0.5 * (P.lo[0] + P.hi[0])
    e = 0.5 * (P.hi[0] - P.lo[0])
    nrm = float(np.sqrt(((e * f0) ** 2).sum()))
    return c + (e * e * f0 / nrm if nrm > 0 else 0.0)


def retract_x0(P, x0):
    """Into the input set: the box clip, or over the ellipsoid the radial retraction
    c + (x - c) / max(1, |(x - c) / e|_2) (its exact projection when the half-widths are equal)."""
    if not getattr(P, "ball", False):
        return np.clip(x0, P.lo[0], P.hi[0])
    c = 0.5 * (P.lo[0] + P.hi[0])
    e = 0.5 * (P.hi[0] - P.lo[0])
    free = e > 0
    r = float(np.sqrt((((x0 - c)[free] / e[free]) ** 2).sum()))
    return np.where(free, c + (x0 - c) / max(1.0, r), c)


def closed_form(P, f, g):
    """Inner minimisation, eqs. (7)-(8): x_k* at the upper end of its box where f_k >= 0.

    Over an ellipsoid input set (P.ball; centre c, half-widths e of the box) the x_0 part,
    min -f_0^T x_0, is attained at x_0* = c + e^2 f_0 / |e f_0|_2 (c where f_0 = 0), value
    -f_0^T c - |e f_0|_2 (Sec. 2: the input set needs only a closed-form linear minimisation)."""
    x = [np.where(f[k] >= 0, P.hi[k], P.lo[k]) for k in range(P.n)]
    x[0] = x0_vertex(P, f[0])
    z = [None] + [np.where(g[k] >= 0, 1.0, 0.0) for k in range(1, P.n)]
    return x, z


def lagrangian(P, st: DualState, f, g, x, z) -> float:
    """The Lagrangian of eq. (6) in its collected form (App. D, last display), b_n included."""
    val = float(P.b[P.n][0])
    for k in range(1, P.n):
        val += float(P.b[k] @ st.alpha[k])
        val += float(st.beta1[k] @ (P.lhat[k] - P.b[k]))
        for sl in st.slots[k]:
            val += float(sl.beta @ sl.lam)
        val -= float(g[k] @ z[k])
    for k in range(P.n):
        val -= float(f[k] @ x[k])
    return val


def lagrangian_constraint_form(P, st: DualState, x, z) -> float:
    """The Lagrangian of App. D, first display: multipliers times constraint residuals."""
    val = float((P.W[P.n] @ x[P.n - 1] + P.b[P.n])[0])
    for k in range(1, P.n):
        xhat = P.W[k] @ x[k - 1] + P.b[k]
        val += float(st.alpha[k] @ (xhat - x[k]))
        val += float(st.beta0[k] @ (x[k] - z[k] * P.uhat[k]))
        val += float(st.beta1[k] @ (x[k] - xhat + (1 - z[k]) * P.lhat[k]))
        Lc, Uc = rx.interval_matrices(P.W[k], P.lo[k - 1], P.hi[k - 1])
        for sl in st.slots[k]:
            WI = P.W[k] * sl.I
            r = ((WI * Lc).sum(1) * (1 - z[k]) - WI @ x[k - 1] - P.b[k] * z[k]
                 - (P.W[k] * (~sl.I) * Uc).sum(1) * z[k] + x[k])
            val += float(sl.beta @ r)
    return val


def supergradient(P, st: DualState, x, z):
    """Eq. (9): returns dict with lists galpha, gbeta0, gbeta1 (k = 1..n-1) and gslots[k][b]."""
    ga, g0, g1, gs = [None], [None], [None], [[]]
    for k in range(1, P.n):
        xhat = P.W[k] @ x[k - 1] + P.b[k]
        ga.append(xhat - x[k])
        g0.append(x[k] - z[k] * P.uhat[k])
        g1.append(x[k] - xhat + (1 - z[k]) * P.lhat[k])
        lst = []
        for sl in st.slots[k]:
            WIx = (P.W[k] * sl.I) @ x[k - 1]
            lst.append(x[k] - WIx + sl.lam * (1 - z[k]) - z[k] * (P.b[k] + sl.mu))
        gs.append(lst)
    return dict(galpha=ga, gbeta0=g0, gbeta1=g1, gslots=gs)


def evaluate(P, st: DualState):
    """d_B at the given duals: (value, f, g, x*, z*) (Alg. 1 return line)."""
    f, g = coefficients(P, st)
    x, z = closed_form(P, f, g)
    return lagrangian(P, st, f, g, x, z), f, g, x, z

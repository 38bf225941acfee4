"""Interval matrices, the separation oracle and mask row sums (oracle; test infrastructure only).

Sec. 2.2 of the paper defines, for layer k with weights W_k and the previous layer's
post-activation bounds l_{k-1}, u_{k-1}:
    Lcheck[i, j] = l[j] if W[i, j] >= 0 else u[j]
    Ucheck[i, j] = u[j] if W[i, j] >= 0 else l[j]
and eq. (3), the linear-time oracle for the most violated constraint of the exponential family:
    I[i, j] = 1  iff  ((1 - z[i]) * Lcheck[i, j] + z[i] * Ucheck[i, j] - x[j]) * W[i, j] >= 0.

`mask` decides eq. (3) exactly for the given floating-point values (no rounding enters the
decision). Multiplying out the sign of W (an exact rearrangement):
    W = 0  -> 1 (the coefficient is 0)
    W > 0  -> a = z (u - l) - (x - l) >= 0
    W < 0  -> a = z (u - l) - (u - x) >= 0
The sign of a is exact by comparisons alone where z is 0 or 1, where u = l or where the
subtrahend vanishes (every Active Set iterate and every fixed input); elsewhere a float64
evaluation decides when it clears its rounding-error bound, and rational arithmetic decides the
few entries that it does not clear. `mask_literal` evaluates the printed formula in float64 (its
rounding flips bits where the coefficient is exactly 0), `mask_exact` in rational arithmetic entry
by entry (slow; small inputs only).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

_EPS = 2.0 ** -53


def interval_matrices(W: np.ndarray, l: np.ndarray, u: np.ndarray):
    """(Lcheck, Ucheck), both [n_k, n_{k-1}] (Sec. 2.2)."""
    pos = W >= 0
    Lc = np.where(pos, l[None, :], u[None, :])
    Uc = np.where(pos, u[None, :], l[None, :])
    return Lc, Uc


def mask(W, l, u, x, z) -> np.ndarray:
    """Eq. (3), decided exactly: bool [n_k, n_{k-1}]."""
    W = np.asarray(W, np.float64)
    l = np.asarray(l, np.float64)
    u = np.asarray(u, np.float64)
    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    n, m = W.shape
    pos = W > 0
    zc = np.broadcast_to(z[:, None], (n, m))
    # subtrahend s = x - l (W > 0) or u - x (W < 0); its sign by comparison
    s_pos = np.where(pos, x[None, :] > l[None, :], u[None, :] > x[None, :])    # s > 0
    s_neg = np.where(pos, x[None, :] < l[None, :], u[None, :] < x[None, :])    # s < 0
    s_zero = ~(s_pos | s_neg)
    d_zero = np.broadcast_to((u == l)[None, :], (n, m))
    # z = 0: a = -s; z = 1: a = (u - l) - s = u - x (W > 0) or x - l (W < 0)
    a_one_ge = np.where(pos, u[None, :] >= x[None, :], x[None, :] >= l[None, :])
    out = np.empty((n, m), bool)
    decided = np.zeros((n, m), bool)
    # a = z (u - l) - s with u - l = 0: a = -s
    case = d_zero
    out[case] = ~s_pos[case]
    decided |= case
    case = ~decided & (zc == 0.0)
    out[case] = ~s_pos[case]
    decided |= case
    case = ~decided & (zc == 1.0)
    out[case] = a_one_ge[case]
    decided |= case
    # s = 0: a = z (u - l), with u - l > 0 here: its sign is the sign of z
    case = ~decided & s_zero
    out[case] = zc[case] >= 0.0
    decided |= case
    rest = ~decided
    if rest.any():
        d = (u - l)[None, :]
        s = np.where(pos, x[None, :] - l[None, :], u[None, :] - x[None, :])
        a = zc * d - s
        tol = 8.0 * _EPS * (np.abs(zc) * np.abs(d) + np.abs(s)) + 1e-300
        sure = rest & (np.abs(a) > tol)
        out[sure] = a[sure] >= 0.0
        for i, j in zip(*np.nonzero(rest & ~sure)):
            zi, lj, uj, xj = (Fraction(float(v)) for v in (z[i], l[j], u[j], x[j]))
            sj = xj - lj if W[i, j] > 0 else uj - xj
            out[i, j] = zi * (uj - lj) - sj >= 0
    out |= W == 0
    return out


def mask_literal(W, l, u, x, z) -> np.ndarray:
    """Eq. (3) evaluated as printed, in float64 (exact at binary z and x in {l, u})."""
    Lc, Uc = interval_matrices(W, l, u)
    zc = np.asarray(z, np.float64)[:, None]
    coef = ((1.0 - zc) * Lc + zc * Uc - np.asarray(x, np.float64)[None, :]) * W
    return coef >= 0


def mask_exact(W, l, u, x, z) -> np.ndarray:
    """Eq. (3) in exact rational arithmetic (slow; small inputs only)."""
    n, m = W.shape
    I = np.zeros((n, m), bool)
    for i in range(n):
        zi = Fraction(float(z[i]))
        for j in range(m):
            w = Fraction(float(W[i, j]))
            lj, uj, xj = Fraction(float(l[j])), Fraction(float(u[j])), Fraction(float(x[j]))
            Lc, Uc = (lj, uj) if w >= 0 else (uj, lj)
            I[i, j] = ((1 - zi) * Lc + zi * Uc - xj) * w >= 0
    return I


def row_sums(W, l, u, I):
    """lam[i] = sum_j W I Lcheck, mu[i] = sum_j W (1 - I) Ucheck: the (.)<>1 terms of eq. (4)."""
    Lc, Uc = interval_matrices(W, l, u)
    lam = (W * I * Lc).sum(axis=1)
    mu = (W * (~I) * Uc).sum(axis=1)
    return lam, mu


def constraint_violation(W, b, l, u, I_row, x_prev, x_i, z_i, i):
    """Violation of the exponential-family constraint of neuron i with mask row I_row (eq. 4):
    x_i - [ (W*I) x_prev + z b - (W*I*Lc)<>(1 - z) + (W*(1-I)*Uc)<>z ]."""
    Lc, Uc = interval_matrices(W[i:i + 1], l, u)
    w = W[i]
    rhs = (w * I_row) @ x_prev + z_i * b[i] - (w * I_row * Lc[0]).sum() * (1 - z_i) \
        + (w * (1 - I_row) * Uc[0]).sum() * z_i
    return x_i - rhs

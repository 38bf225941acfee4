"""Interval matrices, the separation oracle and mask row sums (oracle; test infrastructure only).

Sec. 2.2 of the paper defines, for layer k with weights W_k and the previous layer's
post-activation bounds l_{k-1}, u_{k-1}:
    Lcheck[i, j] = l[j] if W[i, j] >= 0 else u[j]
    Ucheck[i, j] = u[j] if W[i, j] >= 0 else l[j]
and eq. (3), the linear-time oracle for the most violated constraint of the exponential family:
    I[i, j] = 1  iff  ((1 - z[i]) * Lcheck[i, j] + z[i] * Ucheck[i, j] - x[j]) * W[i, j] >= 0.

Where floating point decides the bit, the decision is taken in float32, the precision of the
paper's implementation and of the CUDA kernels, in the equivalent threshold form
    W = 0 or l = u                   -> 1
    W > 0  -> z >= (x - l) / (u - l)
    W < 0  -> z >= (u - x) / (u - l)
with the quotient rounded to nearest in float32 (each operation rounded). It equals the real-number
rule of eq. (3) whenever z is 0 or 1 and x is l or u (every Active Set iterate), and whenever z is not
within one float32 ulp of the quotient. When l = u the variable is fixed, x = l = u, and the
coefficient is exactly zero, so the bit is 1. `mask_exact` evaluates eq. (3) in rational arithmetic.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def interval_matrices(W: np.ndarray, l: np.ndarray, u: np.ndarray):
    """(Lcheck, Ucheck), both [n_k, n_{k-1}] (Sec. 2.2)."""
    pos = W >= 0
    Lc = np.where(pos, l[None, :], u[None, :])
    Uc = np.where(pos, u[None, :], l[None, :])
    return Lc, Uc


def mask(W, l, u, x, z) -> np.ndarray:
    """Eq. (3) with float32 decisions: bool [n_k, n_{k-1}]."""
    l32 = np.asarray(l, np.float32)
    u32 = np.asarray(u, np.float32)
    x32 = np.asarray(x, np.float32)
    z32 = np.asarray(z, np.float32)
    fixed = l32 == u32
    with np.errstate(divide="ignore", invalid="ignore"):
        den = np.where(fixed, np.float32(1), u32 - l32)
        tp = (x32 - l32) / den
        tn = (u32 - x32) / den
    tp = tp.astype(np.float32)
    tn = tn.astype(np.float32)
    zc = z32[:, None]
    I = np.where(W > 0, zc >= tp[None, :], zc >= tn[None, :])
    I = I | (W == 0) | fixed[None, :]
    return I


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

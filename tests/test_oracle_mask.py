"""Pins of the separation oracle, eq. (3), against brute force over every mask (Prop. 1)."""
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

from oracle import relaxation as rx
from paper_2101_05844_gb300.synth import SplitMix64


def _row_case(rng, m, binary):
    W = rng.normal(m)
    W[rng.uniform(m) < 0.15] = 0.0                     # exact zeros: ties
    W = W.astype(np.float32).astype(np.float64)
    l = (rng.uniform(m) - 0.5).astype(np.float32).astype(np.float64)
    u = l + (rng.uniform(m) * 2).astype(np.float32).astype(np.float64)
    u = u.astype(np.float32).astype(np.float64)
    fixed = rng.uniform(m) < 0.15
    u[fixed] = l[fixed]                                  # l = u: fixed inputs
    if binary:
        x = np.where(rng.uniform(m) < 0.5, l, u)
        z = np.array([float(rng.uniform(1)[0] < 0.5)])
    else:
        x = (l + rng.uniform(m) * (u - l)).astype(np.float32).astype(np.float64)
        x = np.clip(x, l, u)
        z = rng.uniform(1).astype(np.float32).astype(np.float64)
    return W[None, :], l, u, x, z


def _coeffs_exact(W, l, u, x, z):
    out = []
    for j in range(W.shape[1]):
        w = Fraction(float(W[0, j]))
        lj, uj, xj = Fraction(float(l[j])), Fraction(float(u[j])), Fraction(float(x[j]))
        Lc, Uc = (lj, uj) if w >= 0 else (uj, lj)
        zi = Fraction(float(z[0]))
        out.append(((1 - zi) * Lc + zi * Uc - xj) * w)
    return out


@pytest.mark.parametrize("binary", [True, False])
def test_oracle_mask_maximises_violation_over_all_masks(binary):
    """Proof of Prop. 1: the oracle's row maximises sum_j I_j c_j over all 2^m masks, and it is the
    largest maximiser under set inclusion (eq. 3 keeps every zero coefficient)."""
    rng = SplitMix64(11 + binary)
    for trial in range(40):
        m = 1 + trial % 10
        W, l, u, x, z = _row_case(rng, m, binary)
        c = _coeffs_exact(W, l, u, x, z)
        I = rx.mask_exact(W, l, u, x, z)[0]
        best = max(sum(ci for ci, b in zip(c, bits) if b) for bits in product((0, 1), repeat=m))
        assert sum(ci for ci, b in zip(c, I) if b) == best
        maximisers = [bits for bits in product((0, 1), repeat=m)
                      if sum(ci for ci, b in zip(c, bits) if b) == best]
        for bits in maximisers:
            assert all(bi <= Ii for bi, Ii in zip(bits, I))


def test_float32_threshold_mask_equals_exact_at_active_set_iterates():
    """At binary z and x in {l, u} (every Active Set iterate) the float32 threshold form, the
    literal float64 form and exact arithmetic agree bit for bit."""
    rng = SplitMix64(5)
    for trial in range(200):
        m = 1 + trial % 12
        W, l, u, x, z = _row_case(rng, m, True)
        e = rx.mask_exact(W, l, u, x, z)
        assert (rx.mask(W, l, u, x, z) == e).all()
        assert (rx.mask_literal(W, l, u, x, z) == e).all()


def test_float32_threshold_mask_matches_exact_away_from_thresholds():
    """For continuous z the float32 decision differs from the exact one only when z lies within
    one float32 ulp of the threshold (x - l)/(u - l) or (u - x)/(u - l)."""
    rng = SplitMix64(6)
    for trial in range(300):
        m = 1 + trial % 12
        W, l, u, x, z = _row_case(rng, m, False)
        a, e = rx.mask(W, l, u, x, z)[0], rx.mask_exact(W, l, u, x, z)[0]
        for j in np.nonzero(a != e)[0]:
            tau = (Fraction(float(x[j])) - Fraction(float(l[j]))) / (Fraction(float(u[j])) - Fraction(float(l[j])))
            if W[0, j] < 0:
                tau = 1 - tau
            ulp = np.spacing(np.float32(z[0]))
            assert abs(Fraction(float(z[0])) - tau) <= Fraction(float(ulp))


def test_threshold_ties_at_exact_equality():
    # z exactly on the threshold: coefficient exactly 0 -> bit 1 (eq. 3 uses >= 0)
    W = np.array([[1.0, -1.0]])
    l = np.array([0.0, 0.0])
    u = np.array([4.0, 4.0])
    x = np.array([1.0, 3.0])
    z = np.array([0.25])
    assert rx.mask(W, l, u, x, z).tolist() == [[True, True]]
    assert rx.mask_exact(W, l, u, x, z).tolist() == [[True, True]]
    z = np.array([np.nextafter(np.float32(0.25), np.float32(0))], dtype=np.float64)
    assert rx.mask(W, l, u, x, z).tolist() == [[False, False]]

"""Pins of the separation oracle, eq. (3), against brute force over every mask (Prop. 1)."""
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

from oracle import relaxation as rx
from paper_2101_05844_gb300.synth import SplitMix64


def _row_case(rng, m, binary, f32=True):
    W = rng.normal(m)
    W[rng.uniform(m) < 0.15] = 0.0                     # exact zeros: ties
    l = rng.uniform(m) - 0.5
    u = l + rng.uniform(m) * 2
    if f32:
        W, l, u = (v.astype(np.float32).astype(np.float64) for v in (W, l, u))
    fixed = rng.uniform(m) < 0.15
    u[fixed] = l[fixed]                                  # l = u: fixed inputs
    if binary:
        x = np.where(rng.uniform(m) < 0.5, l, u)
        z = np.array([float(rng.uniform(1)[0] < 0.5)])
    else:
        x = l + rng.uniform(m) * (u - l)
        z = rng.uniform(1)
        if f32:
            x, z = x.astype(np.float32).astype(np.float64), z.astype(np.float32).astype(np.float64)
        x = np.clip(x, l, u)
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
@pytest.mark.parametrize("f32", [True, False])
def test_oracle_mask_maximises_violation_over_all_masks(binary, f32):
    """Proof of Prop. 1: the oracle's row maximises sum_j I_j c_j over all 2^m masks (m <= 12
    inputs), and it is the largest maximiser under set inclusion (eq. 3 keeps every zero
    coefficient). Checked for `mask` itself, at Active Set iterates (binary z, x at an end of its
    box) and at continuous points, on float32 and on float64 values."""
    rng = SplitMix64(11 + binary + 2 * f32)
    for trial in range(24):
        m = 1 + trial % 12
        W, l, u, x, z = _row_case(rng, m, binary, f32)
        c = _coeffs_exact(W, l, u, x, z)
        I = rx.mask(W, l, u, x, z)[0]
        sums = {bits: sum(ci for ci, b in zip(c, bits) if b) for bits in product((0, 1), repeat=m)}
        best = max(sums.values())
        assert sum(ci for ci, b in zip(c, I) if b) == best
        for bits, v in sums.items():
            if v == best:
                assert all(bi <= Ii for bi, Ii in zip(bits, I))


@pytest.mark.parametrize("f32", [True, False])
def test_mask_equals_exact_rational_evaluation(f32):
    """`mask` equals eq. (3) evaluated in rational arithmetic entry by entry, on continuous rows
    (with zero weights, fixed inputs, z = 0 and z = 1 mixed in) and at Active Set iterates."""
    rng = SplitMix64(21 + f32)
    for trial in range(240):
        m = 1 + trial % 12
        W, l, u, x, z = _row_case(rng, m, trial % 3 == 0, f32)
        if trial % 7 == 1:
            z = np.array([0.0 if trial % 2 else 1.0])
        np.testing.assert_array_equal(rx.mask(W, l, u, x, z), rx.mask_exact(W, l, u, x, z))


def test_mask_decides_within_an_ulp_of_the_threshold():
    """z on the threshold (coefficient exactly 0: bit 1, eq. 3 uses >= 0), and one float64 ulp to
    either side, for both signs of W; a float rounding of the coefficient would get some of these
    wrong."""
    W = np.array([[1.0, -1.0]])
    l = np.array([0.1, 0.1])
    u = np.array([0.7, 0.7])
    x = np.array([0.25, 0.55])
    # thresholds: (x - l) / (u - l) = 0.25 for W > 0 and (u - x) / (u - l) = 0.25 for W < 0, in
    # exact arithmetic; the float64 values of 0.1, 0.25, 0.55, 0.7 make them slightly different
    for j, sgn in ((0, 1), (1, -1)):
        lj, uj, xj = (Fraction(float(v)) for v in (l[j], u[j], x[j]))
        tau = (xj - lj) / (uj - lj) if sgn > 0 else (uj - xj) / (uj - lj)
        t = float(tau)
        for zz in (np.nextafter(t, 0), t, np.nextafter(t, 1)):
            want = Fraction(float(zz)) >= tau
            got = rx.mask(W[:, j:j + 1], l[j:j + 1], u[j:j + 1], x[j:j + 1], np.array([zz]))[0, 0]
            assert got == want, (j, zz, float(tau))
    # an exactly representable threshold: z = 1/4 gives coefficient 0 and bit 1
    W = np.array([[1.0, -1.0]])
    l, u, x = np.array([0.0, 0.0]), np.array([4.0, 4.0]), np.array([1.0, 3.0])
    assert rx.mask(W, l, u, x, np.array([0.25])).tolist() == [[True, True]]
    assert rx.mask(W, l, u, x, np.array([np.nextafter(0.25, 0.0)])).tolist() == [[False, False]]


def test_literal_float64_formula_flips_bits_that_mask_gets_right():
    """At fixed inputs (l = u) the printed coefficient is exactly 0, but its float64 evaluation
    ((1 - z) l + z l - x) W rounds to a small nonzero value for many continuous z: the literal
    form then drops bits that eq. (3) sets. `mask` keeps them (it decides exactly)."""
    rng = SplitMix64(8)
    flips = 0
    for trial in range(200):
        l = rng.uniform(6) * 3 - 1
        W = rng.normal(6)[None, :]
        z = rng.uniform(1)
        x = l.copy()
        exact = rx.mask_exact(W, l, l, x, z)
        assert exact.all()
        np.testing.assert_array_equal(rx.mask(W, l, l, x, z), exact)
        flips += int((rx.mask_literal(W, l, l, x, z) != exact).sum())
    assert flips > 0


def _ru32(q: Fraction) -> np.float32:
    """The smallest float32 >= q (by stepping, from the float32 nearest to float(q))."""
    f = np.float32(float(q))
    while Fraction(float(f)) < q:
        f = np.nextafter(f, np.float32(np.inf))
    while True:
        g = np.nextafter(f, np.float32(-np.inf))
        if Fraction(float(g)) >= q:
            f = g
        else:
            return f


def test_rounded_up_float32_threshold_decides_exactly():
    """The reading the CUDA kernels take for Saddle Point masks: with float32 x, l, u, z, the
    real-number decision z >= tau (eq. 3 in threshold form) equals the float32 compare
    z >= RU_fp32(tau), tau rounded up to float32, for both signs of W."""
    rng = SplitMix64(31)
    for trial in range(400):
        W, l, u, x, z = _row_case(rng, 1 + trial % 8, False, True)
        e = rx.mask_exact(W, l, u, x, z)[0]
        z32 = np.float32(z[0])
        for j in range(W.shape[1]):
            if W[0, j] == 0 or l[j] == u[j]:
                continue
            lj, uj, xj = (Fraction(float(v)) for v in (l[j], u[j], x[j]))
            tau = (xj - lj) / (uj - lj) if W[0, j] > 0 else (uj - xj) / (uj - lj)
            assert bool(z32 >= _ru32(tau)) == bool(e[j])
            # and on the threshold itself: z = RU(tau) selects, the float32 below it does not
            t = _ru32(tau)
            zt = np.array([float(t)])
            assert rx.mask_exact(W[:, j:j + 1], l[j:j + 1], u[j:j + 1], x[j:j + 1], zt)[0, 0]
            zb = np.array([float(np.nextafter(t, np.float32(-np.inf)))])
            assert not rx.mask_exact(W[:, j:j + 1], l[j:j + 1], u[j:j + 1], x[j:j + 1], zb)[0, 0]

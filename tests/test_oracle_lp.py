"""Pins of the oracle's LP relaxations against the paper's worked example (App. F.1, Fig. 4)."""
import json
import os
from fractions import Fraction

import numpy as np

from oracle import lp

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig4_lp.json")))


def test_fig4_first_layer_post_activation_bounds():
    Ws, bs, w3, b3, lo0, hi0 = lp.fig4_network()
    lh, uh, lo, hi = lp.layer_bounds_lp(Ws, bs, lo0, hi0, "M")
    assert list(lo[1]) == GOLD["printed"]["l_1"]
    assert list(hi[1]) == GOLD["printed"]["u_1"]


def test_fig4_uhat2_lp_is_tighter_than_interval():
    Ws, bs, w3, b3, lo0, hi0 = lp.fig4_network()
    lh, uh, lo, hi = lp.layer_bounds_lp(Ws, bs, lo0, hi0, "M")
    assert uh[2][1] == GOLD["printed"]["uhat_2[1]"]
    # M^+_2[1]: the interval maximum of [-2, 1] x_1 over [l_1, u_1]
    W2 = Ws[1]
    mplus = np.maximum(W2[1], 0) @ hi[1] + np.minimum(W2[1], 0) @ lo[1] + bs[1][1]
    assert mplus == GOLD["printed"]["M^+_2[1]"]


def test_fig4_output_bounds_match_printed_values():
    Ws, bs, w3, b3, lo0, hi0 = lp.fig4_network()
    lh, uh, lo, hi = lp.layer_bounds_lp(Ws, bs, lo0, hi0, "M")
    N = lp.NetLP(Ws, bs, lh, uh, lo, hi)
    vM = N.solve("M", w3, b3)
    vAp = N.solve("Aprime", w3, b3)
    assert round(float(vM), 4) == GOLD["printed"]["lhat_3 with M_k"]
    assert round(float(vAp), 4) == GOLD["printed"]["lhat_3 with A'_k"]
    # the example's point: M_k is tighter than A'_k here
    assert vM > vAp


def test_fig4_anderson_with_preactivation_bounds_is_tightest():
    """A_k is contained in both M_k and A'_k (Sec. 2.2 and App. F), so its LP bound is >= both."""
    Ws, bs, w3, b3, lo0, hi0 = lp.fig4_network()
    lh, uh, lo, hi = lp.layer_bounds_lp(Ws, bs, lo0, hi0, "M")
    N = lp.NetLP(Ws, bs, lh, uh, lo, hi)
    vA = N.solve("A", w3, b3)
    assert vA >= N.solve("M", w3, b3)
    assert vA >= N.solve("Aprime", w3, b3)
    assert vA == Fraction(-81, 76)  # exact value of this LP (not printed in the paper)


def test_simplex_on_textbook_lp():
    # min -x - y s.t. x + 2y <= 4, 3x + y <= 6, 0 <= x, y <= 10 -> optimum at (8/5, 6/5)
    val, v = lp.simplex_min([-1, -1], [[1, 2], [3, 1]], [4, 6], [0, 0], [10, 10])
    assert v == [Fraction(8, 5), Fraction(6, 5)] and val == Fraction(-14, 5)
    # infeasible: x >= 5 (as -x <= -5) with x <= 1
    assert lp.simplex_min([1], [[-1]], [-5], [0], [1])[0] is None

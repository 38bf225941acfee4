"""Pins of the oracle's dual (Sec. 3-4, App. B, App. D) against closed forms, the primal LP,
directional derivatives and sampling."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import active_set as AS
from oracle import dual as du
from oracle import lp
from oracle import network as nw
from oracle import relaxation as rx
from paper_2101_05844_gb300 import synth
from tests.helpers import fig4_problem, netlp_for, sample_min_output


def _random_state(P, rng, n_slots=2, scale=0.3):
    st = du.DualState.zeros(P)
    for k in range(1, P.n):
        nk = P.widths[k]
        for arr in (st.alpha, st.beta0, st.beta1):
            v = rng.uniform(nk) * scale
            v[rng.uniform(nk) < 0.3] = 0
            arr[k] = v
        for s in range(n_slots):
            x = np.where(rng.uniform(P.widths[k - 1]) < 0.5, P.lo[k - 1], P.hi[k - 1])
            z = (rng.uniform(nk) < 0.5).astype(float)
            I = rx.mask(P.W[k], P.lo[k - 1], P.hi[k - 1], x, z)
            du.add_slot(P, st, k, I, beta=rng.uniform(nk) * scale)
    return st


def _random_point(P, rng):
    x = [P.lo[k] + rng.uniform(P.widths[k]) * (P.hi[k] - P.lo[k]) for k in range(P.n)]
    z = [None] + [rng.uniform(P.widths[k]) for k in range(1, P.n)]
    return x, z


@pytest.mark.parametrize("name", ["mlp_tiny", "small_conv", "mlp_5_7_6_3"])
def test_zero_duals_give_interval_bound(name):
    """App. B.3: with every dual at zero the Big-M bound is the interval-propagation bound."""
    prob = synth.problem(name, seed=1)
    for P in nw.problems(prob):
        val = du.evaluate(P, du.DualState.zeros(P))[0]
        assert val == pytest.approx(P.ibp_output_bound(), abs=1e-12, rel=1e-12)


@pytest.mark.parametrize("name", ["mlp_tiny", "small_conv"])
def test_lagrangian_collected_equals_constraint_form(name):
    prob = synth.problem(name, seed=2)
    rng = synth.SplitMix64(3)
    for P in nw.problems(prob)[:2]:
        st = _random_state(P, rng)
        for _ in range(5):
            x, z = _random_point(P, rng)
            f, g = du.coefficients(P, st)
            a = du.lagrangian(P, st, f, g, x, z)
            b = du.lagrangian_constraint_form(P, st, x, z)
            assert a == pytest.approx(b, rel=1e-12, abs=1e-12)


def test_lagrangian_equals_lp_objective_plus_multiplier_residuals():
    """The Lagrangian of eq. (6) equals objective + sum of multipliers times constraint rows of
    the primal LP (4), the rows written independently from the primal problem."""
    prob = synth.problem("mlp_4_3_3_1", seed=4)
    P = nw.problems(prob)[0]
    rng = synth.SplitMix64(9)
    st = _random_state(P, rng, n_slots=2)
    N = netlp_for(P)
    masks = {(k, i): [sl.I[i] for sl in st.slots[k]] for k in range(1, P.n) for i in range(P.widths[k])}
    rows = N.rows("M+", masks)
    for _ in range(4):
        x, z = _random_point(P, rng)
        v = np.zeros(N.nvar)
        v[:P.widths[0]] = x[0]
        for k in range(1, P.n):
            v[N.xoff[k]:N.xoff[k] + P.widths[k]] = x[k]
            v[N.zoff[k]:N.zoff[k] + P.widths[k]] = z[k]
        tot = float((P.W[P.n] @ x[P.n - 1] + P.b[P.n])[0])
        seen = {}
        for label, d, r in rows:
            res = sum(float(c) * v[j] for j, c in d.items()) - float(r)
            kind, k, i = label[:3]
            if kind == "alpha":
                mult = st.alpha[k][i]
            elif kind == "beta0":
                mult = st.beta0[k][i]
            elif kind == "beta1":
                mult = st.beta1[k][i]
            else:
                idx = seen.get((k, i), 0)
                seen[(k, i)] = idx + 1
                mult = st.slots[k][idx].beta[i]
            tot += mult * res
        f, g = du.coefficients(P, st)
        assert du.lagrangian(P, st, f, g, x, z) == pytest.approx(tot, rel=1e-11, abs=1e-11)


def test_adding_a_zero_dual_mask_leaves_bound_unchanged():
    prob = synth.problem("small_conv", seed=5)
    P = nw.problems(prob)[0]
    st = _random_state(P, synth.SplitMix64(1), n_slots=1)
    v0, f, g, x, z = du.evaluate(P, st)
    for k in range(1, P.n):
        du.add_slot(P, st, k, rx.mask(P.W[k], P.lo[k - 1], P.hi[k - 1], x[k - 1], z[k]))
    assert du.evaluate(P, st)[0] == v0


@pytest.mark.parametrize("name", ["mlp_tiny", "small_conv"])
def test_supergradient_is_directional_derivative(name):
    """Eq. (9): d is linear around a point with a unique minimiser, with slope the supergradient."""
    prob = synth.problem(name, seed=6)
    P = nw.problems(prob)[0]
    rng = synth.SplitMix64(2)
    checked = 0
    for trial in range(10):
        st = _random_state(P, rng, n_slots=2)
        v0, f, g, x, z = du.evaluate(P, st)
        if min(np.abs(f[k]).min() for k in range(P.n)) < 1e-6 or \
           min(np.abs(g[k]).min() for k in range(1, P.n)) < 1e-6:
            continue
        gr = du.supergradient(P, st, x, z)
        h = 1e-7
        dirs, pred = [], 0.0
        for k in range(1, P.n):
            for arr, gk in ((st.alpha, gr["galpha"][k]), (st.beta0, gr["gbeta0"][k]),
                            (st.beta1, gr["gbeta1"][k])):
                d = rng.uniform(P.widths[k]) - 0.5
                arr[k] = arr[k] + h * d
                pred += h * float(gk @ d)
            for sl, gs in zip(st.slots[k], gr["gslots"][k]):
                d = rng.uniform(P.widths[k]) - 0.5
                sl.beta = sl.beta + h * d
                pred += h * float(gs @ d)
        v1, f1, g1, x1, z1 = du.evaluate(P, st)
        assert all((a == b).all() for a, b in zip(x, x1))
        assert (v1 - v0) == pytest.approx(pred, rel=1e-6, abs=1e-12)
        checked += 1
    assert checked >= 3


def test_weak_duality_against_sampled_outputs():
    """Every bound (Big-M, Active Set, the best over the run) is at most the network's minimum over
    10^6 uniform samples of the box and all its 2^8 vertices (weak duality, Sec. 3)."""
    prob = synth.problem("mlp_tiny", seed=7)
    P = nw.problems(prob)[0]
    opt = AS.Options(bigm_iters=60, as_iters=140, omega=40, max_cuts=5)
    fin, best, s = AS.solve(P, opt)
    assert max(s.trace + [fin]) == best
    m = sample_min_output(P, 1_000_000, seed=3)
    assert best <= m + 1e-9
    assert best > P.ibp_output_bound()       # the solver tightened the interval bound


def test_dual_bounds_below_exact_lps_on_tiny_network():
    """Weak duality against the exact LP optima: Big-M <= LP(M) <= LP(A), Active Set <= LP(A)."""
    prob = synth.problem("mlp_3_4_4_1", seed=8)
    P = nw.problems(prob)[0]
    N = netlp_for(P)
    vM = float(N.solve("M", P.W[P.n][0], P.b[P.n][0]))
    vA = float(N.solve("A", P.W[P.n][0], P.b[P.n][0]))
    assert vM <= vA + 1e-12
    bm, bm_best, _ = AS.solve(P, AS.Options(bigm_iters=600))
    assert bm_best <= vM + 1e-9
    fin, best, _ = AS.solve(P, AS.Options(bigm_iters=300, as_iters=900, as_lr0=1e-2,
                                          as_lr1=1e-4, omega=100, max_cuts=8))
    assert best <= vA + 1e-9
    assert best >= bm_best - 1e-9


def test_fig4_duals_converge_to_the_lp_optima():
    """Big-M reaches LP(M) = -27/22 (printed -1.2273) and Active Set reaches LP(A) = -81/76 on the
    Fig. 4 network, each from below."""
    P, _ = fig4_problem()
    _, bm, _ = AS.solve(P, AS.Options(bigm_iters=2000))
    assert -27 / 22 - 2e-4 <= bm <= -27 / 22 + 1e-12
    opt = AS.Options(bigm_iters=1000, as_iters=3000, as_lr0=1e-2, as_lr1=1e-4, omega=100,
                     max_cuts=16)
    _, best, _ = AS.solve(P, opt)
    assert -81 / 76 - 2e-4 <= best <= -81 / 76 + 1e-12


def test_active_set_best_bound_never_below_bigm_switch_point():
    prob = synth.problem("mlp_tiny", seed=9)
    P = nw.problems(prob)[0]
    opt = AS.Options(bigm_iters=50, as_iters=100, omega=30, max_cuts=4)
    s = AS.ActiveSet(P, opt).step(50)
    at_switch = s.bound()
    s.step(100)
    assert s.best >= at_switch
    assert max(len(s.st.slots[k]) for k in range(1, P.n)) == 4

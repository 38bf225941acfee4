"""Pins of the oracle's step rules: Adam (Kingma and Ba, as Sec. 8.1 names it), the step-size and
mask-addition schedules of Alg. 1 / Sec. 4.2.2 / Sec. 8.1, and Saddle Point's primal
initialisation (App. C.2), each against values worked out by hand or against a property that a
wrong sign, index or counter breaks."""
import numpy as np
import pytest

from oracle import active_set as AS
from oracle import dual as du
from oracle import network as nw
from oracle import relaxation as rx
from oracle import saddle as SPm
from paper_2101_05844_gb300 import synth
from tests.helpers import fig4_problem


def test_adam_steps_match_hand_computed_values():
    """Three projected ascent steps from theta = 0.2, lr = 0.01, beta1 = 0.9, beta2 = 0.999,
    eps = 1e-8, gradients 0.5, -0.3, 0.1. By hand:
      step 1: m = 0.05, v = 2.5e-4, m_hat = 0.05 / 0.1 = 0.5, v_hat = 2.5e-4 / 1e-3 = 0.25,
              theta = 0.2 + 0.01 * 0.5 / (0.5 + 1e-8) = 0.2099999998000000040
      step 2: m = 0.045 - 0.03 = 0.015, v = 2.4975e-4 + 9e-5 = 3.3975e-4,
              m_hat = 0.015 / 0.19, v_hat = 3.3975e-4 / 1.999e-3 = 0.16995997999,
              theta = 0.2119149801058224945
      step 3: m = 0.0135 + 0.01 = 0.0235, v = 3.39410250e-4 + 1e-5 = 3.4941025e-4,
              m_hat = 0.0235 / 0.271, v_hat = 3.4941025e-4 / 2.997001e-3 = 0.11658663110,
              theta = 0.2144546319383631747
    Planted mistakes (no bias correction, the moments' weights swapped, a descent sign) move
    step 1 or step 2 by more than 1e-4."""
    opt = AS.Options()
    th, m, v = np.array([0.2]), np.zeros(1), np.zeros(1)
    want_m = [0.05, 0.015, 0.0235]
    want_v = [2.5e-4, 3.3975e-4, 3.4941025e-4]
    want_th = [0.2099999998000000040, 0.2119149801058224945, 0.2144546319383631747]
    for step, g in enumerate((0.5, -0.3, 0.1), start=1):
        AS.adam(th, m, v, np.array([g]), 0.01, step, opt)
        assert m[0] == pytest.approx(want_m[step - 1], rel=1e-13)
        assert v[0] == pytest.approx(want_v[step - 1], rel=1e-13)
        assert th[0] == pytest.approx(want_th[step - 1], rel=1e-13, abs=1e-15)


def test_adam_projection_clips_at_zero_and_constant_gradients_move_by_lr():
    """The projection of Alg. 1 keeps duals nonnegative; with bias correction, a constant gradient
    gives steps of exactly lr (up to eps) at every step count, the first one included."""
    opt = AS.Options()
    th, m, v = np.array([0.001]), np.zeros(1), np.zeros(1)
    AS.adam(th, m, v, np.array([-1.0]), 0.01, 1, opt)
    assert th[0] == 0.0
    th, m, v = np.array([0.0, 0.5]), np.zeros(2), np.zeros(2)
    for step in range(1, 6):
        before = th.copy()
        AS.adam(th, m, v, np.array([2.0, -0.25]), 0.01, step, opt)
        np.testing.assert_allclose(th - before, [0.01, -0.01], rtol=1e-7)


def test_linear_step_size_schedule_values():
    """Sec. 8.1's linear decrease from lr_0 at the first planned iteration to lr_1 at the last."""
    assert [AS.linear_lr(1e-2, 1e-4, t, 5) for t in range(5)] == pytest.approx(
        [1e-2, 7.525e-3, 5.05e-3, 2.575e-3, 1e-4], rel=1e-14)
    assert AS.linear_lr(1e-3, 1e-6, 0, 1) == 1e-3
    assert AS.linear_lr(1e-3, 1e-6, 399, 400) == pytest.approx(1e-6, rel=1e-12)


@pytest.mark.parametrize("omega,cap,want", [
    # omega = 3, 2 masks per addition (Sec. 8.1), additions at t = 0, 1, 3, 4, 6, 7, 9, ...
    (3, 1, {0: 0}),
    (3, 2, {0: 0, 1: 1}),
    (3, 3, {0: 0, 1: 1, 3: 2}),
    (3, 5, {0: 0, 1: 1, 3: 2, 4: 3, 6: 4}),
    (3, 7, {0: 0, 1: 1, 3: 2, 4: 3, 6: 4, 7: 5, 9: 6}),
    # omega = 450 (the paper's value), cap 7 (the paper's)
    (450, 7, {0: 0, 1: 1, 450: 2, 451: 3, 900: 4, 901: 5, 1350: 6}),
    (450, 4, {0: 0, 1: 1, 450: 2, 451: 3}),
])
def test_mask_addition_schedule_tables(omega, cap, want):
    """Slot added at each Active Set iteration t (Alg. 1 with Sec. 4.2.2's frequency): every
    omega iterations two masks, one per iteration, until the cap; -1 elsewhere."""
    opt = AS.Options(omega=omega, vars_per_add=2, max_cuts=cap)
    got = {t: AS.addition_slot(t, opt, cap) for t in range(3 * omega + 2 if omega < 100 else 1400)}
    assert {t: b for t, b in got.items() if b >= 0} == want


def test_new_slot_takes_a_bias_corrected_first_step_of_its_own():
    """A mask added at Active Set iteration t starts at zero with zero moments and its own step
    count: its first step is Adam's bias-corrected first step, lr_t sign(g), whatever the global
    iteration (a shared counter would shrink it by a factor of about 0.48 here). alpha, beta_0,
    beta_1 keep their moments across the Big-M -> Active Set switch (their first Active Set step
    is not lr-sized in general)."""
    prob = synth.problem("mlp_tiny", seed=3)
    P = nw.problems(prob)[0]
    opt = AS.Options(bigm_iters=6, as_iters=12, omega=4, max_cuts=3)
    s = AS.ActiveSet(P, opt).step(6 + 4)            # next: Active Set iteration t = 4 adds slot 2
    _, f, g, x, z = du.evaluate(P, s.st)
    gnew = []
    for k in range(1, P.n):
        I = rx.mask(P.W[k], P.lo[k - 1], P.hi[k - 1], x[k - 1], z[k])
        lam, mu = rx.row_sums(P.W[k], P.lo[k - 1], P.hi[k - 1], I)
        gnew.append(x[k] - (P.W[k] * I) @ x[k - 1] + lam * (1 - z[k]) - z[k] * (P.b[k] + mu))
    s.step(1)
    lr = AS.linear_lr(opt.as_lr0, opt.as_lr1, 4, opt.as_iters)
    for k in range(1, P.n):
        sl = s.st.slots[k][2]
        assert sl.added_at == 4
        gk = gnew[k - 1]
        want = np.maximum(lr * gk / (np.abs(gk) + opt.adam_eps), 0.0)
        np.testing.assert_allclose(sl.beta, want, rtol=1e-9, atol=1e-15)
        assert (sl.beta[np.abs(gk) > 1e-6] > 0).any() or (gk <= 0).all()


def _restricted_primal_view(P, x, z, mu_a, mu_b):
    """App. C.2's primal view with the duals restricted to Big-M (E_k empty): the max over
    alpha in [0, mu_alpha] and beta_0, beta_1 >= 0 with beta_0 + beta_1 <= mu_beta of the bilinear
    objective, i.e. W_n x_{n-1} + b_n + sum mu_alpha (xhat - x)_+ + mu_beta max(0, x - z uhat,
    x - xhat + (1 - z) lhat)."""
    val = float((P.W[P.n] @ x[P.n - 1] + P.b[P.n])[0])
    for k in range(1, P.n):
        xhat = P.W[k] @ x[k - 1] + P.b[k]
        val += float(mu_a[k] @ np.maximum(xhat - x[k], 0.0))
        v0 = x[k] - z[k] * P.uhat[k]
        v1 = x[k] - xhat + (1 - z[k]) * P.lhat[k]
        val += float(mu_b[k] @ np.maximum(0.0, np.maximum(v0, v1)))
    return val


def test_primal_initialisation_step_descends_the_restricted_primal_view():
    """App. C.2: one projected subgradient step of the primal initialisation lowers the Big-M
    restricted primal view on the Fig. 4 network (App. F.1), from interior points where the view is
    linear nearby; the opposite move raises it, so a flipped sign of the step (ascent instead of
    descent, or -f taken for the subgradient in x) fails."""
    P, _ = fig4_problem()
    rng = synth.SplitMix64(4)
    checked = 0
    for trial in range(30):
        x = [P.lo[k] + (0.2 + 0.6 * rng.uniform(P.widths[k])) * (P.hi[k] - P.lo[k]) for k in range(P.n)]
        z = [None] + [0.2 + 0.6 * rng.uniform(P.widths[k]) for k in range(1, P.n)]
        mu_a = [None] + [0.1 + rng.uniform(P.widths[k]) for k in range(1, P.n)]
        mu_b = [None] + [0.1 + rng.uniform(P.widths[k]) for k in range(1, P.n)]
        # stay away from the kinks of the view: every max() decided by more than 1e-3
        ok = True
        for k in range(1, P.n):
            xhat = P.W[k] @ x[k - 1] + P.b[k]
            v0, v1 = x[k] - z[k] * P.uhat[k], x[k] - xhat + (1 - z[k]) * P.lhat[k]
            gaps = np.concatenate([np.abs(xhat - x[k]), np.abs(v0 - v1), np.abs(np.maximum(v0, v1))])
            ok &= bool(gaps.min() > 1e-3)
        if not ok:
            continue
        opt = AS.Options(sp_init_steps=1, sp_init_lr0=1e-5, sp_init_lr1=1e-5)
        sp = SPm.SaddlePoint.from_state(P, opt, [None] + [np.zeros(P.widths[k]) for k in range(1, P.n)],
                                        [None] + [np.zeros(P.widths[k]) for k in range(1, P.n)],
                                        [None] + [np.zeros(P.widths[k - 1]) for k in range(1, P.n)],
                                        [None] + [np.zeros(P.widths[k]) for k in range(1, P.n)],
                                        [None] + [np.zeros(P.widths[k]) for k in range(1, P.n)],
                                        mu_a, mu_b, x, z, 0)
        before = _restricted_primal_view(P, x, z, mu_a, mu_b)
        sp._primal_init()
        after = _restricted_primal_view(P, sp.x, sp.z, mu_a, mu_b)
        back_x = [2 * a - b for a, b in zip(x, sp.x)]
        back_z = [None] + [2 * z[k] - sp.z[k] for k in range(1, P.n)]
        against = _restricted_primal_view(P, back_x, back_z, mu_a, mu_b)
        moved = sum(float(np.abs(a - b).sum()) for a, b in zip(x, sp.x))
        assert moved > 0
        assert after < before - 1e-12
        assert against > before + 1e-12
        checked += 1
    assert checked >= 5

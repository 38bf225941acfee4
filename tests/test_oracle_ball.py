"""Pins of the ellipsoid (l2-ball) input set in the oracle (Sec. 2: any input set with a closed-form
linear minimisation): the exact range of layer 1, a closed-form minimum on an affine region,
weak duality against sampled inputs, and the box LP below the ball's bound."""
import numpy as np
import pytest

from oracle import active_set as AS
from oracle import bab
from oracle import dual as du
from oracle import lp
from oracle import network as nw
from oracle import relaxation as rx
from paper_2101_05844_gb300 import synth


def _ellipsoid_points(lo, hi, n, seed):
    """n points uniform in the ellipsoid inscribed in [lo, hi]."""
    rng = synth.SplitMix64(seed)
    d = lo.size
    g = rng.normal(n * d).reshape(n, d)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = rng.uniform(n) ** (1.0 / d)
    c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
    return c[None, :] + e[None, :] * g * r[:, None]


def _ball_prob(name, seed, S=1, scale=1.0, equal=False):
    prob = synth.problem(name, S=S, seed=seed)
    lo, hi = prob["lo"].astype(np.float64), prob["hi"].astype(np.float64)
    c = 0.5 * (lo + hi)
    e = 0.5 * (hi - lo) * scale
    if not equal:   # unequal half-widths: an ellipsoid
        e = e * (0.5 + synth.SplitMix64(seed + 7).uniform(e.size).reshape(e.shape))
    return dict(prob, lo=(c - e).astype(np.float32), hi=(c + e).astype(np.float32), ball=True)


def test_layer1_interval_is_the_exact_range_over_the_ellipsoid():
    prob = _ball_prob("mlp_5_7_6_3", 1)
    lo, hi = prob["lo"][0].astype(np.float64), prob["hi"][0].astype(np.float64)
    W, b, _ = nw.dense_layers(prob["net"])[0]
    lh, uh, _, _ = nw.ibp([W], [b], lo, hi, ball=True)
    c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
    for i in range(W.shape[0]):
        d = e * e * W[i] / np.linalg.norm(e * W[i])
        for x, v in ((c + d, uh[1][i]), (c - d, lh[1][i])):
            assert np.sum(((x - c) / e) ** 2) == pytest.approx(1.0, abs=1e-12)   # on the surface
            assert W[i] @ x + b[i] == pytest.approx(v, abs=1e-12)                  # attains the bound
    X = _ellipsoid_points(lo, hi, 4000, 3)
    A = X @ W.T + b[None, :]
    assert np.all(A >= lh[1][None, :] - 1e-12) and np.all(A <= uh[1][None, :] + 1e-12)
    box_l, box_u, _, _ = nw.ibp([W], [b], lo, hi)
    assert np.all(lh[1] >= box_l[1] - 1e-12) and np.all(uh[1] <= box_u[1] + 1e-12)


def test_interior_inputs_give_masks_equal_to_z():
    """Eq. (3) at a binary z and inputs strictly inside their box: the bit is z (1 where W = 0)."""
    rng = synth.SplitMix64(5)
    W = rng.normal(6 * 5).reshape(6, 5)
    W[0, 0] = 0.0
    lo, hi = -np.ones(5), np.ones(5)
    x = 0.9 * (rng.uniform(5) * 2 - 1)
    z = (rng.uniform(6) < 0.5).astype(np.float64)
    I = rx.mask(W, lo, hi, x, z)
    np.testing.assert_array_equal(I, rx.mask_exact(W, lo, hi, x, z))
    expect = np.repeat(z[:, None] > 0, 5, axis=1) | (W == 0)
    np.testing.assert_array_equal(I, expect)


def test_affine_region_reaches_the_closed_form_minimum():
    """A small ellipsoid on which no neuron is ambiguous: f is affine there, f(x) = a . x + f0, and
    its minimum is f(c) - |D a|_2. Converged Big-M duals reach it from below."""
    prob = _ball_prob("mlp_4_3_3_1", 2, scale=0.05)
    P = nw.problems(prob)[0]
    for k in range(1, P.n):
        assert not np.any((P.lhat[k] < 0) & (P.uhat[k] > 0))
    dense = nw.dense_layers(prob["net"])
    lo, hi = P.lo[0], P.hi[0]
    c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
    A = np.eye(lo.size)
    a0 = np.zeros(lo.size)
    h0 = c.copy()
    for W, b, _ in dense[:-1]:   # the active pattern at the centre holds on the whole ellipsoid
        act = (W @ h0 + b) > 0
        A, a0, h0 = act[:, None] * (W @ A), act * (W @ a0 + b), np.maximum(W @ h0 + b, 0.0)
    Wn, bn, _ = dense[-1]
    a = prob["C"][0] @ Wn @ A
    f_c = float(prob["C"][0] @ (Wn @ h0 + bn))
    exact = f_c - float(np.linalg.norm(e * a))
    X = _ellipsoid_points(lo, hi, 3000, 9)
    vals = [float(prob["C"][0] @ bab.forward(dense, x)) for x in X]
    assert min(vals) >= exact - 1e-12 and min(vals) <= exact + 0.05 * (max(vals) - min(vals))
    _, best, _ = AS.solve(P, AS.Options(bigm_iters=3000))
    assert exact - 1e-4 <= best <= exact + 1e-9


@pytest.mark.parametrize("name,seed", [("mlp_5_7_6_3", 1), ("small_conv", 2)])
def test_bounds_are_below_every_sampled_input(name, seed):
    prob = _ball_prob(name, seed)
    P = nw.problems(prob)[0]
    s = AS.ActiveSet(P, AS.Options(bigm_iters=60, as_iters=60, omega=15, max_cuts=3)).step(120)
    x0 = du.evaluate(P, s.st)[3][0]
    c, e = 0.5 * (P.lo[0] + P.hi[0]), 0.5 * (P.hi[0] - P.lo[0])
    assert np.sum(((x0 - c) / e) ** 2) == pytest.approx(1.0, abs=1e-9)   # x_0* on the surface
    dense = nw.dense_layers(prob["net"])
    X = _ellipsoid_points(P.lo[0], P.hi[0], 3000, seed)

    m = min(float(prob["C"][0] @ bab.forward(dense, x)) for x in X)
    assert s.best <= m + 1e-9
    assert s.best >= P.ibp_output_bound() - 1e-9


def test_ball_bound_is_above_the_box_lp():
    """With equal half-widths the ball lies inside the box, so its relaxation lies inside the box's:
    converged Big-M over the ball ends above the exact LP(M) over the box, and below the sampled
    minimum over the ball."""
    prob = _ball_prob("mlp_4_3_3_1", 3, equal=True)
    P = nw.problems(prob)[0]
    box = nw.problems(dict(prob, ball=False))[0]
    v_box = float(lp.NetLP(box.W[1:box.n], box.b[1:box.n], box.lhat, box.uhat, box.lo, box.hi)
                  .solve("M", box.W[box.n][0], box.b[box.n][0]))
    _, best, _ = AS.solve(P, AS.Options(bigm_iters=2000))
    assert best >= v_box - 1e-4
    dense = nw.dense_layers(prob["net"])
    X = _ellipsoid_points(P.lo[0], P.hi[0], 4000, 4)
    assert best <= min(float(bab.forward(dense, x)[0]) for x in X) + 1e-9


def test_intermediate_bounds_over_the_ellipsoid():
    """App. E's staged solves over the ellipsoid: zero iterations give its interval propagation;
    solves tighten it and still contain the pre-activations of sampled inputs."""
    from oracle import intermediate as IM
    prob = _ball_prob("mlp_4_3_3_3_1", 2)
    lo, hi = prob["lo"][0].astype(np.float64), prob["hi"][0].astype(np.float64)
    dense = nw.dense_layers(prob["net"])
    Ws, bs = [d[0] for d in dense[:-1]], [d[1] for d in dense[:-1]]
    il, iu, _, _ = nw.ibp(Ws, bs, lo, hi, ball=True)
    l0, u0 = IM.intermediate_bounds(prob["net"], lo, hi, AS.Options(), dense=dense, ball=True)
    for k in range(1, len(l0)):
        np.testing.assert_allclose(l0[k], il[k], atol=1e-12)
        np.testing.assert_allclose(u0[k], iu[k], atol=1e-12)
    lh, uh = IM.intermediate_bounds(prob["net"], lo, hi, AS.Options(bigm_iters=200), dense=dense, ball=True)
    X = _ellipsoid_points(lo, hi, 3000, 6)
    h = X.T
    gain = 0.0
    for k, (W, b) in enumerate(zip(Ws, bs), start=1):
        a = W @ h + b[:, None]
        assert np.all(a.min(axis=1) >= lh[k] - 1e-9) and np.all(a.max(axis=1) <= uh[k] + 1e-9)
        gain += np.sum(iu[k] - il[k]) - np.sum(uh[k] - lh[k])
        h = np.maximum(a, 0.0)
    assert gain > 0


@pytest.mark.parametrize("seed,verdict", [(4, "verified"), (4, "falsified"), (7, "verified")])
def test_branch_and_bound_over_the_ellipsoid(seed, verdict):
    """The property f(x) - t > 0 over the ellipsoid, t below every sampled value by a tenth of the
    sampled range (verified), or midway through the sampled range (falsified, the point found lies
    in the ellipsoid and has a negative value)."""
    prob = _ball_prob("mlp_4_5_5_1", seed)
    lo, hi = prob["lo"][0].astype(np.float64), prob["hi"][0].astype(np.float64)
    dense = nw.dense_layers(prob["net"])
    vals = np.array([bab.forward(dense, x)[0] for x in _ellipsoid_points(lo, hi, 4000, seed)])
    t = vals.min() - 0.1 * np.ptp(vals) if verdict == "verified" else 0.5 * (vals.min() + vals.max())
    net = [dict(L) for L in prob["net"]]
    net[-1]["b"] = (net[-1]["b"].astype(np.float64) - t).astype(np.float32)
    opt = bab.BabOptions(loose=AS.Options(bigm_iters=100),
                         tight=AS.Options(bigm_iters=50, as_iters=100, omega=30, max_cuts=3),
                         batch=8, max_domains=600)
    res = bab.BaB(net, lo, hi, np.ones(1), opt, ball=True).run()
    assert res["status"] == verdict
    if verdict == "falsified":
        x = res["x"]
        c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
        assert np.sum(((x - c) / e) ** 2) <= 1 + 1e-9
        assert bab.forward(nw.dense_layers(net), x)[0] < 0
    else:
        vals_t = np.array([bab.forward(nw.dense_layers(net), x)[0] for x in _ellipsoid_points(lo, hi, 2000, 1)])
        assert 0 < res["lower"] <= vals_t.min()


@pytest.mark.parametrize("name,seed", [("mlp_5_7_6_3", 1), ("small_conv", 2)])
def test_saddle_point_over_the_ellipsoid(name, seed):
    """Saddle Point from Active Set duals over the ellipsoid: the primal iterate stays inside it
    (its start is retracted, then convex combinations of points inside), x_bar_0 lies on its
    surface, and every bound lies below the sampled minimum."""
    from oracle import saddle as SPm
    prob = _ball_prob(name, seed)
    P = nw.problems(prob)[0]
    opt = AS.Options(bigm_iters=40, as_iters=40, omega=10, max_cuts=3, sp_init_steps=20)
    s = AS.ActiveSet(P, opt).step(80)
    sp = SPm.SaddlePoint(P, opt, s.st)
    c, e = 0.5 * (P.lo[0] + P.hi[0]), 0.5 * (P.hi[0] - P.lo[0])
    dense = nw.dense_layers(prob["net"])
    m = min(float(prob["C"][0] @ bab.forward(dense, x)) for x in _ellipsoid_points(P.lo[0], P.hi[0], 3000, 2))
    for _ in range(30):
        assert np.sum(((sp.x[0] - c) / e) ** 2) <= 1 + 1e-9
        val, xb, _ = sp.evaluate()
        assert np.sum(((xb[0] - c) / e) ** 2) == pytest.approx(1.0, abs=1e-9)
        assert val <= m + 1e-9
        sp.step(1)


def test_saddle_point_approaches_the_affine_closed_form():
    """On the small ellipsoid where the network is affine (see above), Saddle Point from Big-M duals
    climbs towards the closed-form minimum f(c) - |D a|_2 and never passes it."""
    from oracle import saddle as SPm
    prob = _ball_prob("mlp_4_3_3_1", 2, scale=0.05)
    P = nw.problems(prob)[0]
    dense = nw.dense_layers(prob["net"])
    lo, hi = P.lo[0], P.hi[0]
    c, e = 0.5 * (lo + hi), 0.5 * (hi - lo)
    A, h0 = np.eye(lo.size), c.copy()
    for W, b, _ in dense[:-1]:
        act = (W @ h0 + b) > 0
        A, h0 = act[:, None] * (W @ A), np.maximum(W @ h0 + b, 0.0)
    a = prob["C"][0] @ dense[-1][0] @ A
    exact = float(prob["C"][0] @ (dense[-1][0] @ h0 + dense[-1][1])) - float(np.linalg.norm(e * a))
    opt = AS.Options(bigm_iters=200, sp_init_steps=20)
    s = AS.ActiveSet(P, opt).step(200)
    sp = SPm.SaddlePoint(P, opt, s.st)
    start = sp.bound()
    sp.step(400)
    assert sp.best <= exact + 1e-9
    assert sp.best >= start - 1e-12
    assert exact - sp.best < 0.5 * (exact - start) or exact - sp.best < 1e-4


def _fd_bound(P, st, mod, chain, splits=None):
    """The bound at fixed duals and masks after mod(Q): intermediate bounds held (chain False) or
    redone by interval propagation over the (perturbed) ellipsoid (chain True)."""
    Q = nw.Problem.__new__(nw.Problem)
    Q.__dict__.update(P.__dict__)
    Q.W = [None if w is None else w.copy() for w in P.W]
    Q.b = [None if w is None else w.copy() for w in P.b]
    Q.lo = [v.copy() for v in P.lo]
    Q.hi = [v.copy() for v in P.hi]
    mod(Q)
    if chain:
        lh, uh, lo, hi = nw.ibp(Q.W[1:Q.n], Q.b[1:Q.n], Q.lo[0], Q.hi[0], splits, ball=True)
        Q.lhat, Q.uhat, Q.lo, Q.hi = lh, uh, lo, hi
    st2 = du.DualState(st.alpha, st.beta0, st.beta1, [[] for _ in range(P.n)])
    for k in range(1, P.n):
        for sl in st.slots[k]:
            du.add_slot(Q, st2, k, sl.I, beta=sl.beta)
    return du.evaluate(Q, st2)[0]


@pytest.mark.parametrize("name,chain", [("mlp_4_5_5_1", False), ("mlp_4_5_5_1", True), ("small_conv", False),
                                        ("small_conv", True)])
def test_input_gradients_over_the_ellipsoid_match_finite_differences(name, chain):
    """The envelope gradient over the ellipsoid (its endpoints parameterise c and e), with the
    intermediate bounds held or carried through interval propagation (layer 1 over the
    ellipsoid), against central differences; it differs from the box formula."""
    from oracle import envelope as ev
    prob = _ball_prob(name, 4)
    P = nw.problems(prob)[0]
    s = AS.ActiveSet(P, AS.Options(bigm_iters=30, as_iters=30, omega=10, max_cuts=3)).step(60)
    g = ev.chain_gradient(P, s.st) if chain else ev.envelope_gradient(P, s.st)
    h = 1e-6
    rng = synth.SplitMix64(3)

    def fd(mod):
        return (_fd_bound(P, s.st, lambda Q: mod(Q, h), chain) - _fd_bound(P, s.st, lambda Q: mod(Q, -h), chain)) / (2 * h)
    for j in range(min(6, P.widths[0])):
        def ml(Q, d):
            Q.lo[0][j] += d

        def mh(Q, d):
            Q.hi[0][j] += d
        assert fd(ml) == pytest.approx(g["dlo0"][j], rel=1e-5, abs=1e-7)
        assert fd(mh) == pytest.approx(g["dhi0"][j], rel=1e-5, abs=1e-7)
    for k in range(1, P.n + 1):
        for _ in range(4):
            i = int(rng.integers(1, 0, P.W[k].shape[0] - 1)[0])
            j = int(rng.integers(1, 0, P.W[k].shape[1] - 1)[0])
            if abs(P.W[k][i, j]) < 10 * h:
                continue

            def mw(Q, d):
                Q.W[k][i, j] += d
            assert fd(mw) == pytest.approx(g["dW"][k][i, j], rel=1e-5, abs=1e-7)
    P.ball = False
    try:
        gb = ev.envelope_gradient(P, s.st)
    finally:
        P.ball = True
    assert np.abs(gb["dlo0"] - g["dlo0"]).max() > 1e-4

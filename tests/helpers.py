"""Shared test fixtures: build oracle problems from the synthetic generator."""
import math
from itertools import product

import numpy as np

from oracle import lp
from oracle import network as nw
from paper_2101_05844_gb300 import synth


def fig4_problem(kind="M"):
    """The Fig. 4 network of App. F.1 as an oracle Problem, intermediate bounds by LPs."""
    Ws, bs, w3, b3, lo0, hi0 = lp.fig4_network()
    lh, uh, lo, hi = lp.layer_bounds_lp(Ws, bs, lo0, hi0, kind)
    net = fig4_net()
    P = nw.Problem(net, lo0, hi0, np.ones(1), bounds=(lh[1:], uh[1:]))
    return P, (Ws, bs, w3, b3, lh, uh, lo, hi)


def fig4_net():
    Ws, bs, w3, b3, lo0, hi0 = lp.fig4_network()
    return [{"kind": "linear", "n_in": 2, "n_out": 2, "W": Ws[0].astype(np.float32),
             "b": bs[0].astype(np.float32)},
            {"kind": "linear", "n_in": 2, "n_out": 2, "W": Ws[1].astype(np.float32),
             "b": bs[1].astype(np.float32)},
            {"kind": "linear", "n_in": 2, "n_out": 1, "W": w3[None].astype(np.float32),
             "b": np.zeros(1, np.float32)}]


def netlp_for(P):
    """NetLP over the hidden layers of an oracle Problem, with its bounds."""
    return lp.NetLP(P.W[1:P.n], P.b[1:P.n], P.lhat, P.uhat, P.lo, P.hi)


def sample_min_output(P, n_samples, seed=0):
    """Minimum of the network output row over random points and all vertices of the box."""
    from paper_2101_05844_gb300.synth import SplitMix64
    rng = SplitMix64(seed)
    n0 = P.widths[0]
    X = P.lo[0][None, :] + rng.uniform(n_samples * n0).reshape(n_samples, n0) * (P.hi[0] - P.lo[0])[None, :]
    if n0 <= 14:
        V = np.array(np.meshgrid(*[[0, 1]] * n0)).reshape(n0, -1).T
        X = np.vstack([X, np.where(V == 1, P.hi[0], P.lo[0])])
    h = X.T
    for k in range(1, P.n):
        h = np.maximum(P.W[k] @ h + P.b[k][:, None], 0.0)
    out = P.W[P.n] @ h + P.b[P.n][:, None]
    return float(out.min())


def exact_min(net, lo, hi, crow):
    """min over the box of crow . f(x): every activation pattern's region is a polytope on which
    f is affine; the minimum is the least of the regions' LP minima."""
    dense = nw.dense_layers(net)
    hidden = dense[:-1]
    Wn, bn, _ = dense[-1]
    NH = sum(W.shape[0] for W, _, _ in hidden)
    n0 = len(lo)
    best = math.inf
    for pat in product((0, 1), repeat=NH):
        A, a = np.eye(n0), np.zeros(n0)
        rows, rhs, off = [], [], 0
        for W, b, _ in hidden:
            Ah, ah = W @ A, W @ a + b
            D = np.array(pat[off:off + W.shape[0]], np.float64)
            for i in range(W.shape[0]):
                if D[i]:   # xhat >= 0
                    rows.append(-Ah[i])
                    rhs.append(ah[i])
                else:      # xhat <= 0
                    rows.append(Ah[i])
                    rhs.append(-ah[i])
            A, a = D[:, None] * Ah, D * ah
            off += W.shape[0]
        obj = crow @ Wn @ A
        val, _ = lp.simplex_min(list(obj), [list(r) for r in rows], rhs, list(lo), list(hi))
        if val is not None:
            best = min(best, float(val) + float(crow @ (Wn @ a + bn)))
    return best


def shifted(net, t):
    """The same network with t subtracted from its (single) output."""
    net = [dict(L) for L in net]
    net[-1]["b"] = (net[-1]["b"].astype(np.float64) - t).astype(np.float32)
    return net


def net_with_shifted_output(name, seed, margin):
    """(net shifted so that the property is f(x) - t > 0, box, exact minimum of the shifted net);
    t = m + margin (M - m) with m, M the exact minimum and maximum of f over the box."""
    prob = synth.problem(name, S=1, seed=seed)
    lo, hi = prob["lo"][0], prob["hi"][0]
    ones = np.ones(1)
    m = exact_min(prob["net"], lo, hi, ones)
    M = -exact_min(prob["net"], lo, hi, -ones)
    net = shifted(prob["net"], m + margin * (M - m))
    return net, lo, hi, exact_min(net, lo, hi, ones)

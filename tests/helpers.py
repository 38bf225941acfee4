"""Shared test fixtures: build oracle problems from the synthetic generator."""
import numpy as np

from oracle import lp
from oracle import network as nw


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

"""Intermediate bounds by dual solves over sub-networks (App. E) (oracle; test infrastructure only).

App. E obtains the pre-activation bounds of hidden layer i by solving, for each neuron j, the
problem min x_hat_i[j] over the network truncated after layer i, with the ReLU relaxation C_k on
layers k = 1 .. i-1 (and the same with the sign of layer i's row flipped for the upper bound).
Here C_k is the relaxation the Big-M / Active Set solver (Alg. 1) bounds: each of these
problems is the sub-network of layers 1 .. i with the property row +e_j (lower bound) or -e_j
(the negated upper bound), solved for T_M + T_A iterations, its final iterate's dual value
taken. Layers are processed in order, each with the bounds already obtained for the layers
before it (App. E: the bounds of layer i enter C_k of every later layer).

Readings where App. E leaves the procedure open:
  * layer 1 keeps its interval bounds: over a box they are the exact range of an affine map;
  * every layer's result is intersected with interval propagation (App. E keeps the tighter of
    two methods' bounds; both are valid, so their intersection is);
  * splits (+1 active, -1 inactive) enter through interval propagation, which clamps lhat to 0 /
    uhat to 0 of a split neuron whose interval straddles zero; a tightened interval lies inside
    the clamped one, so it never straddles zero again and needs no second clamp;
  * if rounding leaves lhat > uhat, both take their midpoint.
"""
from __future__ import annotations

import numpy as np

from . import active_set as AS
from . import network as nw


def intermediate_bounds(net: list, lo0, hi0, opt: AS.Options, splits=None, dense=None, ball=False):
    """1-based lists (lhat, uhat) of every hidden layer's pre-activation bounds for one box.

    net: layer dicts of the whole network (the last layer linear); lo0, hi0: the input box;
    opt: the iteration schedule of each sub-network solve; splits: int8 over the hidden neurons,
    layer-major, or None; ball: the input set is the ellipsoid inscribed in the box.
    """
    dense = dense if dense is not None else nw.dense_layers(net)
    n = len(net)
    Ws = [d[0] for d in dense[:-1]]
    bs = [d[1] for d in dense[:-1]]
    lhat, uhat, _, _ = nw.ibp(Ws, bs, lo0, hi0, splits, ball)
    lhat = [None] + [v.copy() for v in lhat[1:]]
    uhat = [None] + [v.copy() for v in uhat[1:]]
    for k in range(2, n):
        nk = Ws[k - 1].shape[0]
        sub, dsub = net[:k], dense[:k]
        bounds = (lhat[1:k], uhat[1:k])
        for i in range(nk):
            vals = []
            for sign in (1.0, -1.0):
                crow = np.zeros(nk)
                crow[i] = sign
                P = nw.Problem(sub, lo0, hi0, crow, bounds=bounds, dense=dsub, ball=ball)
                final, _, _ = AS.solve(P, opt)
                vals.append(final)
            l = max(lhat[k][i], vals[0])
            u = min(uhat[k][i], -vals[1])
            if l > u:
                l = u = 0.5 * (l + u)
            lhat[k][i], uhat[k][i] = l, u
    return lhat, uhat


def batch(prob: dict, opt: AS.Options):
    """intermediate_bounds of every box of a synthetic problem dict: float64 [S][NH] (lhat, uhat)."""
    dense = nw.dense_layers(prob["net"])
    L, U = [], []
    for s in range(prob["lo"].shape[0]):
        sp = None if prob.get("splits") is None else prob["splits"][s]
        lh, uh = intermediate_bounds(prob["net"], prob["lo"][s], prob["hi"][s], opt, sp, dense,
                                     bool(prob.get("ball", False)))
        L.append(np.concatenate(lh[1:]))
        U.append(np.concatenate(uh[1:]))
    return np.array(L), np.array(U)

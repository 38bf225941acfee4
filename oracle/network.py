"""Dense linear operators and interval bound propagation (oracle; test infrastructure only).

The paper writes every layer, convolutional ones included, as its equivalent linear operator
(Sec. 2, "W_k, b_k"; App. G opens with the same convention). This module builds those dense
matrices entry by entry from the definition of a 2-D convolution with zero padding.
"""
from __future__ import annotations

import numpy as np


def conv_dense(L: dict):
    """Dense matrix of a conv layer and, for each nonzero entry, its filter index.

    Returns (W [n_out, n_in] float64, b [n_out] float64, taps) where taps is a list of
    (row, col, filter_flat_index) for every (output, input) pair the filter connects.
    Output neuron (co, oy, ox) reads input (ci, oy*stride - pad + ky, ox*stride - pad + kx).
    """
    c, h, w = L["in_shape"]
    oc, oh, ow = L["out_shape"]
    kh, kw, st, pd = L["kh"], L["kw"], L["stride"], L["pad"]
    F = L["W"].astype(np.float64)
    W = np.zeros((oc * oh * ow, c * h * w))
    taps = []
    for co in range(oc):
        for oy in range(oh):
            for ox in range(ow):
                row = (co * oh + oy) * ow + ox
                for ci in range(c):
                    for ky in range(kh):
                        y = oy * st - pd + ky
                        if y < 0 or y >= h:
                            continue
                        for kx in range(kw):
                            x = ox * st - pd + kx
                            if x < 0 or x >= w:
                                continue
                            col = (ci * h + y) * w + x
                            W[row, col] = F[co, ci, ky, kx]
                            taps.append((row, col, ((co * c + ci) * kh + ky) * kw + kx))
    b = np.repeat(L["b"].astype(np.float64), oh * ow)
    return W, b, taps


def dense_layers(net: list[dict]):
    """[(W_k, b_k, taps_k)] for k = 1..n, dense float64 (taps is None for linear layers)."""
    out = []
    for L in net:
        if L["kind"] == "linear":
            out.append((L["W"].astype(np.float64), L["b"].astype(np.float64), None))
        else:
            out.append(conv_dense(L))
    return out


def ibp(Ws: list, bs: list, lo0: np.ndarray, hi0: np.ndarray, splits=None, ball=False):
    """Interval bound propagation (Gowal et al.; App. E of the paper, last paragraph).

    Ws, bs are the hidden layers' dense operators (k = 1..n-1). Returns (lhat, uhat, lo, hi) as
    1-based lists: lhat[k], uhat[k] pre-activation bounds for k = 1..n-1; lo[k], hi[k]
    post-activation bounds lo = max(lhat, 0), hi = max(uhat, 0), with lo[0], hi[0] the input box.

    splits (int8 over all hidden neurons, layer-major) clamps a neuron whose interval straddles
    zero: +1 (active) sets lhat = 0, -1 (inactive) sets uhat = 0, before the next layer is
    propagated. A split on a neuron that does not straddle zero changes nothing.

    ball: the input set is the ellipsoid inscribed in the box, {x : sum_j ((x_j - c_j) / e_j)^2 <= 1}
    with c = (lo0 + hi0) / 2 and e = (hi0 - lo0) / 2 (an l2 ball of radius e when the half-widths
    are equal; Sec. 2 allows any input set with a closed-form linear minimisation). Layer 1's bounds
    are then the exact range of W_1 x + b_1 over it: W_1 c + b_1 -+ |W_1 D|_2 row by row, D = diag(e).
    """
    lo = [np.asarray(lo0, np.float64)]
    hi = [np.asarray(hi0, np.float64)]
    lhat, uhat = [None], [None]
    off = 0
    for k, (W, b) in enumerate(zip(Ws, bs)):
        if ball and k == 0:
            c = 0.5 * (lo[0] + hi[0])
            r = np.sqrt(((W * (0.5 * (hi[0] - lo[0]))[None, :]) ** 2).sum(axis=1))
            lh = W @ c + b - r
            uh = W @ c + b + r
        else:
            Wp = np.maximum(W, 0.0)
            Wn = np.minimum(W, 0.0)
            lh = Wp @ lo[-1] + Wn @ hi[-1] + b
            uh = Wp @ hi[-1] + Wn @ lo[-1] + b
        if splits is not None:
            sp = splits[off:off + W.shape[0]]
            amb = (lh < 0) & (uh > 0)
            lh = np.where(amb & (sp > 0), 0.0, lh)
            uh = np.where(amb & (sp < 0), 0.0, uh)
        off += W.shape[0]
        lhat.append(lh)
        uhat.append(uh)
        lo.append(np.maximum(lh, 0.0))
        hi.append(np.maximum(uh, 0.0))
    return lhat, uhat, lo, hi


class Problem:
    """One bounding subproblem in dense form, 1-based layer lists as in the paper.

    W[k], b[k] for k = 1..n (W[n] is the property-folded output row [1, n_{n-1}], b[n] a
    scalar array of shape [1]); lhat/uhat[k] for k = 1..n-1; lo/hi[k] for k = 0..n-1.
    """

    def __init__(self, net, lo0, hi0, crow, splits=None, bounds=None, dense=None, ball=False):
        dense = dense if dense is not None else dense_layers(net)
        self.net = net
        self.ball = ball   # x_0 in the ellipsoid inscribed in [lo0, hi0] (see ibp)
        self.taps = [None] + [d[2] for d in dense]
        self.W = [None] + [d[0] for d in dense[:-1]]
        self.b = [None] + [d[1] for d in dense[:-1]]
        Wl, bl, _ = dense[-1]
        crow = np.asarray(crow, np.float64)
        self.crow = crow
        self.W.append((crow @ Wl)[None, :])
        self.b.append(np.array([crow @ bl]))
        self.n = len(self.W) - 1
        self.widths = [len(lo0)] + [self.W[k].shape[0] for k in range(1, self.n)]
        if bounds is None:
            self.lhat, self.uhat, self.lo, self.hi = ibp(self.W[1:self.n], self.b[1:self.n],
                                                         lo0, hi0, splits, ball)
        else:
            lh, uh = bounds
            self.lhat = [None] + [np.asarray(v, np.float64) for v in lh]
            self.uhat = [None] + [np.asarray(v, np.float64) for v in uh]
            self.lo = [np.asarray(lo0, np.float64)] + [np.maximum(v, 0.0) for v in self.lhat[1:]]
            self.hi = [np.asarray(hi0, np.float64)] + [np.maximum(v, 0.0) for v in self.uhat[1:]]

    def ibp_output_bound(self) -> float:
        """Lower bound of the output row by one more interval step."""
        W, b = self.W[self.n], self.b[self.n]
        lo, hi = self.lo[self.n - 1], self.hi[self.n - 1]
        return float((np.maximum(W, 0) @ lo + np.minimum(W, 0) @ hi + b)[0])


def problems(prob: dict, bounds=None, dense=None) -> list[Problem]:
    """One Problem per subproblem of a synthetic problem dict (prob["ball"]: ellipsoid inputs)."""
    dense = dense if dense is not None else dense_layers(prob["net"])
    out = []
    S = prob["lo"].shape[0]
    for s in range(S):
        sp = None if prob.get("splits") is None else prob["splits"][s]
        bd = None if bounds is None else bounds[s]
        out.append(Problem(prob["net"], prob["lo"][s], prob["hi"][s], prob["C"][s], sp, bd, dense,
                           bool(prob.get("ball", False))))
    return out

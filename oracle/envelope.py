"""Gradient of the Active Set bound at fixed duals (oracle; test infrastructure only).

The paper does not differentiate its bounds. The quantity here is the envelope (Danskin) gradient:
d(theta) = min over (x, z) of L(x, z, alpha, beta; theta) at fixed duals alpha, beta and fixed
masks I, with the intermediate bounds lhat, uhat, l_k, u_k (k >= 1) held fixed and the signs of W
held fixed. theta is the weights and biases of every layer and the input box (l_0, u_0). Where the
minimiser is unique, dd/dtheta = dL/dtheta at (x*, z*), using the constraint form of L (App. D):
  dW_k[i, j] = (alpha - beta_1)[i] x_{k-1}[j]
               + sum_I beta_I[i] ( I[i,j] ((1 - z[i]) Lcheck[i,j] - x_{k-1}[j])
                                   - z[i] (1 - I[i,j]) Ucheck[i,j] )
  db_k[i]    = (alpha - beta_1)[i] - sum_I beta_I[i] z[i]
  dW_n       = x_{n-1}*,  db_n = 1           (the property-folded output row)
  dl_0[j]    = -f_0[j] [x_0*[j] = l_0[j]] + sum_i sum_I beta_I[i] ( (1 - z[i]) W I [W >= 0]
                                                                  - z[i] W (1 - I) [W < 0] )[i, j]
  du_0[j]    = -f_0[j] [x_0*[j] = u_0[j]] + sum_i sum_I beta_I[i] ( (1 - z[i]) W I [W < 0]
                                                                  - z[i] W (1 - I) [W >= 0] )[i, j]
(the last terms come from Lcheck and Ucheck of layer 1, which are built from l_0 and u_0).
chain_gradient below also lets the intermediate bounds follow theta through interval propagation.
Parity unpinned against the paper (it has no such gradient); pinned by finite differences.
"""
from __future__ import annotations

import numpy as np

from . import dual as du
from . import relaxation as rx


def _x0_box_terms(P, f0, x0):
    """d/dl_0, d/du_0 of the x_0 part of the bound, min over the input set of -f_0^T x_0. Box: x_0*
    at an end of its interval (half to each end where l = u). Ellipsoid inscribed in the box
    (P.ball), centre c = (l + u) / 2, half-widths e = (u - l) / 2: the value -f c - |e f|_2 gives
    -f / 2 -+ e f^2 / (2 |e f|) (the norm's subgradient 0 where e f = 0)."""
    if getattr(P, "ball", False):
        e = 0.5 * (P.hi[0] - P.lo[0])
        nrm = float(np.sqrt(((e * f0) ** 2).sum()))
        d = e * f0 * f0 / (2.0 * nrm) if nrm > 0 else np.zeros_like(f0)
        return -0.5 * f0 + d, -0.5 * f0 - d
    same = P.lo[0] == P.hi[0]
    dlo = np.where(same, -0.5 * f0, np.where(x0 == P.lo[0], -f0, 0.0))
    dhi = np.where(same, -0.5 * f0, np.where(x0 == P.hi[0], -f0, 0.0))
    return dlo, dhi


def envelope_gradient(P, st: du.DualState):
    """Returns dict: dW[k] dense (k = 1..n), db[k], dlo0, dhi0 for one subproblem."""
    val, f, g, x, z = du.evaluate(P, st)
    n = P.n
    dW, db = [None] * (n + 1), [None] * (n + 1)
    for k in range(1, n):
        W = P.W[k]
        Lc, Uc = rx.interval_matrices(W, P.lo[k - 1], P.hi[k - 1])
        r = st.alpha[k] - st.beta1[k]
        G = np.outer(r, x[k - 1])
        gb = r.copy()
        for sl in st.slots[k]:
            If = sl.I.astype(np.float64)
            G += sl.beta[:, None] * (If * ((1 - z[k])[:, None] * Lc - x[k - 1][None, :])
                                     - z[k][:, None] * (1 - If) * Uc)
            gb -= sl.beta * z[k]
        dW[k], db[k] = G, gb
    dW[n] = x[n - 1][None, :].copy()
    db[n] = np.ones(1)
    W1 = P.W[1]
    pos = W1 >= 0
    dlo, dhi = _x0_box_terms(P, f[0], x[0])
    # where l_0 = u_0 both indicators hold; the box then moves as one point and f_0 enters once
    if n >= 2:
        for sl in st.slots[1]:
            If = sl.I.astype(np.float64)
            a = (1 - z[1])[:, None] * W1 * If
            c = z[1][:, None] * W1 * (1 - If)
            dlo = dlo + sl.beta @ (a * pos - c * ~pos)
            dhi = dhi + sl.beta @ (a * ~pos - c * pos)
    return dict(value=val, dW=dW, db=db, dlo0=dlo, dhi0=dhi, x=x, z=z)


def filter_gradient(dWdense: np.ndarray, taps, filt_shape) -> np.ndarray:
    """Sum a dense-operator gradient back onto the conv filter entries it was built from."""
    out = np.zeros(int(np.prod(filt_shape)))
    for row, col, fi in taps:
        out[fi] += dWdense[row, col]
    return out.reshape(filt_shape)


def bias_gradient(db_dense: np.ndarray, L: dict) -> np.ndarray:
    """Sum a per-neuron bias gradient of a conv layer over the channel's positions."""
    if L["kind"] == "linear":
        return db_dense
    oc, oh, ow = L["out_shape"]
    return db_dense.reshape(oc, oh * ow).sum(axis=1)


def chain_gradient(P, st: du.DualState, splits=None):
    """The envelope gradient through the interval propagation that produced the bounds.

    Here lhat_k, uhat_k (k >= 1) are not held fixed but follow theta through interval propagation
    (App. E, last paragraph), l_k = max(lhat_k, 0), u_k = max(uhat_k, 0), with a split clamping a
    straddling neuron to a constant. At fixed duals and masks the bound depends on them through
      * x_k* at an end of its box: dd/dl_k = -f_k [x_k* = l_k], dd/du_k = -f_k [x_k* = u_k];
      * Lcheck, Ucheck of layer k+1 (the l_0, u_0 terms above, for every k);
      * the Big-M rows: dd/dlhat_k = beta_{k,1} (1 - z_k), dd/duhat_k = -beta_{k,0} z_k;
    and interval propagation, lhat_k = W+ l_{k-1} + W- u_{k-1} + b, uhat_k = W+ u_{k-1} + W- l_{k-1}
    + b, carries these back, layer by layer, to W, b and the box. The kink of max(., 0) at 0 takes
    the zero derivative; a clamped entry (split +1 with lhat = 0, split -1 with uhat = 0) is a
    constant. P must hold the interval bounds of its box (Problem built without `bounds`).
    """
    val, f, g, x, z = du.evaluate(P, st)
    base = envelope_gradient(P, st)
    n = P.n
    Lb, Ub = [None] * n, [None] * n
    for k in range(n):
        lo, hi = P.lo[k], P.hi[k]
        same = lo == hi
        a = np.where(same, -0.5 * f[k], np.where(x[k] == lo, -f[k], 0.0))
        c = np.where(same, -0.5 * f[k], np.where(x[k] == hi, -f[k], 0.0))
        if k == 0:
            a, c = _x0_box_terms(P, f[0], x[0])
        if k + 1 <= n - 1:
            W = P.W[k + 1]
            pos = W >= 0
            for sl in st.slots[k + 1]:
                If = sl.I.astype(np.float64)
                A = (1 - z[k + 1])[:, None] * W * If
                Cm = z[k + 1][:, None] * W * (1 - If)
                a = a + sl.beta @ (A * pos - Cm * ~pos)
                c = c + sl.beta @ (A * ~pos - Cm * pos)
        Lb[k], Ub[k] = a, c
    offs = np.cumsum([0] + [P.widths[k] for k in range(1, n)])
    dW = [None if w is None else w.copy() for w in base["dW"]]
    db = [None if v is None else v.copy() for v in base["db"]]
    for k in range(n - 1, 0, -1):
        lh, uh = P.lhat[k], P.uhat[k]
        Ah = st.beta1[k] * (1 - z[k]) + np.where(lh > 0, Lb[k], 0.0)
        Uh = -st.beta0[k] * z[k] + np.where(uh > 0, Ub[k], 0.0)
        if splits is not None:
            sp = np.asarray(splits)[offs[k - 1]:offs[k]]
            Ah = np.where((sp > 0) & (lh == 0), 0.0, Ah)
            Uh = np.where((sp < 0) & (uh == 0), 0.0, Uh)
        W = P.W[k]
        if k == 1 and getattr(P, "ball", False):
            # lhat_1, uhat_1 = W c + b -+ r with r_i = |W_i o e|_2 over the ellipsoid; c = (l + u) / 2,
            # e = (u - l) / 2
            c = 0.5 * (P.lo[0] + P.hi[0])
            e = 0.5 * (P.hi[0] - P.lo[0])
            r = np.sqrt(((W * e[None, :]) ** 2).sum(axis=1))
            q = np.where(r[:, None] > 0, W * W * e[None, :] / np.where(r > 0, r, 1.0)[:, None], 0.0)   # dr/de
            dc = W.T @ (Ah + Uh)
            de = q.T @ (Uh - Ah)
            Lb[0] = Lb[0] + 0.5 * dc - 0.5 * de
            Ub[0] = Ub[0] + 0.5 * dc + 0.5 * de
            drdw = np.where(r[:, None] > 0, W * (e * e)[None, :] / np.where(r > 0, r, 1.0)[:, None], 0.0)
            dW[1] = dW[1] + (Ah + Uh)[:, None] * c[None, :] + (Uh - Ah)[:, None] * drdw
            db[1] = db[1] + Ah + Uh
            continue
        Wp, Wn = np.maximum(W, 0.0), np.minimum(W, 0.0)
        Lb[k - 1] = Lb[k - 1] + Wp.T @ Ah + Wn.T @ Uh
        Ub[k - 1] = Ub[k - 1] + Wn.T @ Ah + Wp.T @ Uh
        pos = W >= 0
        lo, hi = P.lo[k - 1][None, :], P.hi[k - 1][None, :]
        dW[k] = dW[k] + Ah[:, None] * np.where(pos, lo, hi) + Uh[:, None] * np.where(pos, hi, lo)
        db[k] = db[k] + Ah + Uh
    return dict(value=val, dW=dW, db=db, dlo0=Lb[0], dhi0=Ub[0], x=x, z=z)

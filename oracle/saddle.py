"""Saddle Point, Alg. 2 of the paper (oracle; test infrastructure only).

All beta variables enter the Lagrangian only through linearly-sized statistics (Sec. 5.1). The
four listed in eq. (10) do not reproduce g_k and the constant term as printed, so this oracle keeps
these four complete linear statistics per hidden layer k (any complete set works: L is linear in
beta, so convex combinations commute with the statistics):
  Sb[k][i] = sum over every mask I of beta_{k,I}[i]                 (all of 2^{W_k}, incl. 0 and 1)
  P[k][j]  = sum over I of ((W_k o I)^T beta_{k,I})[j]              (length n_{k-1})
  G[k][i]  = the coefficient of z_k[i] in the Lagrangian, g_k of eq. (6)
  C[k][i]  = the constant term: sum_I beta_I lam_I + beta_{k,1} (lhat - b)
Then f_k = alpha_k - W_{k+1}^T alpha_{k+1} - Sb_k + P_{k+1}, g_k = G_k, and
  d = sum_k (b_k^T alpha_k + sum_i C_k[i]) + b_n - sum_k f_k^T x_k* - sum_k G_k^T z_k*.

Readings (Sec. 5.2, 8.1, App. C):
  * gamma_t = 1 / (t + 10), t from 0 (Sec. 8.1; the theory's 1/(1+t) is gamma0 = 1);
  * caps eq. (16): mu_alpha = alpha0 where > 0 else c_alpha; mu_beta[i] = sum of all beta0[i]
    where > 0 else c_beta, with c_alpha = c_beta = 1e-3 ("small positive constants");
  * primal init (App. C.2, simplified): start at the closed-form minimiser of the initial duals,
    then 100 projected subgradient steps on the Big-M-restricted primal view, step 1e-2 -> 1e-5
    linearly; the subgradient of the primal view in x_k is -f_k(alpha*, beta*) (L holds
    -f_k^T x_k), so the descent step adds eta * f_k, and likewise eta * g_k for z_k;
  * the dual conditional gradient's argmax over {beta_0, beta_1, beta_I*} breaks ties towards the
    lower index (beta_0, then beta_1, then beta_I*); beta_bar = mu_beta on the winner when its
    gradient is >= 0, else zero (eq. 12);
  * alpha_bar and beta_bar use the current iterate (x^t, z^t); (x_bar, z_bar) is the closed-form
    minimiser at (alpha^t, zeta^t) (Alg. 2);
  * a row of the oracle mask that selects none of the row's free inputs (nonzero weight, l < u;
    a fixed input adds the same term selected or not) is the all-zero constraint, and one that
    selects all of them is the all-ones constraint; those two constraints are the looser,
    interval-bound versions of the beta_0 and beta_1 constraints, which Sec. 2.2 treats
    separately from E_k. Their gradient never exceeds that of beta_0 (resp. beta_1) in exact
    arithmetic, and equals it when the intermediate bounds are interval bounds, so such a row does
    not compete in the choice of eq. (12) (in exact arithmetic this changes no choice, since ties
    go to beta_0 and beta_1);
  * over an ellipsoid input set (P.ball) x_bar_0 is its closed-form vertex (dual.x0_vertex), and
    the primal initialisation's steps on x_0 end in the radial retraction into it
    (dual.retract_x0: the exact projection for a ball, a feasible point for any ellipsoid; App.
    C.2 asks only for a feasible start, and the bound is valid for any primal iterate).
"""
from __future__ import annotations

import numpy as np

from . import dual as du
from . import relaxation as rx
from .active_set import Options, linear_lr


def degenerate_rows(W, I, lo, hi):
    """Rows whose mask selects none, or all, of the row's free inputs: inputs with a nonzero
    weight and l < u. A fixed input (l = u) contributes the same term to the constraint of eq. (4)
    whether selected or not, so such rows are the all-zero or the all-ones constraint."""
    nz = (W != 0) & (lo != hi)[None, :]
    return ~(nz & I).any(axis=1) | ~(nz & ~I).any(axis=1)


class SaddlePoint:
    def __init__(self, P, opt: Options, init: du.DualState, explicit: bool = False):
        self.P, self.opt = P, opt
        n = P.n
        self.alpha = [None] + [init.alpha[k].copy() for k in range(1, n)]
        self.Sb, self.Pst, self.G, self.C = [None], [None], [None], [None]
        self.explicit = explicit
        self.betas = {} if explicit else None
        for k in range(1, n):
            W = P.W[k]
            Sb = init.beta0[k] + init.beta1[k]
            Pk = W.T @ init.beta1[k]
            G = init.beta0[k] * P.uhat[k] + init.beta1[k] * P.lhat[k]
            C = init.beta1[k] * (P.lhat[k] - P.b[k])
            for sl in init.slots[k]:
                Sb = Sb + sl.beta
                Pk = Pk + (W * sl.I).T @ sl.beta
                G = G + sl.beta * (sl.lam + sl.mu + P.b[k])
                C = C + sl.beta * sl.lam
            self.Sb.append(Sb)
            self.Pst.append(Pk)
            self.G.append(G)
            self.C.append(C)
            if explicit:
                for i in range(P.widths[k]):
                    self._add(k, i, "z", init.beta0[k][i])
                    self._add(k, i, "o", init.beta1[k][i])
                    for sl in init.slots[k]:
                        self._add(k, i, sl.I[i].tobytes(), sl.beta[i])
        self.mu_a = [None] + [np.where(self.alpha[k] > 0, self.alpha[k], opt.sp_c_alpha)
                              for k in range(1, n)]
        self.mu_b = [None] + [np.where(self.Sb[k] > 0, self.Sb[k], opt.sp_c_beta)
                              for k in range(1, n)]
        f = self.coefficients()
        self.x = [np.where(f[k] >= 0, P.hi[k], P.lo[k]) for k in range(n)]
        self.x[0] = du.x0_vertex(P, f[0])
        self.z = [None] + [np.where(self.G[k] >= 0, 1.0, 0.0) for k in range(1, n)]
        self._primal_init()
        self.t = 0
        self.best = -np.inf
        self.trace = []

    @classmethod
    def from_state(cls, P, opt: Options, alpha, Sb, Pst, G, C, mu_a, mu_b, x, z, t: int):
        """A solver at a given iterate (1-based lists as in the paper; Pst[k] has n_{k-1} entries),
        skipping conversion and primal initialisation."""
        sp = cls.__new__(cls)
        sp.P, sp.opt, sp.explicit, sp.betas = P, opt, False, None
        cp = lambda L: [None if v is None else np.asarray(v, np.float64).copy() for v in L]
        sp.alpha, sp.Sb, sp.Pst, sp.G, sp.C = cp(alpha), cp(Sb), cp(Pst), cp(G), cp(C)
        sp.mu_a, sp.mu_b = cp(mu_a), cp(mu_b)
        sp.x, sp.z = cp(x), cp(z)
        sp.t, sp.best, sp.trace = t, -np.inf, []
        return sp

    def decision_margin(self, sums_only: bool = False) -> float:
        """Smallest gap, over every decision the next iteration takes, between the deciding value
        and its threshold: the sign of f (x_bar), of G (z_bar), of xhat - x (alpha_bar), the
        top-two gap and the sign of the conditional-gradient choice, and |z - tau| of the mask
        thresholds tau = (x - l) / (u - l) (W > 0), (u - x) / (u - l) (W < 0) of ambiguous
        inputs. sums_only: only the decisions taken on sums (f, xhat - x, the choice), the ones
        whose value depends on the summation's precision."""
        P, n = self.P, self.P.n
        m = min(np.abs(fk).min() for fk in self.coefficients())
        for k in range(1, n):
            W, b, x, z, xp = P.W[k], P.b[k], self.x[k], self.z[k], self.x[k - 1]
            if not sums_only:
                m = min(m, np.abs(self.G[k]).min())
            xhat = W @ xp + b
            m = min(m, np.abs(xhat - x).min())
            I = rx.mask(W, P.lo[k - 1], P.hi[k - 1], xp, z)
            lam, mu = rx.row_sums(W, P.lo[k - 1], P.hi[k - 1], I)
            vI = x - (W * I) @ xp + (1 - z) * lam - z * (b + mu)
            vI = np.where(degenerate_rows(W, I, P.lo[k - 1], P.hi[k - 1]), -np.inf, vI)
            V = np.sort(np.stack([x - z * P.uhat[k], x - xhat + (1 - z) * P.lhat[k], vI]), axis=0)
            m = min(m, (V[2] - V[1]).min(), np.abs(V[2]).min())
            lo, hi = P.lo[k - 1], P.hi[k - 1]
            amb = lo != hi
            if amb.any() and not sums_only:
                den = (hi - lo)[amb]
                tp = (xp[amb] - lo[amb]) / den
                tn = (hi[amb] - xp[amb]) / den
                Wa = W[:, amb]
                dp = np.where(Wa > 0, np.abs(z[:, None] - tp[None, :]), np.inf)
                dn = np.where(Wa < 0, np.abs(z[:, None] - tn[None, :]), np.inf)
                m = min(m, dp.min(), dn.min())
        return float(m)

    # ---------------------------------------------------------------- explicit beta bookkeeping
    def _add(self, k, i, key, val):
        if val != 0.0:
            self.betas[(k, i, key)] = self.betas.get((k, i, key), 0.0) + float(val)

    def explicit_stats(self):
        """(Sb, P, G, C) recomputed from the explicit list of non-zero beta variables."""
        P, n = self.P, self.P.n
        Sb = [None] + [np.zeros(P.widths[k]) for k in range(1, n)]
        Pk = [None] + [np.zeros(P.widths[k - 1]) for k in range(1, n)]
        G = [None] + [np.zeros(P.widths[k]) for k in range(1, n)]
        C = [None] + [np.zeros(P.widths[k]) for k in range(1, n)]
        for (k, i, key), v in self.betas.items():
            W = P.W[k]
            Sb[k][i] += v
            if key == "z":
                G[k][i] += v * P.uhat[k][i]
            elif key == "o":
                Pk[k] += W[i] * v
                G[k][i] += v * P.lhat[k][i]
                C[k][i] += v * (P.lhat[k][i] - P.b[k][i])
            else:
                row = np.frombuffer(key, dtype=bool)
                lam, mu = rx.row_sums(W[i:i + 1], P.lo[k - 1], P.hi[k - 1], row[None, :])
                Pk[k] += W[i] * row * v
                G[k][i] += v * (lam[0] + mu[0] + P.b[k][i])
                C[k][i] += v * lam[0]
        return Sb, Pk, G, C

    # ---------------------------------------------------------------- the method
    def coefficients(self):
        P, n = self.P, self.P.n
        f = [None] * n
        for k in range(n):
            up = P.W[n].T @ np.ones(1) if k == n - 1 else P.W[k + 1].T @ self.alpha[k + 1]
            fk = -up
            if k >= 1:
                fk = fk + self.alpha[k] - self.Sb[k]
            if k + 1 <= n - 1:
                fk = fk + self.Pst[k + 1]
            f[k] = fk
        return f

    def evaluate(self):
        """(d, x_bar, z_bar): bound and primal conditional gradient at (alpha, zeta)."""
        P, n = self.P, self.P.n
        f = self.coefficients()
        xb = [np.where(f[k] >= 0, P.hi[k], P.lo[k]) for k in range(n)]
        xb[0] = du.x0_vertex(P, f[0])
        zb = [None] + [np.where(self.G[k] >= 0, 1.0, 0.0) for k in range(1, n)]
        val = float(P.b[n][0])
        for k in range(1, n):
            val += float(P.b[k] @ self.alpha[k]) + float(self.C[k].sum()) - float(self.G[k] @ zb[k])
        for k in range(n):
            val -= float(f[k] @ xb[k])
        return val, xb, zb

    def _primal_init(self):
        P, n, opt = self.P, self.P.n, self.opt
        T = opt.sp_init_steps
        for t in range(T):
            eta = linear_lr(opt.sp_init_lr0, opt.sp_init_lr1, t, T)
            ab, b0, b1 = [None], [None], [None]
            for k in range(1, n):
                xhat = P.W[k] @ self.x[k - 1] + P.b[k]
                ab.append(np.where(xhat - self.x[k] >= 0, self.mu_a[k], 0.0))
                v0 = self.x[k] - self.z[k] * P.uhat[k]
                v1 = self.x[k] - xhat + (1 - self.z[k]) * P.lhat[k]
                on = np.maximum(v0, v1) >= 0
                pick0 = v0 >= v1
                b0.append(np.where(on & pick0, self.mu_b[k], 0.0))
                b1.append(np.where(on & ~pick0, self.mu_b[k], 0.0))
            fs = []
            for k in range(n):
                if k == n - 1:
                    fk = -(P.W[n].T @ np.ones(1))
                else:
                    fk = -(P.W[k + 1].T @ (ab[k + 1] - b1[k + 1]))
                if k >= 1:
                    fk = fk + ab[k] - b0[k] - b1[k]
                fs.append(fk)
            for k in range(n):
                if k == 0:   # into the input set (a box, or the ellipsoid inscribed in it)
                    self.x[0] = du.retract_x0(P, self.x[0] + eta * fs[0])
                else:
                    self.x[k] = np.clip(self.x[k] + eta * fs[k], P.lo[k], P.hi[k])
            for k in range(1, n):
                gk = b0[k] * P.uhat[k] + b1[k] * P.lhat[k]
                self.z[k] = np.clip(self.z[k] + eta * gk, 0.0, 1.0)

    def step(self, n_iters: int):
        P, n = self.P, self.P.n
        for _ in range(n_iters):
            gamma = 1.0 / (self.t + self.opt.sp_gamma0)
            val, xb, zb = self.evaluate()
            self.best = max(self.best, val)
            self.trace.append(val)
            new = {}
            for k in range(1, n):
                W, b = P.W[k], P.b[k]
                x, z, xp = self.x[k], self.z[k], self.x[k - 1]
                xhat = W @ xp + b
                abar = np.where(xhat - x >= 0, self.mu_a[k], 0.0)
                I = rx.mask(W, P.lo[k - 1], P.hi[k - 1], xp, z)
                lam, mu = rx.row_sums(W, P.lo[k - 1], P.hi[k - 1], I)
                v0 = x - z * P.uhat[k]
                v1 = x - xhat + (1 - z) * P.lhat[k]
                vI = x - (W * I) @ xp + (1 - z) * lam - z * (b + mu)
                vI = np.where(degenerate_rows(W, I, P.lo[k - 1], P.hi[k - 1]), -np.inf, vI)
                V = np.stack([v0, v1, vI])
                sel = np.argmax(V, axis=0)          # first maximum: ties to the lower index
                on = V.max(axis=0) >= 0
                bb = np.where(on, self.mu_b[k], 0.0)
                Sbar = bb
                Gbar = bb * np.choose(sel, [P.uhat[k], P.lhat[k], lam + mu + b])
                Cbar = bb * np.choose(sel, [np.zeros_like(b), P.lhat[k] - b, lam])
                rowsel = np.where(sel == 1, 1.0, 0.0)[:, None] + np.where(sel == 2, 1.0, 0.0)[:, None] * I
                Pbar = (W * rowsel).T @ bb
                new[k] = (abar, Sbar, Pbar, Gbar, Cbar, sel, on, I)
            self.last_sel = [None] + [np.where(new[k][6], new[k][5], 3) for k in range(1, n)]
            for k in range(n):
                self.x[k] = (1 - gamma) * self.x[k] + gamma * xb[k]
            for k in range(1, n):
                abar, Sbar, Pbar, Gbar, Cbar, sel, on, I = new[k]
                self.z[k] = (1 - gamma) * self.z[k] + gamma * zb[k]
                self.alpha[k] = (1 - gamma) * self.alpha[k] + gamma * abar
                self.Sb[k] = (1 - gamma) * self.Sb[k] + gamma * Sbar
                self.Pst[k] = (1 - gamma) * self.Pst[k] + gamma * Pbar
                self.G[k] = (1 - gamma) * self.G[k] + gamma * Gbar
                self.C[k] = (1 - gamma) * self.C[k] + gamma * Cbar
                if self.explicit:
                    for key in list(self.betas):
                        if key[0] == k:
                            self.betas[key] *= (1 - gamma)
                    for i in range(P.widths[k]):
                        if on[i]:
                            key = ("z", "o", I[i].tobytes())[sel[i]]
                            self._add(k, i, key, gamma * self.mu_b[k][i])
            self.t += 1
        return self

    def bound(self) -> float:
        val = self.evaluate()[0]
        self.best = max(self.best, val)
        return val

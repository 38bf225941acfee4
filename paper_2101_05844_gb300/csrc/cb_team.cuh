// Active Set iteration kernels with lane teams.
//
// A unit is one (output neuron, subproblem) pair of a row pass, or one (input neuron,
// subproblem) pair of a col pass; subproblems vary fastest, so the lanes of a warp read the same
// weights (broadcast loads) and, for conv layers, walk the same taps. A team of T lanes (a power
// of two chosen per layer on the host) splits one unit's reduction; the team then reduces with
// shuffles. Conv taps are walked without integer division in the loop, and col-pass units of a
// strided conv are ordered by stride parity (a permutation table) so that a warp's lanes take the
// same branches.
//
// The masks of all active-set slots for one (i, j) pair form a bitset (cb_slot_mask). The col pass
// uses the per-row sums the row pass leaves behind after its Adam step:
//   rp[i]    = -(alpha_i - beta1_i) + sum_b z_b[i] beta_b[i]      (rows whose mask is all ones)
//   bz[b][i] = (1 - z_b[i]) beta_b[i]
// so that, with p_b = [x at its lower bound] or fixed, q_b = [x at its upper bound] or fixed,
//   sum_i W_ij (-(alpha - beta1)_i + sum_b I_b(i,j) beta_b[i])
//     = sum_i W_ij rp[i] + sum_b ( p_b sum_{W_ij > 0} W_ij bz[b][i] + q_b sum_{W_ij < 0} W_ij bz[b][i] ),
// the masked backward product of eq. (6) regrouped by the sign of W (exact: eq. 3 at binary iterates
// sets I_b(i, j) from z_b[i], the sign of W_ij and p_b / q_b only).
#pragma once
#include "cb_kernels.cuh"

namespace cb {

struct TSegs {
    int n;
    int layer[CB_MAXL];
    int start[CB_MAXL + 1];   // first block of each segment
    int T[CB_MAXL];           // team size (1, 2, 4, 8, 16 or 32)
    const int* perm[CB_MAXL]; // col pass of a strided conv: unit order -> input index (or null)
};

template <class Fn>
__device__ __forceinline__ void row_walk_team(const DLayer& L, int i, int lane, int T, Fn fn) {
    if (L.kind == 0) {
        const float* Wr = L.W + (size_t)i * L.n_in;
        for (int j = lane; j < L.n_in; j += T) fn(j, __ldg(Wr + j));
        return;
    }
    const int hw = L.ho * L.wo;
    const int co = i / hw, rem = i - co * hw;
    const int oy = rem / L.wo, ox = rem - oy * L.wo;
    const int y0 = oy * L.st - L.pd, x0 = ox * L.st - L.pd;
    const int ky0 = max(0, -y0), ky1 = min(L.kh, L.hi - y0);
    const int kx0 = max(0, -x0), kx1 = min(L.kw, L.wi - x0);
    const float* Wc = L.W + (size_t)co * L.ci * L.kh * L.kw;
    // lanes stride over (channel, kernel row) pairs
    int c = lane / L.kh, ky = lane - c * L.kh;
    const int cstep = T / L.kh, kstep = T - cstep * L.kh;
    while (c < L.ci) {
        if (ky >= ky0 && ky < ky1) {
            const float* Wk = Wc + (c * L.kh + ky) * L.kw;
            const int jrow = (c * L.hi + y0 + ky) * L.wi + x0;
            for (int kx = kx0; kx < kx1; ++kx) fn(jrow + kx, __ldg(Wk + kx));
        }
        c += cstep;
        ky += kstep;
        if (ky >= L.kh) {
            ky -= L.kh;
            ++c;
        }
    }
}

template <class Fn>
__device__ __forceinline__ void col_walk_team(const DLayer& L, int j, int lane, int T, Fn fn) {
    if (L.kind == 0) {
        const float* Wc = L.W + j;
        for (int i = lane; i < L.n_out; i += T) fn(i, __ldg(Wc + (size_t)i * L.n_in));
        return;
    }
    const int hw = L.hi * L.wi;
    const int c = j / hw, rem = j - c * hw;
    const int y = rem / L.wi, x = rem - y * L.wi;
    // first kernel row (column) that reaches this input and its output row (column); further ones
    // step by the stride in the kernel and by -1 in the output
    const int ky_s = (y + L.pd) % L.st, kx_s = (x + L.pd) % L.st;
    const int oy_s = (y + L.pd - ky_s) / L.st, ox_s = (x + L.pd - kx_s) / L.st;
    const size_t cstride = (size_t)L.ci * L.kh * L.kw;
    const float* Wb = L.W + (size_t)c * L.kh * L.kw;
    for (int co = lane; co < L.co; co += T) {
        const float* Wco = Wb + co * cstride;
        const int ib = co * L.ho * L.wo;
        for (int ky = ky_s, oy = oy_s; ky < L.kh && oy >= 0; ky += L.st, --oy) {
            if (oy >= L.ho) continue;
            for (int kx = kx_s, ox = ox_s; kx < L.kw && ox >= 0; kx += L.st, --ox) {
                if (ox >= L.wo) continue;
                fn(ib + oy * L.wo + ox, __ldg(Wco + ky * L.kw + kx));
            }
        }
    }
}

__device__ __forceinline__ float team_sum(float v, int T) {
    for (int o = T >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- Active Set col pass (phase A)
template <int NS>
__device__ __forceinline__ void as_colA_body(const DNet& net, const DState& st, const DSched& sc, const DLayer& L,
                                             int k, bool valid, int s, int j, int lane, int T, int mode) {
    const int m = k - 1;
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    const size_t NT = net.NT, NH = net.NH, cap = net.cap;
    float acc = 0.f, P[NS > 0 ? NS : 1], Q[NS > 0 ? NS : 1];
#pragma unroll
    for (int b = 0; b < NS; ++b) P[b] = Q[b] = 0.f;
    if (valid && k <= net.n - 1) {
        const size_t rb = (size_t)s * NH + L.h_out;
        const float* rp = st.rp + rb;
        const float* bz = st.bz + (size_t)s * cap * NH + L.h_out;
        col_walk_team(L, j, lane, T, [&](int i, float w) {
            acc += w * rp[i];
            const float wp = fmaxf(w, 0.f), wn = fminf(w, 0.f);
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                const float bb = bz[(size_t)b * NH + i];
                P[b] += wp * bb;
                Q[b] += wn * bb;
            }
        });
    }
    if (T > 1) {
        acc = team_sum(acc, T);
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            P[b] = team_sum(P[b], T);
            Q[b] = team_sum(Q[b], T);
        }
    }
    if (!valid || lane != 0) return;
    const int cap_s = st.caps[s];
    const int nsl = min(sp.nadd_before, cap_s);
    const int bo = sp.nadd_before & 1;
    const bool add_iter = (mode == 0) && sp.b_new >= 0;
    const bool add = add_iter && sp.b_new < cap_s;
    const size_t xo = (size_t)s * NT + L.in_off + j;
    const float lo = st.lo[xo], hi = st.hi[xo];
    const unsigned xs = st.xsnap[bo][xo];
    const bool fixed = st.efix[xo];
    float f;
    if (k <= net.n - 1) {
        f = acc;
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            const bool up = (xs >> b) & 1u;
            if (fixed || !up) f += P[b];
            if (fixed || up) f += Q[b];
        }
    } else {
        f = -net.Wout[(size_t)s * L.n_in + j];
    }
    double term = 0.0;
    if (m >= 1) {
        const size_t h = (size_t)s * NH + L.h_in + j;
        const size_t hs = (size_t)s * cap * NH + L.h_in + j;
        float sb = 0.f, gk = st.beta0[h] * st.uhat[h] + st.beta1[h] * st.lhat[h];
        double cterm = 0.0;
        for (int b = 0; b < nsl; ++b) {
            const float bb = st.bs[hs + (size_t)b * NH];
            sb += bb;
            gk += bb * st.kap[hs + (size_t)b * NH];
            cterm += (double)bb * st.lam[hs + (size_t)b * NH];
        }
        f += st.alpha[h] - st.beta0[h] - st.beta1[h] - sb;
        const bool z = gk >= 0.f;
        st.zcur[h] = z;
        const float bm = net.L[m - 1].b[j];
        term = (double)bm * st.alpha[h] + (double)st.beta1[h] * ((double)st.lhat[h] - bm) + cterm -
               (z ? (double)gk : 0.0);
        if (add_iter) {
            const unsigned zs_old = st.zsnap[bo][h];
            st.zsnap[bo ^ 1][h] = (uint8_t)(zs_old | ((add && z) ? (1u << sp.b_new) : 0u));
        }
    }
    const bool up = f >= 0.f;
    const float xv = up ? hi : lo;
    st.xval[xo] = xv;
    st.fval[xo] = f;
    term -= (double)f * xv;
    st.terms[xo] = term;
    if (add_iter) st.xsnap[bo ^ 1][xo] = (uint8_t)(xs | ((add && up) ? (1u << sp.b_new) : 0u));
}

__device__ __forceinline__ int tseg_of(const TSegs& sg, int blk) {
    int q = 0;
    while (q + 1 < sg.n && blk >= sg.start[q + 1]) ++q;
    return q;
}

// Col pass over layers k = 1..n (phase A of an iteration, or the bound evaluation with mode 1):
// f_m for every neuron j of layer m = k-1 (Sec. 4.1), x*, z* (eqs. 7-8), per-neuron bound terms
// (eq. 6) and, on addition iterations, the new slot's snapshot bits (Alg. 1, Prop. 1).
__global__ void __launch_bounds__(CB_THREADS) k_as_colA_t(DNet net, DState st, DSched sc, TSegs sg, int mode) {
    const int q = tseg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    const DLayer& L = net.L[li];
    const int T = sg.T[q];
    const int t = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    const int unit = t / T, lane = t - unit * T;
    const bool valid = unit < net.S * L.n_in;
    const int o = valid ? unit / net.S : 0, s = valid ? unit - o * net.S : 0;
    const int j = (valid && sg.perm[q]) ? sg.perm[q][o] : o;
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    const int ns = min(sp.nadd_before, sc.maxcut);
    switch (ns) {
        case 0: as_colA_body<0>(net, st, sc, L, li + 1, valid, s, j, lane, T, mode); break;
        case 1: as_colA_body<1>(net, st, sc, L, li + 1, valid, s, j, lane, T, mode); break;
        case 2: as_colA_body<2>(net, st, sc, L, li + 1, valid, s, j, lane, T, mode); break;
        case 3: as_colA_body<3>(net, st, sc, L, li + 1, valid, s, j, lane, T, mode); break;
        case 4: as_colA_body<4>(net, st, sc, L, li + 1, valid, s, j, lane, T, mode); break;
        case 5: as_colA_body<5>(net, st, sc, L, li + 1, valid, s, j, lane, T, mode); break;
        case 6: as_colA_body<6>(net, st, sc, L, li + 1, valid, s, j, lane, T, mode); break;
        case 7: as_colA_body<7>(net, st, sc, L, li + 1, valid, s, j, lane, T, mode); break;
        default: as_colA_body<8>(net, st, sc, L, li + 1, valid, s, j, lane, T, mode); break;
    }
}

// ---------------------------------------------------------------- Active Set row pass (phase B)
// Row pass over hidden layers: W x*, the masked products (W o I_b) x* of every slot and, on
// addition iterations, lambda and kappa of the new slot; the supergradient (eq. 9), Adam steps and
// projection (Alg. 1); then the per-row sums rp and bz for the next col pass.
template <int NS, bool ADD>
__device__ __forceinline__ void as_rowB_body(const DNet& net, const DState& st, const DSched& sc, const DLayer& L,
                                             bool valid, int s, int i, int lane, int T, const Step& sp, int it) {
    const size_t NT = net.NT, NH = net.NH, cap = net.cap;
    const int cap_s = valid ? st.caps[s] : 0;
    const int newb = (ADD && sp.b_new < cap_s) ? sp.b_new : -1;
    const int bn = (sp.nadd_before + (sp.b_new >= 0 ? 1 : 0)) & 1;
    const size_t h = (size_t)s * NH + L.h_out + i;
    const unsigned zs = valid ? st.zsnap[bn][h] : 0u;
    float acc0 = 0.f, lamN = 0.f, muN = 0.f;
    float acc[NS > 0 ? NS : 1];
#pragma unroll
    for (int b = 0; b < NS; ++b) acc[b] = 0.f;
    if (valid) {
        const size_t ib = (size_t)s * NT + L.in_off;
        const float* xv = st.xval + ib;
        const uint8_t* xsn = st.xsnap[bn] + ib;
        const uint8_t* fx = st.efix + ib;
        const float* lo = st.lo + ib;
        const float* hi = st.hi + ib;
        // products rounded once and added without contraction: where the mask selects exactly the
        // inputs at their interval end (Lcheck = x), the masked product and lambda of a new slot
        // then cancel exactly in the supergradient, as they do in exact arithmetic
        row_walk_team(L, i, lane, T, [&](int j, float w) {
            const float wx = __fmul_rn(w, xv[j]);
            acc0 = __fadd_rn(acc0, wx);
            if (NS > 0) {
                const unsigned xs = xsn[j];
                const unsigned f = fx[j] ? 0xFFu : 0u;
                const unsigned msk = w > 0.f ? ((~xs) | f) : (w < 0.f ? (xs | f) : 0xFFu);
#pragma unroll
                for (int b = 0; b < NS; ++b)
                    if ((msk >> b) & 1u) acc[b] = __fadd_rn(acc[b], wx);
                if (ADD && newb >= 0) {
                    const float l = lo[j], u = hi[j];
                    if (((zs | msk) >> (newb & 7)) & 1u) lamN = __fadd_rn(lamN, __fmul_rn(w, w >= 0.f ? l : u));
                    else muN = __fadd_rn(muN, __fmul_rn(w, w >= 0.f ? u : l));
                }
            }
        });
    }
    if (T > 1) {
        acc0 = team_sum(acc0, T);
#pragma unroll
        for (int b = 0; b < NS; ++b) acc[b] = team_sum(acc[b], T);
        if (ADD) {
            lamN = team_sum(lamN, T);
            muN = team_sum(muN, T);
        }
    }
    if (!valid || lane != 0) return;
    const int nsl = min(sp.nadd_before + (sp.b_new >= 0 ? 1 : 0), cap_s);
    const float bi = L.b[i];
    const float xhat = acc0 + bi;
    const float x = st.xval[(size_t)s * NT + L.out_off + i];
    const float z = st.zcur[h] ? 1.f : 0.f;
    const int step = it + 1;
    float bc1 = bias_corr(st.bc1_tab, sc.ntab, step, sc.b1);
    float bc2 = bias_corr(st.bc2_tab, sc.ntab, step, sc.b2);
    adam(st.alpha[h], st.ma[h], st.va[h], xhat - x, sp.lr, bc1, bc2, sc);
    adam(st.beta0[h], st.m0[h], st.v0[h], x - z * st.uhat[h], sp.lr, bc1, bc2, sc);
    adam(st.beta1[h], st.m1[h], st.v1[h], x - xhat + (1.f - z) * st.lhat[h], sp.lr, bc1, bc2, sc);
    float rsum = -(st.alpha[h] - st.beta1[h]);
    const size_t hs0 = (size_t)s * cap * NH + L.h_out + i;
#pragma unroll
    for (int b = 0; b < NS; ++b) {
        if (b >= nsl) continue;
        const size_t hs = hs0 + (size_t)b * NH;
        float lam, kap;
        if (ADD && b == newb) {
            lam = lamN;
            kap = lamN + muN + bi;
            st.lam[hs] = lam;
            st.kap[hs] = kap;
        } else {
            lam = st.lam[hs];
            kap = st.kap[hs];
        }
        const bool zb = (zs >> b) & 1u;
        const float prod = zb ? acc0 : acc[b];
        const float gb = x - prod + lam * (1.f - z) - z * (kap - lam);
        const int sstep = sp.t - cb_slot_added_at(b, sc) + 1;
        bc1 = bias_corr(st.bc1_tab, sc.ntab, sstep, sc.b1);
        bc2 = bias_corr(st.bc2_tab, sc.ntab, sstep, sc.b2);
        adam(st.bs[hs], st.ms[hs], st.vs[hs], gb, sp.lr, bc1, bc2, sc);
        const float bv = st.bs[hs];
        if (zb) rsum += bv;
        st.bz[hs] = zb ? 0.f : bv;
    }
    st.rp[h] = rsum;
}

__global__ void __launch_bounds__(CB_THREADS) k_as_rowB_t(DNet net, DState st, DSched sc, TSegs sg) {
    const int q = tseg_of(sg, blockIdx.x);
    const DLayer& L = net.L[sg.layer[q]];
    const int T = sg.T[q];
    const int t = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    const int unit = t / T, lane = t - unit * T;
    const bool valid = unit < net.S * L.n_out;
    const int i = valid ? unit / net.S : 0, s = valid ? unit - i * net.S : 0;
    const int it = st.ctr[0];
    const Step sp = cb_step(it, sc, st.lr_tab);
    const int ns = min(sp.nadd_before + (sp.b_new >= 0 ? 1 : 0), sc.maxcut);
    if (sp.b_new >= 0) {
        switch (ns) {
            case 1: as_rowB_body<1, true>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 2: as_rowB_body<2, true>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 3: as_rowB_body<3, true>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 4: as_rowB_body<4, true>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 5: as_rowB_body<5, true>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 6: as_rowB_body<6, true>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 7: as_rowB_body<7, true>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            default: as_rowB_body<8, true>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
        }
    } else {
        switch (ns) {
            case 0: as_rowB_body<0, false>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 1: as_rowB_body<1, false>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 2: as_rowB_body<2, false>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 3: as_rowB_body<3, false>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 4: as_rowB_body<4, false>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 5: as_rowB_body<5, false>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 6: as_rowB_body<6, false>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            case 7: as_rowB_body<7, false>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
            default: as_rowB_body<8, false>(net, st, sc, L, valid, s, i, lane, T, sp, it); break;
        }
    }
    if (last_block(&st.done[0]) && threadIdx.x == 0) {
        st.ctr[0] = it + 1;
        st.done[0] = 0;
    }
}

// rp and bz from the current duals and snapshots (after a state import).
__global__ void k_rowprep(DNet net, DState st, DSched sc) {
    const size_t n = (size_t)net.S * net.NH;
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    const int bo = sp.nadd_before & 1;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(u / net.NH), hh = (int)(u - (size_t)s * net.NH);
        const int nsl = min(sp.nadd_before, st.caps[s]);
        const unsigned zs = st.zsnap[bo][u];
        float r = -(st.alpha[u] - st.beta1[u]);
        for (int b = 0; b < net.cap; ++b) {
            const size_t hs = ((size_t)s * net.cap + b) * net.NH + hh;
            const float bv = b < nsl ? st.bs[hs] : 0.f;
            const bool zb = (zs >> b) & 1u;
            if (zb) r += bv;
            st.bz[hs] = zb ? 0.f : bv;
        }
        st.rp[u] = r;
    }
}

// efix[s][j] = (l == u): fixed inputs, whose mask bit is 1 for every slot.
__global__ void k_efix(DNet net, DState st) {
    const size_t n = (size_t)net.S * net.NT;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x)
        st.efix[u] = st.lo[u] == st.hi[u];
}

}  // namespace cb

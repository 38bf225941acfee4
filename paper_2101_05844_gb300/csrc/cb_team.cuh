// Active Set iteration kernels with lane teams.
//
// A unit is one (output neuron, subproblem) pair of a row pass, or one (input neuron,
// subproblem) pair of a col pass; neurons vary fastest, so the lanes of a warp read neighbouring
// entries of one subproblem's vectors and, for conv layers, share weights (broadcast loads). A team of T lanes (a power
// of two chosen per layer on the host) splits one unit's reduction; the team then reduces with
// shuffles. Conv taps are walked without integer division in the loop, and col-pass units of a
// strided conv are ordered by stride parity (a permutation table) so that a warp's lanes take the
// same branches.
//
// The masks of all active-set slots for one (i, j) pair form a bitset (cb_slot_mask). The col pass
// uses the per-row record the row pass leaves behind after its Adam step (one to three float4):
//   rp[i]    = -(alpha_i - beta1_i) + sum_b z_b[i] beta_b[i]      (rows whose mask is all ones)
//   bz[b][i] = (1 - z_b[i]) beta_b[i]
// and the row pass reads one 8-byte record per input: x* and the slot masks for W > 0 and W < 0.
// so that, with p_b = [x at its lower bound] or fixed, q_b = [x at its upper bound] or fixed,
//   sum_i W_ij (-(alpha - beta1)_i + sum_b I_b(i,j) beta_b[i])
//     = sum_i W_ij rp[i] + sum_b ( p_b sum_{W_ij > 0} W_ij bz[b][i] + q_b sum_{W_ij < 0} W_ij bz[b][i] ),
// the masked backward product of eq. (6) regrouped by the sign of W (exact: eq. 3 at binary iterates
// sets I_b(i, j) from z_b[i], the sign of W_ij and p_b / q_b only).
#pragma once
#include <cuda_bf16.h>

#include "cb_kernels.cuh"

namespace cb {

#define CB_MAXTAP 9

struct TSegs {
    int n;
    int layer[CB_MAXL];
    int start[CB_MAXL + 1];   // first block of each segment
    int T[CB_MAXL];           // team size (1, 2, 4, 8, 16 or 32)
    const int* perm[CB_MAXL]; // col pass of a strided conv: unit order -> input index (or null)
};

template <class Fn>
__device__ __forceinline__ void col_walk_team(const DLayer& L, int j, int lane, int T, Fn fn) {
    if (L.kind == 0) {
        const float* Wc = L.W + j;
#pragma unroll 4
        for (int i = lane; i < L.n_out; i += T) fn(i, __ldg(Wc + (size_t)i * L.n_in));
        return;
    }
    const int hw = L.hi * L.wi;
    const int c = j / hw, rem = j - c * hw;
    const int y = rem / L.wi, x = rem - y * L.wi;
    // the taps of this input, found once: kernel rows (columns) step by the stride from the first
    // one that reaches the input, output rows (columns) by -1; at most CB_MAXTAP taps are held in
    // registers (kernels up to 3x3 at stride 1, 5x5 at stride 2, 7x7 at stride 3), else the walk
    // falls back to the loops
    const int ky_s = (y + L.pd) % L.st, kx_s = (x + L.pd) % L.st;
    const int oy_s = (y + L.pd - ky_s) / L.st, ox_s = (x + L.pd - kx_s) / L.st;
    const size_t cstride = (size_t)L.ci * L.kh * L.kw;
    const float* Wb = L.W + (size_t)c * L.kh * L.kw;
    const int plane = L.ho * L.wo;
    int tw[CB_MAXTAP], ti[CB_MAXTAP], nt = 0;
    bool fits = true;
    for (int ky = ky_s, oy = oy_s; ky < L.kh && oy >= 0; ky += L.st, --oy) {
        if (oy >= L.ho) continue;
        for (int kx = kx_s, ox = ox_s; kx < L.kw && ox >= 0; kx += L.st, --ox) {
            if (ox >= L.wo) continue;
            if (nt < CB_MAXTAP) {
#pragma unroll
                for (int a = 0; a < CB_MAXTAP; ++a)
                    if (a == nt) { tw[a] = ky * L.kw + kx; ti[a] = oy * L.wo + ox; }
                ++nt;
            } else {
                fits = false;
            }
        }
    }
    if (fits) {
        for (int co = lane; co < L.co; co += T) {
            const float* Wco = Wb + co * cstride;
            const int ib = co * plane;
#pragma unroll
            for (int a = 0; a < CB_MAXTAP; ++a)
                if (a < nt) fn(ib + ti[a], __ldg(Wco + tw[a]));
        }
        return;
    }
    for (int co = lane; co < L.co; co += T) {
        const float* Wco = Wb + co * cstride;
        const int ib = co * plane;
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

// ---------------------------------------------------------------- Active Set walks
// Group and base position of row-pass unit i (output neuron i of layer L).
__device__ __forceinline__ void row_group(const DLayer& L, int i, int& g, int& base) {
    if (L.kind == 0) {
        g = i;
        base = 0;
        return;
    }
    const int hw = L.ho * L.wo;
    const int co = i / hw, rem = i - co * hw;
    const int oy = rem / L.wo, ox = rem - oy * L.wo;
    g = co;
    base = oy * L.st * L.Wp + ox * L.st;
}

// Group and base position of col-pass unit j (input neuron j of layer L).
__device__ __forceinline__ void col_group(const DLayer& L, int j, int& g, int& base) {
    if (L.kind == 0) {
        g = j;
        base = 0;
        return;
    }
    const int hw = L.hi * L.wi;
    const int c = j / hw, rem = j - c * hw;
    const int y = rem / L.wi, x = rem - y * L.wi;
    const int ty = y + L.pd, tx = x + L.pd;
    const int Y0 = ty / L.st, X0 = tx / L.st;
    const int py = ty - Y0 * L.st, px = tx - X0 * L.st;
    g = (c * L.st + py) * L.st + px;
    base = (Y0 + L.hl) * L.Wpo + X0 + L.wl;
}

// Record position of input neuron j (row-pass input records) and output neuron i (col-pass
// output records) of layer L.
__device__ __forceinline__ int xin_pos(const DLayer& L, int j) {
    if (L.kind == 0) return j;
    const int hw = L.hi * L.wi;
    const int c = j / hw, rem = j - c * hw;
    const int y = rem / L.wi, x = rem - y * L.wi;
    return (c * L.Hp + y + L.pd) * L.Wp + x + L.pd;
}
__device__ __forceinline__ int arec_pos(const DLayer& L, int i) {
    if (L.kind == 0) return i;
    const int hw = L.ho * L.wo;
    const int co = i / hw, rem = i - co * hw;
    const int oy = rem / L.wo, ox = rem - oy * L.wo;
    return (co * L.Hpo + oy + L.hl) * L.Wpo + ox + L.wl;
}

// Output records of layer L for subproblem s: RS / 4 planes of float4, plane q holding entries
// 4q .. 4q + 3 of every position, so that lanes reading neighbouring positions read one
// contiguous run per plane.
__device__ __forceinline__ float4* arec_planes(const DNet& net, const DState& st, const DLayer& L, int s) {
    return reinterpret_cast<float4*>(st.arec + (size_t)s * net.AT + L.ao);
}
__device__ __forceinline__ float* arec_entry(const DNet& net, const DState& st, const DLayer& L, int s, int p, int e) {
    return reinterpret_cast<float*>(arec_planes(net, st, L, s) + (size_t)(e >> 2) * L.apos + p) + (e & 3);
}

// The first NV entries of the record at q (planes apos apart).
template <int NV>
__device__ __forceinline__ void load_rec(const float4* q, int apos, float (&v)[12]) {
    const float4 a = q[0];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    if (NV > 4) { const float4 b = q[apos]; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w; }
    if (NV > 8) { const float4 c = q[2 * apos]; v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w; }
}

// Records of the float32 slot row sums (k_slot_sums_t below): per input {l, u, p bits | q bits
// << 8} in the first Saddle Point input plane, which Active Set leaves unused.
__device__ __forceinline__ float4* slot_rec_plane(const DNet& net, const DState& st, const DLayer& L, int s) {
    return st.spin + (size_t)s * net.XT + (size_t)L.xo;
}
// The record of an input with box [lo, hi] and snapshot bits xs (bit b: at its upper end when slot b
// was added); a fixed input (lo = hi) is selected by every mask, an interior one (layer 0 over an
// ellipsoid) by none: its bit is z alone.
__device__ __forceinline__ float4 slot_rec(float lo, float hi, unsigned xs, bool fixed, bool interior) {
    const unsigned fxm = fixed ? 0xFFu : 0u;
    const unsigned pm = (interior ? 0u : (~xs & 0xFFu)) | fxm, qm = (interior ? 0u : (xs & 0xFFu)) | fxm;
    return make_float4(lo, hi, __uint_as_float(pm | (qm << 8)), 0.f);
}

// B taps of a lane's stride T starting at t (taps at or past tb read as {0, +0.f}: a zero weight
// at the unit's base position, which adds nothing). Loading a whole batch of taps, then all of their
// records, keeps B independent loads in flight per lane instead of one dependent pair at a time.
template <int B>
__device__ __forceinline__ void load_taps(const int2* tap, int t, int tb, int T, int2 (&e)[B]) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int tt = t + b * T;
        e[b] = tt < tb ? tap[tt] : make_int2(0, 0);
    }
}

// ---------------------------------------------------------------- BF16 form: staged plane stores
// A block of the BF16 form's conv passes is one tile of 8 channels (its warps) x 32 positions (its
// lanes) of one subproblem (tc_tile_unit). The channels-last bf16 planes hold the 8 channels of a
// position in one 16-byte piece, so the block gathers its values in shared memory, position-major,
// and stores whole pieces: one 16-byte store per (plane, position) instead of eight 2-byte stores
// scattered a channel stride apart.
// 4-byte asynchronous copy global -> shared (L1-allocating): a value in flight holds no register.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

constexpr int CB_STAGE_PLANES = 2 * (CB_MAXCUT + 1);
struct TcStage {
    __align__(16) uint16_t v[CB_STAGE_PLANES][CB_THREADS];
};
// this thread's entry of plane e: position (lane) major, channel (warp) minor
__device__ __forceinline__ uint16_t& stage_at(TcStage& st, int e) {
    return st.v[e][(threadIdx.x & 31) * 8 + (threadIdx.x >> 5)];
}
__device__ __forceinline__ uint16_t bf16_bits_rn(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
// Stores planes 0 .. nplanes - 1 of the stage: plane e of the tile goes to dst(e) + the position's
// offset; pos_off(p) gives the element offset of position p (channel octet cb of the tile added).
template <class Dst, class PosOff>
__device__ __forceinline__ void stage_store(const TcStage& st, int nplanes, int P, int pb, Dst dst, PosOff pos_off) {
    for (int c = threadIdx.x; c < nplanes * 32; c += CB_THREADS) {
        const int e = c >> 5, pos = c & 31, p = pb * 32 + pos;
        if (p >= P) continue;
        *reinterpret_cast<uint4*>(dst(e) + pos_off(p)) = *reinterpret_cast<const uint4*>(&st.v[e][pos * 8]);
    }
}

// Channel and position of a conv tile's unit (BF16 form), worked out once by the kernel.
struct TcPos {
    int c, y, x;
};
// a / st for the small strides of conv layers, without a division for strides 1 and 2
__device__ __forceinline__ int div_stride(int a, int st) { return st == 1 ? a : (st == 2 ? a >> 1 : a / st); }

// ---------------------------------------------------------------- Active Set col pass (phase A)
// The masked backward product of eq. (6) for input j, regrouped by the sign of W: at binary
// iterates eq. (3) gives I_b(i, j) = 1 on rows with z_b[i] = 1 (their beta is in the record's
// first entry) and otherwise I_b(i, j) = p_b(j) where W_ij > 0, q_b(j) where W_ij < 0, with
// p_b = [x_j at its lower bound when slot b was added] or fixed, q_b = [at its upper bound] or
// fixed. Walking the positive taps, then the negative ones, the lanes accumulate, per slot,
//   Pp_b = sum_{W_ij > 0} W_ij bz_b[i],  Pn_b = sum_{W_ij < 0} W_ij bz_b[i]
// with no per-pair mask work; the input's own bits pick p_b Pp_b + q_b Pn_b at the end.
template <int NS>
__device__ __forceinline__ void as_colA_body(const DNet& net, const DState& st, const DSched& sc, const DLayer& L,
                                             int k, bool valid, int s, int j, int lane, int T, int mode) {
    const int m = k - 1;
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    const size_t NT = net.NT, NH = net.NH, cap = net.cap;
    float acc = 0.f, Pp[NS > 0 ? NS : 1], Pn[NS > 0 ? NS : 1];
#pragma unroll
    for (int b = 0; b < NS; ++b) Pp[b] = Pn[b] = 0.f;
    if (valid && k <= net.n - 1) {
        int g, base;
        col_group(L, j, g, base);
        const float4* ar = arec_planes(net, st, L, s) + base;
        const int apos = L.apos;
        const int t0 = L.cgrp[2 * g], t1 = L.cgrp[2 * g + 1], t2 = L.cgrp[2 * g + 2];
        constexpr int B = 2;   // records of up to 12 floats: two in flight fit 64 registers
        for (int ph = 0; ph < 2; ++ph) {
            const int ta = ph ? t1 : t0, tb = ph ? t2 : t1;
            for (int t = ta + lane; t < tb; t += B * T) {
                int2 e[B];
                load_taps<B>(L.ctap, t, tb, T, e);
                float v[B][12];
#pragma unroll
                for (int q = 0; q < B; ++q) load_rec<1 + NS>(ar + e[q].x, apos, v[q]);
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    const float w = __int_as_float(e[q].y);
                    acc = fmaf(w, v[q][0], acc);
#pragma unroll
                    for (int b = 0; b < NS; ++b) {
                        if (ph) Pn[b] = fmaf(w, v[q][1 + b], Pn[b]);
                        else Pp[b] = fmaf(w, v[q][1 + b], Pp[b]);
                    }
                }
            }
        }
    }
    if (T > 1) {
        acc = team_sum(acc, T);
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            Pp[b] = team_sum(Pp[b], T);
            Pn[b] = team_sum(Pn[b], T);
        }
    }
    if (!valid || lane != 0) return;
    const bool want_terms = mode != 2;
    const int cap_s = st.caps[s];
    const int nsl = min(sp.nadd_before, cap_s);
    const int bo = sp.nadd_before & 1;
    const bool add_iter = (mode != 1) && sp.b_new >= 0;
    const bool add = add_iter && sp.b_new < cap_s;
    const size_t xo = (size_t)s * NT + L.in_off + j;
    const float lo = st.lo[xo], hi = st.hi[xo];
    const unsigned xs = st.xsnap[bo][xo];
    const bool fixed = st.efix[xo];
    const unsigned fxm = fixed ? 0xFFu : 0u;
    float f;
    if (k <= net.n - 1) {
        // an interior input (layer 0 over an ellipsoid) is at neither end of its box: eq. (3) gives z
        const bool interior = net.ball && L.in_off == 0;
        const unsigned pm = (interior ? 0u : ((~xs) & 0xFFu)) | fxm, qm = (interior ? 0u : xs) | fxm;
        f = acc;
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            if ((pm >> b) & 1u) f += Pp[b];
            if ((qm >> b) & 1u) f += Pn[b];
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
        // all slot loads first (NS >= nsl), then the sums in slot order
        float bbv[NS > 0 ? NS : 1], kpv[NS > 0 ? NS : 1], lmv[NS > 0 ? NS : 1];
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            bbv[b] = kpv[b] = lmv[b] = 0.f;
            if (b < nsl) {
                bbv[b] = st.bs[hs + (size_t)b * NH];
                kpv[b] = st.kap[hs + (size_t)b * NH];
                if (want_terms) lmv[b] = st.lam[hs + (size_t)b * NH];
            }
        }
#pragma unroll
        for (int b = 0; b < NS; ++b)
            if (b < nsl) {
                sb += bbv[b];
                gk += bbv[b] * kpv[b];
                if (want_terms) cterm += (double)bbv[b] * lmv[b];
            }
        f += st.alpha[h] - st.beta0[h] - st.beta1[h] - sb;
        const bool z = gk >= 0.f;
        st.zcur[h] = z;
        if (want_terms) {
            const float bm = net.L[m - 1].b[j];
            term = (double)bm * st.alpha[h] + (double)st.beta1[h] * ((double)st.lhat[h] - bm) + cterm -
                   (z ? (double)gk : 0.0);
        }
        if (add_iter) {
            const unsigned zs_old = st.zsnap[bo][h];
            st.zsnap[bo ^ 1][h] = (uint8_t)(zs_old | ((add && z) ? (1u << sp.b_new) : 0u));
        }
    }
    const bool up = f >= 0.f;
    const float xv = up ? hi : lo;
    st.xval[xo] = xv;
    st.fval[xo] = f;
    if (want_terms) st.terms[xo] = term - (double)f * xv;
    unsigned xs_new = xs;
    if (add_iter) {
        xs_new = xs | ((add && up) ? (1u << sp.b_new) : 0u);
        st.xsnap[bo ^ 1][xo] = (uint8_t)xs_new;
    }
    if (k <= net.n - 1) {
        const unsigned mpos = ((~xs_new) & 0xFFu) | fxm, mneg = (xs_new & 0xFFu) | fxm;
        // row-pass input record: x* and the slot masks p_b (bits 0-7) and q_b (bits 8-15)
        reinterpret_cast<float2*>(st.xin + (size_t)s * net.XT + L.xo)[xin_pos(L, j)] =
            make_float2(xv, __uint_as_float(mpos | (mneg << 8)));
    }
}

// Floats per thread of the BF16 col pass's prefetch (as_colA_tc): the W+ and W- products of slot 0
// and of every slot, l and u, five dual and bound values, three per slot.
__host__ __device__ constexpr int colA_tc_vals(int cap) { return 9 + 5 * cap; }

// The BF16 form's col pass for one unit (one lane per unit): as as_colA_body with tc, but every
// value it reads from the state is first copied to shared memory with cp.async (this thread's
// column of buf, colA_tc_vals(cap) floats a CB_THREADS apart), all copies in flight together
// without holding registers.
template <int NS>
__device__ __forceinline__ void as_colA_tc(const DNet& net, const DState& st, const DSched& sc, const DLayer& L,
                                           int k, bool valid, int s, int j, int mode, TcStage* stg, TcPos tp,
                                           float* buf) {
    const int m = k - 1;
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    const size_t NT = net.NT, NH = net.NH, cap = net.cap;
    float* my = buf + threadIdx.x;
    auto at = [&](int v) -> float& { return my[v * CB_THREADS]; };
    enum { V_LO = 2 * NS + 2, V_HI, V_A, V_B0, V_B1, V_UH, V_LH, V_SL };
    const bool want_terms = mode != 2;
    const bool prod = k <= net.n - 1;   // the output layer's inputs have no products
    const int cap_s = valid ? st.caps[s] : 0;
    const int nsl = min(sp.nadd_before, cap_s);
    const int bo = sp.nadd_before & 1;
    const size_t xo = (size_t)s * NT + L.in_off + j;
    const size_t h = (size_t)s * NH + L.h_in + j, hs = (size_t)s * cap * NH + L.h_in + j;
    unsigned xs = 0u;
    bool fixed = false;
    if (valid) {
        if (prod) {
            const BfLayer& B = net.bf[k - 1];
            int c = j, ph = 0, q = 0;
            if (L.kind == 1) {
                c = tp.c;
                const int ty = tp.y + L.pd, tx = tp.x + L.pd;
                const int Y0 = div_stride(ty, L.st), X0 = div_stride(tx, L.st);
                ph = (ty - Y0 * L.st) * L.st + (tx - X0 * L.st);
                q = (Y0 - B.Y0a[ph]) * B.nX[ph] + (X0 - B.X0a[ph]);
            }
            const int P = B.nY[ph] * B.nX[ph];
            const size_t slot = (size_t)net.S * 2 * L.ci * P, neg = (size_t)L.ci * P;
            const float* d = B.Dcol[ph] + ((size_t)s * 2 * L.ci + c) * P + q;
#pragma unroll
            for (int b = 0; b <= NS; ++b) {
                cp_async4(&at(2 * b), d + b * slot);
                cp_async4(&at(2 * b + 1), d + b * slot + neg);
            }
        }
        cp_async4(&at(V_LO), st.lo + xo);
        cp_async4(&at(V_HI), st.hi + xo);
        if (m >= 1) {
            cp_async4(&at(V_A), st.alpha + h);
            cp_async4(&at(V_B0), st.beta0 + h);
            cp_async4(&at(V_B1), st.beta1 + h);
            cp_async4(&at(V_UH), st.uhat + h);
            cp_async4(&at(V_LH), st.lhat + h);
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                if (b >= nsl) continue;
                cp_async4(&at(V_SL + 3 * b), st.bs + hs + (size_t)b * NH);
                cp_async4(&at(V_SL + 3 * b + 1), st.kap + hs + (size_t)b * NH);
                if (want_terms) cp_async4(&at(V_SL + 3 * b + 2), st.lam + hs + (size_t)b * NH);
            }
        }
        xs = st.xsnap[bo][xo];
        fixed = st.efix[xo];
    }
    cp_async_wait_all();
    if (!valid) return;
    const bool add_iter = (mode != 1) && sp.b_new >= 0;
    const bool add = add_iter && sp.b_new < cap_s;
    const float lo = at(V_LO), hi = at(V_HI);
    const unsigned fxm = fixed ? 0xFFu : 0u;
    float f;
    if (prod) {
        // an interior input (layer 0 over an ellipsoid) is at neither end of its box: eq. (3) gives z
        const bool interior = net.ball && L.in_off == 0;
        const unsigned pm = (interior ? 0u : ((~xs) & 0xFFu)) | fxm, qm = (interior ? 0u : xs) | fxm;
        f = at(0) + at(1);
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            if ((pm >> b) & 1u) f += at(2 + 2 * b);
            if ((qm >> b) & 1u) f += at(3 + 2 * b);
        }
    } else {
        f = -net.Wout[(size_t)s * L.n_in + j];
    }
    double term = 0.0;
    if (m >= 1) {
        const float al = at(V_A), b0 = at(V_B0), b1 = at(V_B1), lh = at(V_LH);
        float sb = 0.f, gk = b0 * at(V_UH) + b1 * lh;
        double cterm = 0.0;
#pragma unroll
        for (int b = 0; b < NS; ++b)
            if (b < nsl) {
                const float bb = at(V_SL + 3 * b);
                sb += bb;
                gk += bb * at(V_SL + 3 * b + 1);
                if (want_terms) cterm += (double)bb * at(V_SL + 3 * b + 2);
            }
        f += al - b0 - b1 - sb;
        const bool z = gk >= 0.f;
        st.zcur[h] = z;
        if (want_terms) {
            const float bm = net.L[m - 1].b[j];
            term = (double)bm * al + (double)b1 * ((double)lh - bm) + cterm - (z ? (double)gk : 0.0);
        }
        if (add_iter) {
            const unsigned zs_old = st.zsnap[bo][h];
            st.zsnap[bo ^ 1][h] = (uint8_t)(zs_old | ((add && z) ? (1u << sp.b_new) : 0u));
        }
    }
    const bool up = f >= 0.f;
    const float xv = up ? hi : lo;
    st.xval[xo] = xv;
    st.fval[xo] = f;
    if (want_terms) st.terms[xo] = term - (double)f * xv;
    unsigned xs_new = xs;
    if (add_iter) {
        xs_new = xs | ((add && up) ? (1u << sp.b_new) : 0u);
        st.xsnap[bo ^ 1][xo] = (uint8_t)xs_new;
    }
    if (prod) {
        // the row pass's tensor-core operand, x* (slot 0) and x* p_b / x* q_b
        const unsigned mpos = ((~xs_new) & 0xFFu) | fxm, mneg = (xs_new & 0xFFu) | fxm;
        const BfLayer& B = net.bf[k - 1];
        const int c = L.kind == 1 ? tp.c : j, y = L.kind == 1 ? tp.y : 0, x = L.kind == 1 ? tp.x : 0;
        const long long off = ((long long)(y + L.pd) * L.Wp + (x + L.pd)) * B.Cip + c;
        const __nv_bfloat16 xb = __float2bfloat16_rn(xv), zero = __float2bfloat16_rn(0.f);
        __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(B.X);
        for (int t = 0; t <= net.cap; ++t) {
            const long long pl = ((long long)t * net.S + s) * 2;
            const bool p = t == 0 || ((mpos >> (t - 1)) & 1u), qq = t == 0 || ((mneg >> (t - 1)) & 1u);
            if (stg) {   // conv tile: the block stores whole 16-byte pieces after the body
                stage_at(*stg, 2 * t) = __bfloat16_as_ushort(p ? xb : zero);
                stage_at(*stg, 2 * t + 1) = __bfloat16_as_ushort(qq ? xb : zero);
            } else {
                X[pl * B.PX + off] = p ? xb : zero;
                X[(pl + 1) * B.PX + off] = qq ? xb : zero;
            }
        }
        // the new slot's float32 lambda, kappa (k_slot_sums_t after the row pass) walk these records
        if (add_iter)
            slot_rec_plane(net, st, L, s)[xin_pos(L, j)] = slot_rec(lo, hi, xs_new, fixed, net.ball && L.in_off == 0);
    }
}

// Ellipsoid input set {sum_j ((x_j - c_j) / e_j)^2 <= 1} inscribed in the box (c, e its centre and
// half-widths; an l2 ball for equal half-widths), one block per subproblem, after the col pass has
// written f_0: the x_0 part of the inner minimisation, min -f_0^T x_0, is attained at
// x_0* = c + e^2 f_0 / |e f_0|_2 (c where f_0 = 0) with value -f_0^T c - |e f_0|_2 (Sec. 2 needs only
// this closed form of the input set). Writes x_0*, that value as the layer's bound term (the
// closed form, not -f_0^T x_0* at a rounded x_0*), and the row-pass records:
// x_0* lies strictly inside the box, so the mask bits of eq. (3) are z alone (cb_slot_mask,
// interior) and the producer bits p_b, q_b are set only for fixed inputs.
constexpr int CB_BALL_THREADS = 1024;
__global__ void __launch_bounds__(CB_BALL_THREADS) k_ball_x0(DNet net, DState st) {
    // float32 per input (the float64 pipe is narrow); the two sums cross threads in float64, and
    // the layer's whole bound term, -f c - |e f|, goes to its first input (the others hold 0)
    const int s = blockIdx.x;
    const DLayer& L = net.L[0];
    const size_t base = (size_t)s * net.NT + L.in_off;
    float p2 = 0.f, pc = 0.f;
    for (int j = threadIdx.x; j < L.n_in; j += CB_BALL_THREADS) {
        const float lo = st.lo[base + j], hi = st.hi[base + j], f = st.fval[base + j];
        const float ef = 0.5f * (hi - lo) * f;
        p2 = fmaf(ef, ef, p2);
        pc = fmaf(f, 0.5f * (lo + hi), pc);
    }
    __shared__ double red[2][CB_BALL_THREADS / 32];
    const double a2 = warp_sum((double)p2), ac = warp_sum((double)pc);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a2;
        red[1][threadIdx.x >> 5] = ac;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < CB_BALL_THREADS / 32 ? red[0][threadIdx.x] : 0.0;
        double w = threadIdx.x < CB_BALL_THREADS / 32 ? red[1][threadIdx.x] : 0.0;
        v = warp_sum(v);
        w = warp_sum(w);
        if (threadIdx.x == 0) {
            red[0][0] = v;
            red[1][0] = w;
        }
    }
    __syncthreads();
    const double nrm = sqrt(red[0][0]);
    const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
    if (threadIdx.x == 0) {
        st.terms[base] = -red[1][0] - nrm;
        st.bnrm[s] = nrm;
    }
    float2* rec = reinterpret_cast<float2*>(st.xin + (size_t)s * net.XT + L.xo);
    for (int j = threadIdx.x; j < L.n_in; j += CB_BALL_THREADS) {
        const size_t xo = base + j;
        const float lo = st.lo[xo], hi = st.hi[xo];
        const float c = 0.5f * (lo + hi), e = 0.5f * (hi - lo);
        const float xv = fminf(fmaxf(c + e * e * st.fval[xo] * inv, lo), hi);
        st.xval[xo] = xv;
        if (j) st.terms[xo] = 0.0;
        const unsigned fxm = st.efix[xo] ? 0xFFu : 0u;
        rec[xin_pos(L, j)] = make_float2(xv, __uint_as_float(fxm | (fxm << 8)));
        if (net.bf) {   // BF16 form: the row products' operand planes, x_0* on slot 0 and on the
                        // slots whose masks hold the input (fixed inputs only, at interior x_0*)
            const BfLayer& B = net.bf[0];
            int c = j, y = 0, xx = 0;
            if (L.kind == 1) {
                const int hw = L.hi * L.wi;
                c = j / hw;
                const int rem = j - c * hw;
                y = rem / L.wi;
                xx = rem - y * L.wi;
            }
            const long long off = ((long long)(y + L.pd) * L.Wp + (xx + L.pd)) * B.Cip + c;
            const __nv_bfloat16 xb = __float2bfloat16_rn(xv), zero = __float2bfloat16_rn(0.f);
            __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(B.X);
            for (int t = 0; t <= net.cap; ++t) {
                const long long pl = ((long long)t * net.S + s) * 2;
                const bool on = t == 0 || fxm != 0u;
                X[pl * B.PX + off] = on ? xb : zero;
                X[(pl + 1) * B.PX + off] = on ? xb : zero;
            }
        }
    }
}

// BF16 form, conv layers: a block of 256 threads takes 8 channels x 32 positions of one subproblem
// (C channels of P positions), so that each warp reads the per-neuron vectors (channel-major)
// contiguously while the block's 8 warps together cover whole 32-byte pieces of the channels-last
// products and operand planes. Returns the neuron index c P + p, or -1 past the layer.
__device__ __forceinline__ int tc_tile_unit(int t, int C, int P, int S, int& s) {
    const int ncb = (C + 7) >> 3, npb = (P + 31) >> 5;
    const int tile = t >> 8, lt = t & 255;
    s = tile / (ncb * npb);
    const int rem = tile - s * (ncb * npb);
    const int cb = rem / npb, pb = rem - cb * npb;
    const int c = cb * 8 + (lt >> 5), p = pb * 32 + (lt & 31);
    if (s >= S || c >= C || p >= P) {
        s = 0;
        return -1;
    }
    return c * P + p;
}

__device__ __forceinline__ int tseg_of(const TSegs& sg, int blk) {
    int q = 0;
    while (q + 1 < sg.n && blk >= sg.start[q + 1]) ++q;
    return q;
}

// Col pass over layers k = 1..n (phase A of an iteration, or the bound evaluation with mode 1):
// f_m for every neuron j of layer m = k-1 (Sec. 4.1), x*, z* (eqs. 7-8), per-neuron bound terms
// (eq. 6) and, on addition iterations, the new slot's snapshot bits (Alg. 1, Prop. 1). TC: the
// BF16 form (sums from the tensor-core products, one lane per unit, conv layers in tiles).
template <bool TC>
__global__ void __launch_bounds__(CB_THREADS, 4) k_as_colA_t(DNet net, DState st, DSched sc, TSegs sg,
                                                                       int mode) {
    const int q = tseg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    const DLayer& L = net.L[li];
    const int T = sg.T[q];
    const int t = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    const int unit = t / T, lane = t - unit * T;
    bool valid = unit < net.S * L.n_in;
    int s = valid ? unit / L.n_in : 0, o = valid ? unit - s * L.n_in : 0;
    const bool staged = TC && L.kind == 1 && li + 1 <= net.n - 1;
    __shared__ TcStage stage;
    TcPos tp{0, 0, 0};
    if (TC && L.kind == 1) {   // one lane per unit, tiled
        o = tc_tile_unit(t, L.ci, L.hi * L.wi, net.S, s);
        valid = o >= 0;
        o = valid ? o : 0;
        const int P = L.hi * L.wi;
        tp.c = o / P;
        const int p = o - tp.c * P;
        tp.y = p / L.wi;
        tp.x = p - tp.y * L.wi;
    }
    if (staged)   // zeros stay where the tile has no unit (channel padding)
        for (int e = 0; e < 2 * (net.cap + 1); ++e) stage_at(stage, e) = 0;
    TcStage* stg = staged ? &stage : nullptr;
    const int j = (valid && sg.perm[q]) ? sg.perm[q][o] : o;
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    const int ns = min(sp.nadd_before, sc.maxcut);
    if constexpr (TC) {
        extern __shared__ float colA_buf[];
        switch (ns) {
            case 0: as_colA_tc<0>(net, st, sc, L, li + 1, valid, s, j, mode, stg, tp, colA_buf); break;
            case 1: as_colA_tc<1>(net, st, sc, L, li + 1, valid, s, j, mode, stg, tp, colA_buf); break;
            case 2: as_colA_tc<2>(net, st, sc, L, li + 1, valid, s, j, mode, stg, tp, colA_buf); break;
            case 3: as_colA_tc<3>(net, st, sc, L, li + 1, valid, s, j, mode, stg, tp, colA_buf); break;
            case 4: as_colA_tc<4>(net, st, sc, L, li + 1, valid, s, j, mode, stg, tp, colA_buf); break;
            case 5: as_colA_tc<5>(net, st, sc, L, li + 1, valid, s, j, mode, stg, tp, colA_buf); break;
            case 6: as_colA_tc<6>(net, st, sc, L, li + 1, valid, s, j, mode, stg, tp, colA_buf); break;
            case 7: as_colA_tc<7>(net, st, sc, L, li + 1, valid, s, j, mode, stg, tp, colA_buf); break;
            default: as_colA_tc<8>(net, st, sc, L, li + 1, valid, s, j, mode, stg, tp, colA_buf); break;
        }
    } else
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
    if (staged) {
        __syncthreads();
        const BfLayer& B = net.bf[li];
        const int ncb = (L.ci + 7) >> 3, npb = (L.hi * L.wi + 31) >> 5;
        const int tile = (blockIdx.x - sg.start[q]), ts = tile / (ncb * npb);
        const int rem = tile - ts * (ncb * npb), cb = rem / npb, pb = rem - cb * npb;
        if (ts < net.S) {
            uint16_t* X = B.X;
            stage_store(stage, 2 * (net.cap + 1), L.hi * L.wi, pb,
                        [&](int e) { return X + (((long long)(e >> 1) * net.S + ts) * 2 + (e & 1)) * B.PX; },
                        [&](int p) {
                            const int y = p / L.wi, x = p - y * L.wi;
                            return ((long long)(y + L.pd) * L.Wp + (x + L.pd)) * B.Cip + cb * 8;
                        });
        }
    }
}

// ---------------------------------------------------------------- Active Set row pass (phase B)
// Row pass over hidden layers: W x* and the masked products (W o I_b) x* of every slot, walking
// the positive taps, whose pairs feed the slots with p_b(j) set, then the negative taps (q_b(j));
// the supergradient (eq. 9), Adam steps and projection (Alg. 1); then the per-row sums rp and bz
// for the next col pass.
//
// A slot added at this iteration takes the oracle mask of the current point, where Lcheck_ij = x_j
// on every selected pair of a row with z = 0 and Ucheck_ij = x_j on every other pair, so that
// lambda = (W o I) x* and kappa = W x* + b there; on rows with z = 1 the mask is all ones and
// lambda = sum_j W_ij Lcheck_ij (precomputed per batch). Taking lambda from the same float32 sum
// as the masked product makes the two cancel exactly in the new slot's supergradient, as they do
// in exact arithmetic.
template <int NS, bool ADD>
__device__ __forceinline__ void as_rowB_body(const DNet& net, const DState& st, const DSched& sc, const DLayer& L,
                                             int li, bool valid, int s, int i, int lane, int T, const Step& sp, int it) {
    const size_t NT = net.NT, NH = net.NH, cap = net.cap;
    const int cap_s = valid ? st.caps[s] : 0;
    const int newb = (ADD && sp.b_new < cap_s) ? sp.b_new : -1;
    const int bn = (sp.nadd_before + (sp.b_new >= 0 ? 1 : 0)) & 1;
    const size_t h = (size_t)s * NH + L.h_out + i;
    const unsigned zs = valid ? st.zsnap[bn][h] : 0u;
    float acc0 = 0.f;
    float acc[NS > 0 ? NS : 1];
#pragma unroll
    for (int b = 0; b < NS; ++b) acc[b] = 0.f;
    if (valid) {
        int g, base;
        row_group(L, i, g, base);
        const float2* xb = reinterpret_cast<const float2*>(st.xin + (size_t)s * net.XT + L.xo) + base;
        const int t0 = L.rgrp[2 * g], t1 = L.rgrp[2 * g + 1], t2 = L.rgrp[2 * g + 2];
        // positive taps take the slot masks p_b (bits 0-7), negative taps q_b (bits 8-15)
        constexpr int B = 6;   // six taps and records in flight fit 64 registers
        for (int ph = 0; ph < 2; ++ph) {
            const int ta = ph ? t1 : t0, tb = ph ? t2 : t1;
            const int sh = ph ? 8 : 0;
            for (int t = ta + lane; t < tb; t += B * T) {
                int2 e[B];
                load_taps<B>(L.rtap, t, tb, T, e);
                float2 r[B];
#pragma unroll
                for (int q = 0; q < B; ++q) r[q] = xb[e[q].x];
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    const float wx = __int_as_float(e[q].y) * r[q].x;
                    const unsigned msk = __float_as_uint(r[q].y) >> sh;
                    acc0 += wx;
#pragma unroll
                    for (int b = 0; b < NS; ++b)
                        if ((msk >> b) & 1u) acc[b] += wx;
                }
            }
        }
    }
    if (T > 1) {
        acc0 = team_sum(acc0, T);
#pragma unroll
        for (int b = 0; b < NS; ++b) acc[b] = team_sum(acc[b], T);
    }
    // epilogue: the team's lanes share the Adam updates (variable v = alpha, beta_0, beta_1, then
    // the slots), each lane handling v = lane, lane + T, ...
    const int nsl = min(sp.nadd_before + (sp.b_new >= 0 ? 1 : 0), cap_s);
    float contrib = 0.f;   // this lane's share of rp = -(alpha - beta_1) + sum_b z_b beta_b
    if (valid) {
        const float bi = L.b[i];
        const float x = st.xval[(size_t)s * NT + L.out_off + i];
        const float z = st.zcur[h] ? 1.f : 0.f;
        const float xhat = acc0 + bi;
        const size_t hs0 = (size_t)s * cap * NH + L.h_out + i;
        const int ap = arec_pos(L, i);
        // the col pass's record entry e of this row
        auto put = [&](int e, float v) { *arec_entry(net, st, L, s, ap, e) = v; };
        if (T == 1) {
            // one lane per unit: every load first, so that they are in flight together (the state
            // arrays may alias as far as the compiler knows, so it would not hoist them itself)
            float th3[3] = {st.alpha[h], st.beta0[h], st.beta1[h]};
            float m3[3] = {st.ma[h], st.m0[h], st.m1[h]};
            float v3[3] = {st.va[h], st.v0[h], st.v1[h]};
            const float uh = st.uhat[h], lh = st.lhat[h];
            const int step = it + 1;
            const float ib1 = inv_bias_corr(st.bc1_tab, sc.ntab, step, sc.b1);
            const float ib2 = inv_bias_corr(st.bc2_tab, sc.ntab, step, sc.b2);
            const float g3[3] = {xhat - x, x - z * uh, x - xhat + (1.f - z) * lh};
#pragma unroll
            for (int v = 0; v < 3; ++v) th3[v] = adam_step(th3[v], m3[v], v3[v], g3[v], sp.lr, ib1, ib2, sc);
            st.alpha[h] = th3[0]; st.beta0[h] = th3[1]; st.beta1[h] = th3[2];
            st.ma[h] = m3[0]; st.m0[h] = m3[1]; st.m1[h] = m3[2];
            st.va[h] = v3[0]; st.v0[h] = v3[1]; st.v1[h] = v3[2];
            contrib = th3[2] - th3[0];
            // the slots in pairs: a pair's loads first, then its updates (larger groups spill)
#pragma unroll
            for (int b0 = 0; b0 < NS; b0 += 2) {
                float bsv[2], msv[2], vsv[2], lamv[2], kapv[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int b = b0 + q;
                    bsv[q] = msv[q] = vsv[q] = lamv[q] = kapv[q] = 0.f;
                    if (b < NS && b < nsl) {
                        const size_t hs = hs0 + (size_t)b * NH;
                        bsv[q] = st.bs[hs];
                        msv[q] = st.ms[hs];
                        vsv[q] = st.vs[hs];
                        if (!(ADD && b == newb)) {
                            lamv[q] = st.lam[hs];
                            kapv[q] = st.kap[hs];
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int b = b0 + q;
                    if (b >= NS) continue;
                    if (b >= nsl) {
                        put(1 + b, 0.f);
                        continue;
                    }
                    const size_t hs = hs0 + (size_t)b * NH;
                    const bool zb = (zs >> b) & 1u;
                    float lam = lamv[q], kap = kapv[q];
                    if (ADD && b == newb) {
                        const float lzh = st.lz[h];
                        lam = zb ? lzh : acc[b];
                        // kappa = lambda + sum W (1 - I) Ucheck + b: W x* + b at box vertices; over
                        // interior inputs (layer 0, ellipsoid) the z = 0 mask holds fixed inputs only
                        kap = zb ? lzh + bi : (net.ball && L.in_off == 0 ? st.uz[h] + bi : xhat);
                        st.lam[hs] = lam;
                        st.kap[hs] = kap;
                    }
                    const float prod = zb ? acc0 : acc[b];
                    const float gb = x - prod + lam * (1.f - z) - z * (kap - lam);
                    const int sstep = sp.t - cb_slot_added_at(b, sc) + 1;
                    const float nv = adam_step(bsv[q], msv[q], vsv[q], gb, sp.lr,
                                               inv_bias_corr(st.bc1_tab, sc.ntab, sstep, sc.b1),
                                               inv_bias_corr(st.bc2_tab, sc.ntab, sstep, sc.b2), sc);
                    st.bs[hs] = nv; st.ms[hs] = msv[q]; st.vs[hs] = vsv[q];
                    if (zb) contrib += nv;
                    put(1 + b, zb ? 0.f : nv);
                }
            }
        } else
        for (int v = lane; v < 3 + NS; v += T) {
            if (v < 3) {
                float* th = v == 0 ? st.alpha : (v == 1 ? st.beta0 : st.beta1);
                float* mm = v == 0 ? st.ma : (v == 1 ? st.m0 : st.m1);
                float* vv = v == 0 ? st.va : (v == 1 ? st.v0 : st.v1);
                const float g = v == 0 ? xhat - x : (v == 1 ? x - z * st.uhat[h] : x - xhat + (1.f - z) * st.lhat[h]);
                const int step = it + 1;
                float m = mm[h], w2 = vv[h];
                const float nv = adam_step(th[h], m, w2, g, sp.lr, inv_bias_corr(st.bc1_tab, sc.ntab, step, sc.b1),
                                           inv_bias_corr(st.bc2_tab, sc.ntab, step, sc.b2), sc);
                th[h] = nv; mm[h] = m; vv[h] = w2;
                if (v == 0) contrib -= nv;
                if (v == 2) contrib += nv;
            } else {
                const int b = v - 3;
                if (b >= nsl) { put(1 + b, 0.f); continue; }
                const size_t hs = hs0 + (size_t)b * NH;
                float lam, kap;
                float ab = 0.f;
#pragma unroll
                for (int bb = 0; bb < NS; ++bb)
                    if (bb == b) ab = acc[bb];
                const bool zb = (zs >> b) & 1u;
                if (ADD && b == newb) {
                    const float lzh = st.lz[h];
                    lam = zb ? lzh : ab;
                    kap = zb ? lzh + bi : (net.ball && L.in_off == 0 ? st.uz[h] + bi : xhat);
                    st.lam[hs] = lam;
                    st.kap[hs] = kap;
                } else {
                    lam = st.lam[hs];
                    kap = st.kap[hs];
                }
                const float prod = zb ? acc0 : ab;
                const float gb = x - prod + lam * (1.f - z) - z * (kap - lam);
                const int sstep = sp.t - cb_slot_added_at(b, sc) + 1;
                float m = st.ms[hs], w2 = st.vs[hs];
                const float nv = adam_step(st.bs[hs], m, w2, gb, sp.lr, inv_bias_corr(st.bc1_tab, sc.ntab, sstep, sc.b1),
                                           inv_bias_corr(st.bc2_tab, sc.ntab, sstep, sc.b2), sc);
                st.bs[hs] = nv; st.ms[hs] = m; st.vs[hs] = w2;
                if (zb) contrib += nv;
                put(1 + b, zb ? 0.f : nv);
            }
        }
    }
    if (T > 1) contrib = team_sum(contrib, T);
    if (valid && lane == 0) *arec_entry(net, st, L, s, arec_pos(L, i), 0) = contrib;
}

// Floats per thread of the BF16 row pass's prefetch (as_rowB_tc): the products of slot 0 and of
// every slot, x, the interval bounds, the nine dual and moment values, five per slot.
__host__ __device__ constexpr int rowB_tc_vals(int cap) { return 13 + 6 * cap; }

// The BF16 form's row pass for one unit (one lane per unit): as as_rowB_body, but every value it
// reads from the state is first copied to shared memory with cp.async (this thread's column of
// buf, rowB_tc_vals(cap) floats a CB_THREADS apart), all copies in flight together without holding
// registers, so that a block keeps about 170 bytes per thread in flight and the pass streams at the
// memory's rate rather than its latency.
template <int NS, bool ADD>
__device__ __forceinline__ void as_rowB_tc(const DNet& net, const DState& st, const DSched& sc, const DLayer& L,
                                           int li, bool valid, int s, int i, const Step& sp, int it, TcStage* stg,
                                           float* buf) {
    const size_t NT = net.NT, NH = net.NH, cap = net.cap;
    const int cap_s = valid ? st.caps[s] : 0;
    const int newb = (ADD && sp.b_new < cap_s) ? sp.b_new : -1;
    const int bn = (sp.nadd_before + (sp.b_new >= 0 ? 1 : 0)) & 1;
    const size_t h = (size_t)s * NH + L.h_out + i;
    const int nsl = min(sp.nadd_before + (sp.b_new >= 0 ? 1 : 0), cap_s);
    int co = i, p = 0;
    if (L.kind == 1) {
        const int hw = L.ho * L.wo;
        co = i / hw;
        p = i - co * hw;
    }
    float* my = buf + threadIdx.x;
    auto at = [&](int v) -> float& { return my[v * CB_THREADS]; };
    enum { V_X = NS + 1, V_UH, V_LH, V_TH, V_M = V_TH + 3, V_V = V_M + 3, V_SL = V_V + 3 };
    const size_t hs0 = (size_t)s * cap * NH + L.h_out + i;
    unsigned zs = 0u;
    float zf = 0.f;
    if (valid) {
        const int P = L.ho * L.wo;
        const size_t slot = (size_t)net.S * P * L.co;
        const float* d = net.bf[li].Drow + ((size_t)s * L.co + co) * P + p;
#pragma unroll
        for (int b = 0; b <= NS; ++b) cp_async4(&at(b), d + b * slot);
        cp_async4(&at(V_X), st.xval + (size_t)s * NT + L.out_off + i);
        cp_async4(&at(V_UH), st.uhat + h);
        cp_async4(&at(V_LH), st.lhat + h);
        cp_async4(&at(V_TH), st.alpha + h);
        cp_async4(&at(V_TH + 1), st.beta0 + h);
        cp_async4(&at(V_TH + 2), st.beta1 + h);
        cp_async4(&at(V_M), st.ma + h);
        cp_async4(&at(V_M + 1), st.m0 + h);
        cp_async4(&at(V_M + 2), st.m1 + h);
        cp_async4(&at(V_V), st.va + h);
        cp_async4(&at(V_V + 1), st.v0 + h);
        cp_async4(&at(V_V + 2), st.v1 + h);
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            if (b >= nsl) continue;
            const size_t hs = hs0 + (size_t)b * NH;
            cp_async4(&at(V_SL + 5 * b), st.bs + hs);
            cp_async4(&at(V_SL + 5 * b + 1), st.ms + hs);
            cp_async4(&at(V_SL + 5 * b + 2), st.vs + hs);
            if (!(ADD && b == newb)) {
                cp_async4(&at(V_SL + 5 * b + 3), st.lam + hs);
                cp_async4(&at(V_SL + 5 * b + 4), st.kap + hs);
            }
        }
        zs = st.zsnap[bn][h];
        zf = st.zcur[h] ? 1.f : 0.f;
    }
    cp_async_wait_all();
    float contrib = 0.f;   // rp = -(alpha - beta_1) + sum_b z_b beta_b
    if (valid) {
        const float acc0 = at(0);
        const float bi = L.b[i];
        const float x = at(V_X), z = zf;
        const float xhat = acc0 + bi;
        auto put = [&](int e, float v) {
            if (stg) {   // conv tile: the block stores whole 16-byte pieces after the body
                stage_at(*stg, e) = bf16_bits_rn(v);
            } else {
                const BfLayer& B = net.bf[li];
                const int oy = p / L.wo, ox = p - oy * L.wo;
                const long long roff = ((long long)(oy + L.hl) * L.Wpo + (ox + L.wl)) * B.Cop + co;
                reinterpret_cast<__nv_bfloat16*>(B.R)[((long long)e * net.S + s) * B.PR + roff] = __float2bfloat16_rn(v);
            }
        };
        const int step = it + 1;
        const float ib1 = inv_bias_corr(st.bc1_tab, sc.ntab, step, sc.b1);
        const float ib2 = inv_bias_corr(st.bc2_tab, sc.ntab, step, sc.b2);
        const float g3[3] = {xhat - x, x - z * at(V_UH), x - xhat + (1.f - z) * at(V_LH)};
        float th3[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            float m = at(V_M + v), w2 = at(V_V + v);
            th3[v] = adam_step(at(V_TH + v), m, w2, g3[v], sp.lr, ib1, ib2, sc);
            at(V_M + v) = m;
            at(V_V + v) = w2;
        }
        st.alpha[h] = th3[0]; st.beta0[h] = th3[1]; st.beta1[h] = th3[2];
        st.ma[h] = at(V_M); st.m0[h] = at(V_M + 1); st.m1[h] = at(V_M + 2);
        st.va[h] = at(V_V); st.v0[h] = at(V_V + 1); st.v1[h] = at(V_V + 2);
        contrib = th3[2] - th3[0];
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            if (b >= nsl) {
                put(1 + b, 0.f);
                continue;
            }
            const size_t hs = hs0 + (size_t)b * NH;
            const bool zb = (zs >> b) & 1u;
            const float accb = at(1 + b);
            float lam = at(V_SL + 5 * b + 3), kap = at(V_SL + 5 * b + 4);
            if (ADD && b == newb) {
                const float lzh = st.lz[h];
                lam = zb ? lzh : accb;
                // kappa = lambda + sum W (1 - I) Ucheck + b: W x* + b at box vertices; over interior
                // inputs (layer 0, ellipsoid) the z = 0 mask holds fixed inputs only
                kap = zb ? lzh + bi : (net.ball && L.in_off == 0 ? st.uz[h] + bi : xhat);
                st.lam[hs] = lam;
                st.kap[hs] = kap;
            }
            const float prod = zb ? acc0 : accb;
            const float gb = x - prod + lam * (1.f - z) - z * (kap - lam);
            const int sstep = sp.t - cb_slot_added_at(b, sc) + 1;
            float m = at(V_SL + 5 * b + 1), w2 = at(V_SL + 5 * b + 2);
            const float nv = adam_step(at(V_SL + 5 * b), m, w2, gb, sp.lr,
                                       inv_bias_corr(st.bc1_tab, sc.ntab, sstep, sc.b1),
                                       inv_bias_corr(st.bc2_tab, sc.ntab, sstep, sc.b2), sc);
            st.bs[hs] = nv; st.ms[hs] = m; st.vs[hs] = w2;
            if (zb) contrib += nv;
            put(1 + b, zb ? 0.f : nv);
        }
        if (stg) {
            stage_at(*stg, 0) = bf16_bits_rn(contrib);
        } else {
            put(0, contrib);
        }
    }
}

template <bool TC>
__global__ void __launch_bounds__(CB_THREADS, 4) k_as_rowB_t(DNet net, DState st, DSched sc, TSegs sg) {
    const int q = tseg_of(sg, blockIdx.x);
    const DLayer& L = net.L[sg.layer[q]];
    const int T = sg.T[q];
    const int t = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    const int unit = t / T, lane = t - unit * T;
    bool valid = unit < net.S * L.n_out;
    int s = valid ? unit / L.n_out : 0, i = valid ? unit - s * L.n_out : 0;
    const bool staged = TC && L.kind == 1;
    __shared__ TcStage stage;
    if (TC && L.kind == 1) {   // one lane per unit, tiled
        i = tc_tile_unit(t, L.co, L.ho * L.wo, net.S, s);
        valid = i >= 0;
        i = valid ? i : 0;
    }
    const int it = st.ctr[0];
    const Step sp = cb_step(it, sc, st.lr_tab);
    const int ns = min(sp.nadd_before + (sp.b_new >= 0 ? 1 : 0), sc.maxcut);
    if (staged)   // zeros stay where the tile has no unit (channel padding)
        for (int e = 0; e <= ns; ++e) stage_at(stage, e) = 0;
    TcStage* stg = staged ? &stage : nullptr;
    const int li = sg.layer[q];
    if constexpr (TC) {
        extern __shared__ float rowB_buf[];
        if (sp.b_new >= 0) {
            switch (ns) {
                case 1: as_rowB_tc<1, true>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 2: as_rowB_tc<2, true>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 3: as_rowB_tc<3, true>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 4: as_rowB_tc<4, true>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 5: as_rowB_tc<5, true>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 6: as_rowB_tc<6, true>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 7: as_rowB_tc<7, true>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                default: as_rowB_tc<8, true>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
            }
        } else {
            switch (ns) {
                case 0: as_rowB_tc<0, false>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 1: as_rowB_tc<1, false>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 2: as_rowB_tc<2, false>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 3: as_rowB_tc<3, false>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 4: as_rowB_tc<4, false>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 5: as_rowB_tc<5, false>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 6: as_rowB_tc<6, false>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                case 7: as_rowB_tc<7, false>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
                default: as_rowB_tc<8, false>(net, st, sc, L, li, valid, s, i, sp, it, stg, rowB_buf); break;
            }
        }
    } else if (sp.b_new >= 0) {
        switch (ns) {
            case 1: as_rowB_body<1, true>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 2: as_rowB_body<2, true>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 3: as_rowB_body<3, true>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 4: as_rowB_body<4, true>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 5: as_rowB_body<5, true>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 6: as_rowB_body<6, true>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 7: as_rowB_body<7, true>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            default: as_rowB_body<8, true>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
        }
    } else {
        switch (ns) {
            case 0: as_rowB_body<0, false>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 1: as_rowB_body<1, false>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 2: as_rowB_body<2, false>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 3: as_rowB_body<3, false>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 4: as_rowB_body<4, false>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 5: as_rowB_body<5, false>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 6: as_rowB_body<6, false>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            case 7: as_rowB_body<7, false>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
            default: as_rowB_body<8, false>(net, st, sc, L, li, valid, s, i, lane, T, sp, it); break;
        }
    }
    if (staged) {
        __syncthreads();
        const BfLayer& B = net.bf[li];
        const int ncb = (L.co + 7) >> 3, npb = (L.ho * L.wo + 31) >> 5;
        const int tile = (blockIdx.x - sg.start[q]), ts = tile / (ncb * npb);
        const int rem = tile - ts * (ncb * npb), cb = rem / npb, pb = rem - cb * npb;
        if (ts < net.S) {
            uint16_t* R = B.R;
            stage_store(stage, ns + 1, L.ho * L.wo, pb,
                        [&](int e) { return R + ((long long)e * net.S + ts) * B.PR; },
                        [&](int p) {
                            const int oy = p / L.wo, ox = p - oy * L.wo;
                            return ((long long)(oy + L.hl) * L.Wpo + (ox + L.wl)) * B.Cop + cb * 8;
                        });
        }
    }
}

// ---------------------------------------------------------------- slot row sums
// lambda_b[i] = sum_j W_ij I_b(i, j) Lcheck_ij and kappa_b[i] = lambda_b[i] + sum_j W_ij (1 - I_b(i, j))
// Ucheck_ij + b_i of active-set slots (g_B of Sec. 4.1, the constants of eq. 4), in float32, from
// the slots' snapshot bits. Eq. (3) at a slot's snapshot point gives I_b(i, j) = 1 on rows with
// z_b = 1 (lambda = lz, kappa = lz + b there) and otherwise I_b(i, j) = p_b(j) where W_ij > 0 and
// q_b(j) where W_ij < 0, with Lcheck = l, Ucheck = u where W > 0 and the reverse where W < 0. A lane
// team walks the row's sign-partitioned tap list over per-input records {l, u, p bits | q bits << 8}
// kept in the first Saddle Point input plane (unused while Active Set runs; padding stays zero).
// The records of every input of the hidden-output layers from the snapshot buffer bo.
__global__ void k_slot_recs(DNet net, DState st, int bo) {
    const size_t n = (size_t)net.S * net.NT;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(u / net.NT), hh = (int)(u - (size_t)s * net.NT);
        int li = 0;
        while (li + 2 < net.n && hh >= net.L[li + 1].in_off) ++li;
        const DLayer& L = net.L[li];
        const int j = hh - L.in_off;
        if (j >= L.n_in) continue;   // the last hidden layer feeds only the output row
        slot_rec_plane(net, st, L, s)[xin_pos(L, j)] =
            slot_rec(st.lo[u], st.hi[u], st.xsnap[bo][u], st.efix[u], net.ball && li == 0);
    }
}

template <int NB>
__device__ __forceinline__ void slot_sums_unit(const DNet& net, const DState& st, const DLayer& L, bool valid, int s,
                                               int i, int lane, int T, int b0, int nsl, int bo) {
    float lam[NB], mu[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) lam[b] = mu[b] = 0.f;
    if (valid) {
        int g, base;
        row_group(L, i, g, base);
        const float4* rb = slot_rec_plane(net, st, L, s) + base;
        const int t0 = L.rgrp[2 * g], t1 = L.rgrp[2 * g + 1], t2 = L.rgrp[2 * g + 2];
        constexpr int B = 4;
        for (int ph = 0; ph < 2; ++ph) {
            const int ta = ph ? t1 : t0, tb = ph ? t2 : t1;
            const int sh = (ph ? 8 : 0) + b0;
            for (int t = ta + lane; t < tb; t += B * T) {
                int2 e[B];
                load_taps<B>(L.rtap, t, tb, T, e);
                float4 r[B];
#pragma unroll
                for (int q = 0; q < B; ++q) r[q] = rb[e[q].x];
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    const float w = __int_as_float(e[q].y);
                    // Lcheck, Ucheck: (l, u) for W > 0, (u, l) for W < 0
                    const float wl = w * (ph ? r[q].y : r[q].x), wu = w * (ph ? r[q].x : r[q].y);
                    const unsigned bits = __float_as_uint(r[q].z) >> sh;
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        if ((bits >> b) & 1u) lam[b] += wl;
                        else mu[b] += wu;
                    }
                }
            }
        }
    }
    if (T > 1) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            lam[b] = team_sum(lam[b], T);
            mu[b] = team_sum(mu[b], T);
        }
    }
    if (!valid || lane != 0) return;
    const size_t h = (size_t)s * net.NH + L.h_out + i;
    const unsigned zs = st.zsnap[bo][h];
    const float bi = L.b[i], lzh = st.lz[h];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int bb = b0 + b;
        if (bb >= nsl) continue;
        const bool zb = (zs >> bb) & 1u;
        const size_t hs = ((size_t)s * net.cap + bb) * net.NH + L.h_out + i;
        st.lam[hs] = zb ? lzh : lam[b];
        st.kap[hs] = zb ? lzh + bi : lam[b] + mu[b] + bi;
    }
}

// Slots b0 .. b0 + NB - 1 of the first nadd additions (snapshot buffer nadd & 1), or with after_add
// the slot the Active Set iteration that just ended added (BF16 form: that iteration took lambda,
// kappa from its bf16 products; the col pass wrote the records); returns at once after other
// iterations. Lane teams as in the float32 row pass, a grid-stride loop over its nvb blocks.
template <int NB>
__global__ void __launch_bounds__(CB_THREADS, 4) k_slot_sums_t(DNet net, DState st, DSched sc, TSegs sg, int nvb,
                                                                int b0, int nadd, int after_add) {
    if (after_add) {
        const int it = st.ctr[0] - 1;
        if (it < sc.TM) return;
        const int b = cb_slot_at(it - sc.TM, sc);
        if (b < 0) return;
        nadd = cb_additions_before(it - sc.TM + 1, sc);
        b0 = b;
    }
    const int bo = nadd & 1;
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        const int q = tseg_of(sg, vb);
        const DLayer& L = net.L[sg.layer[q]];
        const int T = sg.T[q];
        const int t = (vb - sg.start[q]) * CB_THREADS + threadIdx.x;
        const int unit = t / T, lane = t - unit * T;
        const bool valid = unit < net.S * L.n_out;
        const int s = valid ? unit / L.n_out : 0, i = valid ? unit - s * L.n_out : 0;
        const int nsl = valid ? min(nadd, st.caps[s]) : 0;
        slot_sums_unit<NB>(net, st, L, valid, s, i, lane, T, b0, nsl, bo);
    }
}

// rp and bz from the current duals and snapshots (after a state import): the float32 output
// records, or with tc the BF16 form's bf16 operand planes.
__global__ void k_rowprep(DNet net, DState st, DSched sc, int tc) {
    const size_t n = (size_t)net.S * net.NH;
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    const int bo = sp.nadd_before & 1;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(u / net.NH), hh = (int)(u - (size_t)s * net.NH);
        int li = 0;
        while (li + 2 < net.n && hh >= net.L[li + 1].h_out) ++li;
        const DLayer& L = net.L[li];
        const int nsl = min(sp.nadd_before, st.caps[s]);
        const unsigned zs = st.zsnap[bo][u];
        const int i = hh - L.h_out;
        const int ap = arec_pos(L, i);
        long long roff = 0;
        if (tc) {
            int co = i, oy = 0, ox = 0;
            if (L.kind == 1) {
                const int hw = L.ho * L.wo;
                co = i / hw;
                oy = (i - co * hw) / L.wo;
                ox = i - co * hw - oy * L.wo;
            }
            roff = ((long long)(oy + L.hl) * L.Wpo + (ox + L.wl)) * net.bf[li].Cop + co;
        }
        auto put = [&](int e, float v) {
            if (tc)
                reinterpret_cast<__nv_bfloat16*>(net.bf[li].R)[((long long)e * net.S + s) * net.bf[li].PR + roff] =
                    __float2bfloat16_rn(v);
            else
                *arec_entry(net, st, L, s, ap, e) = v;
        };
        float r = -(st.alpha[u] - st.beta1[u]);
        for (int b = 0; b < (tc ? net.cap : net.RS - 1); ++b) {
            float bv = 0.f;
            bool zb = false;
            if (b < net.cap) {
                const size_t hs = ((size_t)s * net.cap + b) * net.NH + hh;
                bv = b < nsl ? st.bs[hs] : 0.f;
                zb = (zs >> b) & 1u;
            }
            if (zb) r += bv;
            put(1 + b, zb ? 0.f : bv);
        }
        put(0, r);
    }
}

// Per-batch row constants: lz[s][i] = sum_j W_ij Lcheck_ij (Lcheck = l_j where W_ij >= 0, u_j
// where W_ij < 0), lambda of the all-ones mask, taken by Active Set slots added on rows with z = 1
// (FP64 accumulation rounded to nearest); nfree[s][i] = the nonzero weights of row i on free
// inputs (l < u), against which Saddle Point recognises a mask selecting all of them. One warp per
// row.
__global__ void k_lz(DNet net, DState st, int li) {
    const DLayer& L = net.L[li];
    const int warp = (blockIdx.x * CB_THREADS + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= net.S * L.n_out) return;
    const int s = warp / L.n_out, i = warp - s * L.n_out;
    const float* lo = st.lo + (size_t)s * net.NT + L.in_off;
    const float* hi = st.hi + (size_t)s * net.NT + L.in_off;
    double a = 0.0, c = 0.0;
    int nf = 0;
    row_walk(L, i, lane, [&](int j, float w) {
        a += (double)w * (w >= 0.f ? lo[j] : hi[j]);
        c += (double)w * (w >= 0.f ? hi[j] : lo[j]);
        nf += (w != 0.f && lo[j] != hi[j]) ? 1 : 0;
    });
    a = warp_sum(a);
    c = warp_sum(c);
    for (int o = 16; o > 0; o >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, o);
    if (lane == 0) {
        st.lz[(size_t)s * net.NH + L.h_out + i] = (float)a;
        st.uz[(size_t)s * net.NH + L.h_out + i] = (float)c;
        st.nfree[(size_t)s * net.NH + L.h_out + i] = nf;
    }
}

// efix[s][j] = (l == u): fixed inputs, whose mask bit is 1 for every slot.
__global__ void k_efix(DNet net, DState st) {
    const size_t n = (size_t)net.S * net.NT;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x)
        st.efix[u] = st.lo[u] == st.hi[u];
}


// ---------------------------------------------------------------------- Saddle Point passes
__device__ __forceinline__ bool team_any(bool v, int T) {
    unsigned x = v ? 1u : 0u;
    for (int o = T >> 1; o > 0; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o);
    return x != 0u;
}

struct Unit {
    int T, lane, s, idx;
    bool valid;
};

__device__ __forceinline__ Unit team_unit(const TSegs& sg, int q, int count, int S) {
    Unit u;
    u.T = sg.T[q];
    const int t = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    const int unit = t / u.T;
    u.lane = t - unit * u.T;
    u.valid = unit < S * count;
    u.s = u.valid ? unit / count : 0;
    const int o = u.valid ? unit - u.s * count : 0;
    u.idx = (u.valid && sg.perm[q]) ? sg.perm[q][o] : o;
    return u;
}

// Saddle Point records, in the Active Set walks' layouts (Active Set and Saddle Point do not run on
// one context at the same time, so the output records reuse the Active Set's array):
//  per output position (the first float4 plane of the output records): {alpha, beta_bar on beta_1,
//      beta_bar on I*, z} of the current iterate, written by the row pass (alpha also by k_sp_prep);
//  per input position, two float4 planes (st.spin): {x, tau+, l, u} for W > 0 and {x, tau-, u, l}
//      for W < 0, i.e. {x, threshold, Lcheck, Ucheck} for the sign of the taps that read it.
__device__ __forceinline__ float4* sp_orec(const DNet& net, const DState& st, const DLayer& L, int s, int i) {
    return arec_planes(net, st, L, s) + arec_pos(L, i);
}
// the W > 0 plane of layer L (the W < 0 plane follows, xpos float4 later): in float4 units a
// layer takes 2 xpos, as it takes 2 xpos floats in the Active Set input records
__device__ __forceinline__ float4* sp_iplane(const DNet& net, const DState& st, const DLayer& L, int s) {
    return st.spin + (size_t)s * net.XT + (size_t)L.xo;
}

// alpha into the output records (Saddle Point start, state import).
__global__ void k_sp_prep(DNet net, DState st) {
    const size_t n = (size_t)net.S * net.NH;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(u / net.NH), hh = (int)(u - (size_t)s * net.NH);
        int li = 0;
        while (li + 2 < net.n && hh >= net.L[li + 1].h_out) ++li;
        *sp_orec(net, st, net.L[li], s, hh - net.L[li].h_out) = make_float4(st.alpha[u], 0.f, 0.f, 0.f);
    }
}

// Phase A epilogue for input j of layer L (k = li + 1, m = k - 1): f_m from acc = (W_k^T alpha_k)[j]
// (Sec. 5.1), the primal conditional gradient (eqs. 7-8 with B = E), the bound terms, and the
// records of input j for the row pass: the thresholds of the oracle eq. (3) at the primal iterate
// x (buffer cur), rounded up to float32 (cb_tau_up) so that the row pass's compares are exact.
// init != 0 also starts the primal iterate at the conditional gradient.
__device__ __forceinline__ void sp_phaseA_epilogue(const DNet& net, const DState& st, const DLayer& L, int k,
                                                   int s, int j, float acc, int cur, int init) {
    const int m = k - 1;
    const size_t NT = net.NT, NH = net.NH;
    const size_t xo = (size_t)s * NT + L.in_off + j;
    float f = k <= net.n - 1 ? st.P[xo] - acc : -net.Wout[(size_t)s * L.n_in + j];
    const float lo = st.lo[xo], hi = st.hi[xo];
    double term = 0.0;
    if (m >= 1) {
        const size_t h = (size_t)s * NH + L.h_in + j;
        f += st.alpha[h] - st.Sb[h];
        const float G = st.G[h];
        const bool z = G >= 0.f;
        st.zbar[h] = z;
        if (init) st.spz[cur][h] = z ? 1.f : 0.f;
        term = (double)net.L[m - 1].b[j] * st.alpha[h] + (double)st.C[h] - (z ? (double)G : 0.0);
    }
    const float xb = f >= 0.f ? hi : lo;
    st.xbar[xo] = xb;
    term -= (double)f * xb;
    st.terms[xo] = term;
    if (net.ball && L.in_off == 0) st.fval[xo] = f;   // for the ellipsoid vertex (k_ball_sp)
    const float x = init ? xb : st.spx[cur][xo];
    if (init) st.spx[cur][xo] = xb;
    if (k <= net.n - 1) {
        float tp = -INFINITY, tn = -INFINITY;
        if (lo != hi) {
            tp = cb_tau_up(x, lo, lo, hi);
            tn = cb_tau_up(hi, x, lo, hi);
        }
        float4* r = sp_iplane(net, st, L, s) + xin_pos(L, j);
        r[0] = make_float4(x, tp, lo, hi);
        r[L.xpos] = make_float4(x, tn, hi, lo);
    }
}

// Phase A (col pass over k = 1..n) at the current (alpha, zeta): the walk for W_k^T alpha_k, then
// the epilogue above. Runs alone at the start of Saddle Point, after a state import and for the
// bound; within the iteration loop it is fused with phase C (k_sp_colCA_t).
__global__ void __launch_bounds__(CB_THREADS) k_sp_colA_t(DNet net, DState st, TSegs sg, int init) {
    const int q = tseg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    const DLayer& L = net.L[li];
    const int k = li + 1;
    const Unit u = team_unit(sg, q, L.n_in, net.S);
    float acc = 0.f;
    if (u.valid && k <= net.n - 1) {
        int g, base;
        col_group(L, u.idx, g, base);
        const float4* ar = arec_planes(net, st, L, u.s) + base;
        const int t0 = L.cgrp[2 * g], t2 = L.cgrp[2 * g + 2];
        constexpr int B = 8;
        for (int t = t0 + u.lane; t < t2; t += B * u.T) {
            int2 e[B];
            load_taps<B>(L.ctap, t, t2, u.T, e);
            float a[B];
#pragma unroll
            for (int q = 0; q < B; ++q) a[q] = ar[e[q].x].x;
#pragma unroll
            for (int q = 0; q < B; ++q) acc = fmaf(__int_as_float(e[q].y), a[q], acc);
        }
    }
    if (u.T > 1) acc = team_sum(acc, u.T);
    if (!u.valid || u.lane != 0) return;
    sp_phaseA_epilogue(net, st, L, k, u.s, u.idx, acc, st.ctr[1] & 1, init);
}

// Phase B (row pass over hidden layers) at the current primal iterate: the oracle mask I*
// (eq. 3), the gradients of beta_0, beta_1, beta_I* (eq. 9 with B = E), the conditional
// gradients alpha_bar (eq. 11) and beta_bar (eq. 12), the convex combination of alpha, Sb, G, C
// (Alg. 2), and the output record for phase C and the next phase A.
__global__ void __launch_bounds__(CB_THREADS) k_sp_rowB_t(DNet net, DState st, DSched sc, TSegs sg) {
    const int q = tseg_of(sg, blockIdx.x);
    const DLayer& L = net.L[sg.layer[q]];
    const Unit u = team_unit(sg, q, L.n_out, net.S);
    const int s = u.s, i = u.idx;
    const int t = st.ctr[1];
    const int cur = t & 1;
    const size_t NT = net.NT, NH = net.NH;
    const size_t h = (size_t)s * NH + L.h_out + i;
    const float z = u.valid ? st.spz[cur][h] : 0.f;
    float a0 = 0.f, A = 0.f, Lam = 0.f, Mu = 0.f;
    int nout = 0;   // pairs with I = 0 (a nonzero weight on a free input)
    if (u.valid) {
        int g, base;
        row_group(L, i, g, base);
        const float4* rb = sp_iplane(net, st, L, s) + base;
        const float4* rn = rb + L.xpos;
        const int t0 = L.rgrp[2 * g], t1 = L.rgrp[2 * g + 1], t2 = L.rgrp[2 * g + 2];
        // {x, threshold, Lcheck, Ucheck} of the tap's sign: the first plane for W > 0, the second
        // for W < 0; I = [z >= threshold] (fixed inputs and padding: always 1)
        constexpr int B = 8;
        for (int ph = 0; ph < 2; ++ph) {
            const float4* rp = ph ? rn : rb;
            const int ta = ph ? t1 : t0, tb = ph ? t2 : t1;
            for (int tt = ta + u.lane; tt < tb; tt += B * u.T) {
                int2 e[B];
                load_taps<B>(L.rtap, tt, tb, u.T, e);
                float4 r[B];
#pragma unroll
                for (int q = 0; q < B; ++q) r[q] = rp[e[q].x];
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    const float w = __int_as_float(e[q].y);
                    const float wx = w * r[q].x;
                    a0 += wx;
                    // a padding tap (w = 0) adds nothing and counts as selected
                    const bool I = z >= r[q].y || w == 0.f;
                    A += I ? wx : 0.f;
                    Lam += I ? w * r[q].z : 0.f;
                    Mu += I ? 0.f : w * r[q].w;
                    nout += I ? 0 : 1;
                }
            }
        }
    }
    if (u.T > 1) {
        a0 = team_sum(a0, u.T);
        A = team_sum(A, u.T);
        Lam = team_sum(Lam, u.T);
        Mu = team_sum(Mu, u.T);
        for (int o = u.T >> 1; o > 0; o >>= 1) nout += __shfl_xor_sync(0xffffffffu, nout, o);
    }
    if (!u.valid || u.lane != 0) return;
    // a row selecting none or all of its free inputs is the all-zero / all-ones constraint, a
    // looser copy of beta_0 / beta_1: it does not compete in the choice of eq. (12)
    const bool degenerate = nout == 0 || nout == st.nfree[h];
    const float gamma = 1.f / ((float)t + sc.gamma0);
    const float bi = L.b[i];
    const float xhat = a0 + bi;
    const float x = st.spx[cur][(size_t)s * NT + L.out_off + i];
    const float uh = st.uhat[h], lh = st.lhat[h];
    const float abar = (xhat - x >= 0.f) ? st.mua[h] : 0.f;
    const float v0 = x - z * uh;
    const float v1 = x - xhat + (1.f - z) * lh;
    const float vI = x - A + (1.f - z) * Lam - z * (bi + Mu);
    int sel = 0;
    float vm = v0;
    if (v1 > vm) { sel = 1; vm = v1; }
    if (!degenerate && vI > vm) { sel = 2; vm = vI; }
    const bool on = vm >= 0.f;
    const float bb = on ? st.mub[h] : 0.f;
    const float gsel = sel == 0 ? uh : (sel == 1 ? lh : Lam + Mu + bi);
    const float csel = sel == 0 ? 0.f : (sel == 1 ? lh - bi : Lam);
    const float om = 1.f - gamma;
    const float an = om * st.alpha[h] + gamma * abar;
    st.alpha[h] = an;
    st.Sb[h] = om * st.Sb[h] + gamma * bb;
    st.G[h] = om * st.G[h] + gamma * (bb * gsel);
    st.C[h] = om * st.C[h] + gamma * (bb * csel);
    st.sel[h] = on ? (uint8_t)sel : (uint8_t)3;
    *sp_orec(net, st, L, s, i) = make_float4(an, sel == 1 ? bb : 0.f, sel == 2 ? bb : 0.f, z);
}

// Phase C of iteration t fused with phase A of iteration t + 1 (col pass over k = 1..n): one walk
// over the output records {alpha, beta_bar on beta_1, beta_bar on I*, z} gives both
// P_bar_k = (W_k o I_dagger)^T beta_bar for input j (the masked backward product of the chosen
// masks) and (W_k^T alpha_k)[j] at the updated alpha. The epilogue takes the convex combination of
// P_k and of the primal iterate (x_m, z_m) into the other buffer (Alg. 2), then runs phase A at
// the new iterate. The launch after it (k_advance) advances the iteration counter.
__global__ void __launch_bounds__(CB_THREADS) k_sp_colCA_t(DNet net, DState st, DSched sc, TSegs sg) {
    const int q = tseg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    const DLayer& L = net.L[li];
    const int k = li + 1, m = k - 1;
    const Unit u = team_unit(sg, q, L.n_in, net.S);
    const int t = st.ctr[1];
    const size_t NT = net.NT, NH = net.NH;
    const size_t xo = (size_t)u.s * NT + L.in_off + u.idx;
    float accC = 0.f, accA = 0.f;
    if (u.valid && k <= net.n - 1) {
        const float4* own = sp_iplane(net, st, L, u.s) + xin_pos(L, u.idx);
        const float tp = own[0].y, tn = own[L.xpos].y;
        int g, base;
        col_group(L, u.idx, g, base);
        const float4* ar = arec_planes(net, st, L, u.s) + base;
        const int t0 = L.cgrp[2 * g], t1 = L.cgrp[2 * g + 1], t2 = L.cgrp[2 * g + 2];
        constexpr int B = 8;
        for (int ph = 0; ph < 2; ++ph) {
            const int ta = ph ? t1 : t0, tb = ph ? t2 : t1;
            const float tau = ph ? tn : tp;
            for (int tt = ta + u.lane; tt < tb; tt += B * u.T) {
                int2 e[B];
                load_taps<B>(L.ctap, tt, tb, u.T, e);
                float4 v[B];
#pragma unroll
                for (int q = 0; q < B; ++q) v[q] = ar[e[q].x];
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    const float w = __int_as_float(e[q].y);
                    accC = fmaf(w, v[q].y + (v[q].w >= tau ? v[q].z : 0.f), accC);
                    accA = fmaf(w, v[q].x, accA);
                }
            }
        }
    }
    if (u.T > 1) {
        accC = team_sum(accC, u.T);
        accA = team_sum(accA, u.T);
    }
    if (u.valid && u.lane == 0) {
        const int cur = t & 1, nxt = cur ^ 1;
        const float gamma = 1.f / ((float)t + sc.gamma0);
        const float om = 1.f - gamma;
        if (k <= net.n - 1) st.P[xo] = om * st.P[xo] + gamma * accC;
        st.spx[nxt][xo] = om * st.spx[cur][xo] + gamma * st.xbar[xo];
        if (m >= 1) {
            const size_t hh = (size_t)u.s * NH + L.h_in + u.idx;
            st.spz[nxt][hh] = om * st.spz[cur][hh] + gamma * (st.zbar[hh] ? 1.f : 0.f);
        }
        sp_phaseA_epilogue(net, st, L, k, u.s, u.idx, accA, nxt, 0);
    }
}

// Saddle Point's start (eq. 10): P_k[j] = (W_k^T beta_{k,1})[j] + sum_b ((W_k o I_b)^T beta_{k,b})[j]
// of the Active Set duals, for the inputs j of every hidden-output layer k, by lane teams over
// each input's fan-out (the col pass's geometry); the slot masks from the snapshot bits (eq. 3 at
// the snapshot points).
__global__ void __launch_bounds__(CB_THREADS) k_sp_convert_P_t(DNet net, DState st, DSched sc, TSegs sg) {
    const int q = tseg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    if (li >= net.n - 1) return;   // the output layer's inputs carry no P (whole block)
    const DLayer& L = net.L[li];
    const Unit u = team_unit(sg, q, L.n_in, net.S);
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    const int nsl = u.valid ? min(sp.nadd_before, st.caps[u.s]) : 0;
    const int bo = sp.nadd_before & 1;
    const size_t xo = (size_t)u.s * net.NT + L.in_off + u.idx;
    float acc = 0.f;
    if (u.valid) {
        const unsigned xs = st.xsnap[bo][xo];
        const bool fixed = st.lo[xo] == st.hi[xo];
        const size_t rb = (size_t)u.s * net.NH + L.h_out;
        const float* b1 = st.beta1 + rb;
        const float* bsl = st.bs + (size_t)u.s * net.cap * net.NH + L.h_out;
        const uint8_t* zs = st.zsnap[bo] + rb;
        const bool interior = net.ball && L.in_off == 0;
        col_walk_team(L, u.idx, u.lane, u.T, [&](int i, float w) {
            float sb = b1[i];
            if (nsl) {
                const unsigned I = cb_slot_mask(zs[i], xs, fixed, w, interior);
                for (int b = 0; b < nsl; ++b)
                    if ((I >> b) & 1u) sb += bsl[(size_t)b * net.NH + i];
            }
            acc += w * sb;
        });
    }
    if (u.T > 1) acc = team_sum(acc, u.T);
    if (u.valid && u.lane == 0) st.P[xo] = acc;
}

// Primal initialisation (App. C.2, Big-M variables), row pass: inner maximisers at (x, z).
__global__ void __launch_bounds__(CB_THREADS) k_spi_row_t(DNet net, DState st, TSegs sg) {
    const int q = tseg_of(sg, blockIdx.x);
    const DLayer& L = net.L[sg.layer[q]];
    const Unit u = team_unit(sg, q, L.n_out, net.S);
    const int cur = st.ctr[1] & 1;
    const size_t NT = net.NT, NH = net.NH;
    float a0 = 0.f;
    if (u.valid) {
        const float* xv = st.spx[cur] + (size_t)u.s * NT + L.in_off;
        row_walk_team(L, u.idx, u.lane, u.T, [&](int j, float w) { a0 += w * xv[j]; });
    }
    if (u.T > 1) a0 = team_sum(a0, u.T);
    if (!u.valid || u.lane != 0) return;
    const size_t h = (size_t)u.s * NH + L.h_out + u.idx;
    const float xhat = a0 + L.b[u.idx];
    const float x = st.spx[cur][(size_t)u.s * NT + L.out_off + u.idx];
    const float z = st.spz[cur][h];
    const float ab = (xhat - x >= 0.f) ? st.mua[h] : 0.f;
    const float v0 = x - z * st.uhat[h];
    const float v1 = x - xhat + (1.f - z) * st.lhat[h];
    const bool on = fmaxf(v0, v1) >= 0.f;
    const bool p0 = v0 >= v1;
    const float b0 = (on && p0) ? st.mub[h] : 0.f;
    const float b1 = (on && !p0) ? st.mub[h] : 0.f;
    st.ab[h] = ab;
    st.b0i[h] = b0;
    st.b1i[h] = b1;
    st.arow[h] = ab - b1;
}

// Primal initialisation, col pass: x_m += eta f_m(alpha*, beta*), z_m += eta g_m(beta*),
// projected on the boxes (the primal view's subgradient in x_m is -f_m).
__global__ void __launch_bounds__(CB_THREADS) k_spi_col_t(DNet net, DState st, DSched sc, TSegs sg) {
    const int q = tseg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    const DLayer& L = net.L[li];
    const int k = li + 1, m = k - 1;
    const Unit u = team_unit(sg, q, L.n_in, net.S);
    const int step = st.ctr[2];
    const size_t NT = net.NT, NH = net.NH;
    float acc = 0.f;
    if (u.valid && k <= net.n - 1) {
        const float* ar = st.arow + (size_t)u.s * NH + L.h_out;
        col_walk_team(L, u.idx, u.lane, u.T, [&](int i, float w) { acc += w * ar[i]; });
    }
    if (u.T > 1) acc = team_sum(acc, u.T);
    if (u.valid && u.lane == 0) {
        const int cur = st.ctr[1] & 1;
        const float eta = sc.sp_lr0 + (sc.sp_lr1 - sc.sp_lr0) * (float)step / (float)max(1, sc.sp_init_steps - 1);
        float f = k <= net.n - 1 ? -acc : -net.Wout[(size_t)u.s * L.n_in + u.idx];
        const size_t xo = (size_t)u.s * NT + L.in_off + u.idx;
        if (m >= 1) {
            const size_t h = (size_t)u.s * NH + L.h_in + u.idx;
            f += st.ab[h] - st.b0i[h] - st.b1i[h];
            const float g = st.b0i[h] * st.uhat[h] + st.b1i[h] * st.lhat[h];
            st.spz[cur][h] = fminf(fmaxf(st.spz[cur][h] + eta * g, 0.f), 1.f);
        }
        if (net.ball && L.in_off == 0)   // over an ellipsoid, k_ball_retract brings x_0 back into it
            st.spx[cur][xo] = st.spx[cur][xo] + eta * f;
        else
            st.spx[cur][xo] = fminf(fmaxf(st.spx[cur][xo] + eta * f, st.lo[xo]), st.hi[xo]);
    }
}

// Saddle Point over the ellipsoid input set, one block per subproblem after each phase A: the
// conditional gradient x_bar_0 = c + e^2 f_0 / |e f_0|_2 and its closed-form bound term (as
// k_ball_x0); at the start (init) the primal iterate x_0 takes x_bar_0 and its phase-B records.
__global__ void __launch_bounds__(CB_BALL_THREADS) k_ball_sp(DNet net, DState st, int init) {
    const int s = blockIdx.x;
    const DLayer& L = net.L[0];
    const size_t base = (size_t)s * net.NT + L.in_off;
    float p2 = 0.f, pc = 0.f;
    for (int j = threadIdx.x; j < L.n_in; j += CB_BALL_THREADS) {
        const float lo = st.lo[base + j], hi = st.hi[base + j], f = st.fval[base + j];
        const float ef = 0.5f * (hi - lo) * f;
        p2 = fmaf(ef, ef, p2);
        pc = fmaf(f, 0.5f * (lo + hi), pc);
    }
    __shared__ double red[2][CB_BALL_THREADS / 32];
    const double a2 = warp_sum((double)p2), ac = warp_sum((double)pc);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a2;
        red[1][threadIdx.x >> 5] = ac;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < CB_BALL_THREADS / 32 ? red[0][threadIdx.x] : 0.0;
        double w = threadIdx.x < CB_BALL_THREADS / 32 ? red[1][threadIdx.x] : 0.0;
        v = warp_sum(v);
        w = warp_sum(w);
        if (threadIdx.x == 0) {
            red[0][0] = v;
            red[1][0] = w;
        }
    }
    __syncthreads();
    const double nrm = sqrt(red[0][0]);
    const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
    if (threadIdx.x == 0) st.terms[base] = -red[1][0] - nrm;
    const int cur = st.ctr[1] & 1;
    for (int j = threadIdx.x; j < L.n_in; j += CB_BALL_THREADS) {
        const size_t xo = base + j;
        const float lo = st.lo[xo], hi = st.hi[xo];
        const float c = 0.5f * (lo + hi), e = 0.5f * (hi - lo);
        const float xb = fminf(fmaxf(c + e * e * st.fval[xo] * inv, lo), hi);
        st.xbar[xo] = xb;
        if (j) st.terms[xo] = 0.0;
        if (init) {
            st.spx[cur][xo] = xb;
            float tp = -INFINITY, tn = -INFINITY;
            if (lo != hi) {
                tp = cb_tau_up(xb, lo, lo, hi);
                tn = cb_tau_up(hi, xb, lo, hi);
            }
            float4* r = sp_iplane(net, st, L, s) + xin_pos(L, j);
            r[0] = make_float4(xb, tp, lo, hi);
            r[L.xpos] = make_float4(xb, tn, hi, lo);
        }
    }
}

// After a primal-initialisation step over an ellipsoid: x_0 <- c + (x_0 - c) / max(1, r) with
// r = |(x_0 - c) / e|_2 over the free inputs (fixed ones stay at c), one block per subproblem: the
// exact projection when the half-widths are equal, a point of the ellipsoid for any of them.
__global__ void __launch_bounds__(CB_BALL_THREADS) k_ball_retract(DNet net, DState st) {
    const int s = blockIdx.x;
    const DLayer& L = net.L[0];
    const size_t base = (size_t)s * net.NT + L.in_off;
    float* x = st.spx[st.ctr[1] & 1] + base;
    float p = 0.f;
    for (int j = threadIdx.x; j < L.n_in; j += CB_BALL_THREADS) {
        const float lo = st.lo[base + j], hi = st.hi[base + j];
        if (lo != hi) {
            const float q = (x[j] - 0.5f * (lo + hi)) / (0.5f * (hi - lo));
            p = fmaf(q, q, p);
        }
    }
    __shared__ double red[CB_BALL_THREADS / 32];
    const double a = warp_sum((double)p);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < CB_BALL_THREADS / 32 ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const float scale = (float)(1.0 / fmax(1.0, sqrt(red[0])));
    for (int j = threadIdx.x; j < L.n_in; j += CB_BALL_THREADS) {
        const float lo = st.lo[base + j], hi = st.hi[base + j], c = 0.5f * (lo + hi);
        x[j] = lo != hi ? fminf(fmaxf(c + (x[j] - c) * scale, lo), hi) : c;
    }
}

}  // namespace cb

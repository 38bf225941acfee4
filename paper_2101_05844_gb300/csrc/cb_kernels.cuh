// Kernels of the convex-barrier library: interval bounds, Big-M / Active Set iterations,
// Saddle Point iterations and the bound reduction, for linear and conv2d layers.
//
// Two access patterns cover every product of the method:
//  * row pass  (one warp per subproblem and output neuron i): reductions over the fan-in of i,
//    i.e. W x, (W o I) x and mask row sums (eq. 9, the forward products);
//  * col pass  (one thread per subproblem and input neuron j): reductions over the fan-out of j,
//    i.e. W^T a and (W o I)^T a (f_k of eq. 6, the backward products).
// Masks are never stored per (i, j). For every (i, j) the masks of all active-set slots form a
// bitset in a register, computed from per-neuron snapshot bytes (Active Set) or per-input
// thresholds (Saddle Point); see cb_slot_mask and cb_sp_mask.
#pragma once
#include "cb_common.cuh"
#include "cb_walk.cuh"

namespace cb {

// Active Set mask bits of every slot for one (i, j) pair (eq. 3 at binary iterates).
// zs: bit b = z*_k[i] when slot b was added; xs: bit b = (x*_{k-1}[j] was at its upper bound).
// With z = 1 the row is all ones; with z = 0 the bit is 1 where the coefficient
// ((1-z) Lcheck + z Ucheck - x) W is >= 0: W > 0 and x at its lower bound, W < 0 and x at its
// upper bound, W = 0, or l = u (fixed input, coefficient exactly 0). An input strictly inside its
// box (interior: layer 0 over an ellipsoid) is at neither end: the bit is z, or 1 where W = 0 or l = u.
__device__ __forceinline__ unsigned cb_slot_mask(unsigned zs, unsigned xs, bool fixed, float w,
                                                 bool interior = false) {
    unsigned xm = fixed ? 0xFFu
                        : (w > 0.f ? (interior ? 0u : (~xs & 0xFFu)) : (w < 0.f ? (interior ? 0u : xs) : 0xFFu));
    return zs | xm;
}

// Saddle Point oracle bit, eq. (3) with continuous (x, z), in the threshold form: W > 0 ->
// z (u - l) >= x - l, W < 0 -> z (u - l) >= u - x (eq. 3 with the sign of W multiplied out), i.e.
// z >= tau for tau = (x - l) / (u - l), resp. (u - x) / (u - l); W = 0 or l = u -> 1 (fixed inputs
// carry thresholds of -inf). The thresholds are cb_tau_up's, so each float32 compare is exact.
__device__ __forceinline__ bool cb_sp_mask(float z, float tp, float tn, float w) {
    return w > 0.f ? (z >= tp) : (w < 0.f ? (z >= tn) : true);
}

// The smallest float32 at or above the real quotient (a - b) / (hi - lo), for float32 a, b, lo <
// hi: the differences are exact in float64 (float32 operands whose magnitudes lie within 2^28 of
// each other), the quotient is rounded up in float64 and again to float32. Rounding up twice
// gives the float32 rounding up of the real quotient (a float32 is a float64), so for every
// float32 z, z >= tau (real) exactly when z >= this value: the mask decision of eq. (3) is exact.
__device__ __forceinline__ float cb_tau_up(float a, float b, float lo, float hi) {
    return __double2float_ru(__ddiv_ru((double)a - (double)b, (double)hi - (double)lo));
}

// Block-to-segment lookup for launches that cover several layers.
struct Segs {
    int n;
    int layer[CB_MAXL];   // 0-based layer index
    int start[CB_MAXL + 1];
};
__device__ __forceinline__ int seg_of(const Segs& sg, int blk) {
    int q = 0;
    while (q + 1 < sg.n && blk >= sg.start[q + 1]) ++q;
    return q;
}

// Advances the iteration counter ctr[i] (0: Active Set, 1: Saddle Point, 2: primal
// initialisation) after the launch that completes an iteration: stream order has every block of
// that launch done before it, and the next launches read the new value.
__global__ void k_advance(int* ctr, int i) { ctr[i] += 1; }

// 1 / (1 - beta^step), the Adam bias corrections, from a table built in FP64 on the host.
__device__ __forceinline__ float inv_bias_corr(const float* tab, int ntab, int step, float beta) {
    return step < ntab ? tab[step] : 1.f / (1.f - powf(beta, (float)step));
}

// One projected Adam ascent step (Kingma and Ba) of a dual variable: returns the new value and
// updates the moments. Fast reciprocal square root and division (a few float32 ulps).
__device__ __forceinline__ float adam_step(float th, float& m, float& v, float g, float lr, float ibc1,
                                           float ibc2, const DSched& sc) {
    m = sc.b1 * m + sc.omb1 * g;
    v = sc.b2 * v + sc.omb2 * g * g;
    const float mh = m * ibc1, vh = v * ibc2;
    const float sq = vh > 0.f ? vh * rsqrtf(vh) : 0.f;
    return fmaxf(th + lr * __fdividef(mh, sq + sc.eps), 0.f);
}

// ------------------------------------------------------------------------- interval bounds
// Interval propagation for hidden layer L (App. E): lhat = W+ l + W- u + b, uhat = W+ u + W- l + b
// accumulated to float64 accuracy (compensated float32 lanes, CompSum), rounded outward to
// float32; splits clamp straddling neurons; then the post-activation box max(., 0). Over an
// ellipsoid (layer 1 of an l2-ball input set) the centre product and the radius in float64.
__global__ void k_ibp(DNet net, DState st, int li, const signed char* splits) {
    const DLayer& L = net.L[li];
    const int warp = (blockIdx.x * CB_THREADS + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= net.S * L.n_out) return;
    const int s = warp / L.n_out, i = warp - s * L.n_out;
    const float* lo = st.lo + (size_t)s * net.NT + L.in_off;
    const float* hi = st.hi + (size_t)s * net.NT + L.in_off;
    double a = 0.0, c = 0.0;
    int nf = 0;
    const bool ell = net.ball && li == 0;
    if (ell) {
        row_walk(L, i, lane, [&](int j, float w) {   // centre product and squared radius of W_i
            const double wd = w, e = 0.5 * ((double)hi[j] - (double)lo[j]);
            a += wd * 0.5 * ((double)lo[j] + (double)hi[j]);
            c += wd * wd * e * e;
            nf += (w != 0.f && lo[j] != hi[j]) ? 1 : 0;
        });
        a = warp_sum(a);
        c = warp_sum(c);
    } else {
        CompSum ca, cc;
        row_walk(L, i, lane, [&](int j, float w) {
            const float l = lo[j], u = hi[j];
            ca.add_prod(w, w >= 0.f ? l : u);
            cc.add_prod(w, w >= 0.f ? u : l);
            nf += (w != 0.f && l != u) ? 1 : 0;
        });
        a = ca.warp_total();
        c = cc.warp_total();
    }
    for (int o = 16; o > 0; o >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, o);
    if (lane == 0 && !ell) {
        // the row constants of the batch, the same sums before the bias (k_lz computes them alone
        // for caller-given bounds and over an ellipsoid's layer 1)
        const size_t h = (size_t)s * net.NH + L.h_out + i;
        st.lz[h] = (float)a;
        st.uz[h] = (float)c;
        st.nfree[h] = nf;
    }
    if (lane == 0) {
        if (ell) {   // the exact range of W_i x + b over {sum ((x - c) / e)^2 <= 1}: W_i c + b -+ |W_i D|
            const double r = sqrt(c);
            st.brad[(size_t)s * net.NH + L.h_out + i] = (float)r;
            c = a + r;
            a = a - r;
        }
        a += (double)L.b[i];
        c += (double)L.b[i];
        const size_t h = (size_t)s * net.NH + L.h_out + i;
        if (splits) {
            const signed char sp = splits[h];
            if (a < 0.0 && c > 0.0) {
                if (sp > 0) a = 0.0;
                if (sp < 0) c = 0.0;
            }
        }
        const float lh = __double2float_rd(a), uh = __double2float_ru(c);
        st.lhat[h] = lh;
        st.uhat[h] = uh;
        const size_t o = (size_t)s * net.NT + L.out_off + i;
        st.lo[o] = fmaxf(lh, 0.f);
        st.hi[o] = fmaxf(uh, 0.f);
    }
}

__global__ void k_fill(double* p, size_t n, double v) {
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) p[u] = v;
}
__global__ void k_fill_int(int* p, size_t n, int v) {
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) p[u] = v;
}

// Device-side check of a box given on the device: sets the status word if lo > hi or non-finite.
__global__ void k_check_box(DNet net, DState st) {
    const int n0 = net.L[0].n_in;
    const size_t n = (size_t)net.S * n0;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const size_t s = u / n0, j = u - s * n0;
        const float l = st.lo[s * net.NT + j], h = st.hi[s * net.NT + j];
        if (!(l <= h) || !isfinite(l) || !isfinite(h)) atomicOr(st.status, 1);
    }
}

// Post-activation box from caller-supplied pre-activation bounds.
__global__ void k_post_from_pre(DNet net, DState st) {
    const size_t n = (size_t)net.S * net.NH;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(u / net.NH), h = (int)(u - (size_t)s * net.NH);
        const int off0 = net.L[0].n_in;   // hidden neurons follow the input layer in [NT]
        st.lo[(size_t)s * net.NT + off0 + h] = fmaxf(st.lhat[u], 0.f);
        st.hi[(size_t)s * net.NT + off0 + h] = fmaxf(st.uhat[u], 0.f);
    }
}

// Property-folded output row: Wout[s] = C[s]^T W_n, bout[s] = C[s] . b_n (FP64 accumulation).
// Property rows folded into the last layer: Wout[s] = C_s^T W_n, bout[s] = C_s^T b_n (FP64 sums
// rounded to float32). One block per subproblem: warp 0 first lists the row's nonzero entries in
// order (ballots over chunks of 32), so that rows like +-e_i cost one term per input; a row with
// more than CB_FOLD_NZ nonzeros takes the dense sum.
#define CB_FOLD_NZ 256
__global__ void k_fold(DNet net, const float* Wlast, const float* blast, const float* C, int n_out,
                       float* Wout, float* bout) {
    __shared__ int nz_o[CB_FOLD_NZ];
    __shared__ double nz_c[CB_FOLD_NZ];
    __shared__ int nnz;
    const int nin = net.L[net.n - 1].n_in;
    const int s = blockIdx.x;
    if (threadIdx.x < 32) {
        int cnt = 0;
        for (int o0 = 0; o0 < n_out; o0 += 32) {
            const int o = o0 + (int)threadIdx.x;
            const double c = o < n_out ? (C ? (double)C[(size_t)s * n_out + o] : 1.0) : 0.0;
            const unsigned m = __ballot_sync(0xffffffffu, c != 0.0);
            const int pos = cnt + __popc(m & ((1u << threadIdx.x) - 1u));
            if (c != 0.0 && pos < CB_FOLD_NZ) {
                nz_o[pos] = o;
                nz_c[pos] = c;
            }
            cnt += __popc(m);
        }
        if (threadIdx.x == 0) nnz = cnt;
    }
    __syncthreads();
    const int k = nnz;
    for (int j = threadIdx.x; j <= nin; j += blockDim.x) {
        double a = 0.0;
        if (k <= CB_FOLD_NZ) {
            for (int q = 0; q < k; ++q)
                a += nz_c[q] * (j < nin ? (double)Wlast[(size_t)nz_o[q] * nin + j] : (double)blast[nz_o[q]]);
        } else {
            for (int o = 0; o < n_out; ++o) {
                const double c = C ? (double)C[(size_t)s * n_out + o] : 1.0;
                a += c * (j < nin ? (double)Wlast[(size_t)o * nin + j] : (double)blast[o]);
            }
        }
        if (j < nin) Wout[(size_t)s * nin + j] = (float)a;
        else bout[s] = (float)a;
    }
}

// ------------------------------------------------------------------------- bound reduction
// d[s] = bout[s] + sum of the per-neuron terms (eq. 6), in a fixed order (deterministic).
// precision 64: FP64 sum; 32: float32 sum. keep_best: best[s] = max(best[s], d[s]).
__global__ void k_reduce(DNet net, DState st, int precision, double* out, int keep_best) {
    const int s = blockIdx.x;
    const double* t = st.terms + (size_t)s * net.NT;
    __shared__ double sd[CB_THREADS];
    __shared__ float sf[CB_THREADS];
    double a = 0.0;
    float af = 0.f;
    for (int j = threadIdx.x; j < net.NT; j += CB_THREADS) {
        a += t[j];
        af += (float)t[j];
    }
    sd[threadIdx.x] = a;
    sf[threadIdx.x] = af;
    __syncthreads();
    for (int w = CB_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sd[threadIdx.x] += sd[threadIdx.x + w];
            sf[threadIdx.x] += sf[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double d = precision == 32 ? (double)(sf[0] + net.bout[s]) : sd[0] + (double)net.bout[s];
        if (out) out[s] = d;
        if (keep_best && !(d <= st.best[s])) st.best[s] = d;
    }
}

// ------------------------------------------------------------------- Saddle Point: convert
// Sufficient statistics of the current Active Set duals (Sec. 5.1), hidden elementwise part:
// Sb = beta0 + beta1 + sum_b beta_b, G = g, C = beta1 (lhat - b) + sum_b beta_b lambda_b, and the
// price caps of eq. (16).
__global__ void k_sp_convert_elem(DNet net, DState st, DSched sc, float c_alpha, float c_beta) {
    const size_t n = (size_t)net.S * net.NH;
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(u / net.NH), hh = (int)(u - (size_t)s * net.NH);
        int li = 0;
        while (li + 1 < net.n - 1 && hh >= net.L[li + 1].h_out) ++li;
        const float bi = net.L[li].b[hh - net.L[li].h_out];
        const int nsl = min(sp.nadd_before, st.caps[s]);
        float Sb = st.beta0[u] + st.beta1[u];
        float G = st.beta0[u] * st.uhat[u] + st.beta1[u] * st.lhat[u];
        float C = st.beta1[u] * (st.lhat[u] - bi);
        for (int b = 0; b < nsl; ++b) {
            const size_t hs = ((size_t)s * net.cap + b) * net.NH + hh;
            const float bb = st.bs[hs];
            Sb += bb;
            G += bb * st.kap[hs];
            C += bb * st.lam[hs];
        }
        st.Sb[u] = Sb;
        st.G[u] = G;
        st.C[u] = C;
        const float a = st.alpha[u];
        st.mua[u] = a > 0.f ? a : c_alpha;
        st.mub[u] = Sb > 0.f ? Sb : c_beta;
    }
}

}  // namespace cb

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
// upper bound, W = 0, or l = u (fixed input, coefficient exactly 0).
__device__ __forceinline__ unsigned cb_slot_mask(unsigned zs, unsigned xs, bool fixed, float w) {
    unsigned xm = fixed ? 0xFFu : (w > 0.f ? (~xs & 0xFFu) : (w < 0.f ? xs : 0xFFu));
    return zs | xm;
}

// Saddle Point oracle bit, eq. (3) with continuous (x, z), in the threshold form decided in
// float32: W > 0 -> z >= (x - l)/(u - l); W < 0 -> z >= (u - x)/(u - l); W = 0 or l = u -> 1
// (fixed inputs carry thresholds of -inf).
__device__ __forceinline__ bool cb_sp_mask(float z, float tp, float tn, float w) {
    return w > 0.f ? (z >= tp) : (w < 0.f ? (z >= tn) : true);
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

// Last block of a launch: every block calls this at exit; returns true in exactly one block,
// after every other block of the launch has finished its writes.
__device__ __forceinline__ bool last_block(unsigned* counter) {
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    return is_last;
}

__device__ __forceinline__ float bias_corr(const float* tab, int ntab, int step, float beta) {
    return step < ntab ? tab[step] : 1.f - powf(beta, (float)step);
}

__device__ __forceinline__ void adam(float& th, float& m, float& v, float g, float lr, float bc1,
                                     float bc2, const DSched& sc) {
    m = sc.b1 * m + sc.omb1 * g;
    v = sc.b2 * v + sc.omb2 * g * g;
    const float mh = m / bc1, vh = v / bc2;
    th = fmaxf(th + lr * mh / (sqrtf(vh) + sc.eps), 0.f);
}

// ------------------------------------------------------------------------- interval bounds
// Interval propagation for hidden layer L (App. E): lhat = W+ l + W- u + b, uhat = W+ u + W- l + b
// accumulated in FP64, rounded outward to float32; splits clamp straddling neurons; then the
// post-activation box max(., 0).
__global__ void k_ibp(DNet net, DState st, int li, const signed char* splits) {
    const DLayer& L = net.L[li];
    const int warp = (blockIdx.x * CB_THREADS + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= net.S * L.n_out) return;
    const int s = warp / L.n_out, i = warp - s * L.n_out;
    const float* lo = st.lo + (size_t)s * net.NT + L.in_off;
    const float* hi = st.hi + (size_t)s * net.NT + L.in_off;
    double a = 0.0, c = 0.0;
    row_walk(L, i, lane, [&](int j, float w) {
        const double wd = w;
        if (w >= 0.f) { a += wd * lo[j]; c += wd * hi[j]; }
        else { a += wd * hi[j]; c += wd * lo[j]; }
    });
    a = warp_sum(a);
    c = warp_sum(c);
    if (lane == 0) {
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
__global__ void k_fold(DNet net, const float* Wlast, const float* blast, const float* C, int n_out,
                       float* Wout, float* bout) {
    const int nin = net.L[net.n - 1].n_in;
    const size_t n = (size_t)net.S * (nin + 1);
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(u / (nin + 1)), j = (int)(u - (size_t)s * (nin + 1));
        double a = 0.0;
        for (int o = 0; o < n_out; ++o) {
            const double c = C ? (double)C[(size_t)s * n_out + o] : 1.0;
            a += c * (j < nin ? (double)Wlast[(size_t)o * nin + j] : (double)blast[o]);
        }
        if (j < nin) Wout[(size_t)s * nin + j] = (float)a;
        else bout[s] = (float)a;
    }
}

// ------------------------------------------------------------- Big-M / Active Set: phase A
// Col pass over layers k = 1..n. For input neuron j of layer k (neuron j of layer m = k-1):
//   f_m[j] = alpha_m - beta0 - beta1 - sum_b beta_b                         (m >= 1)
//            - (W_k^T (alpha_k - beta1_k))[j] + sum_b ((W_k o I_b)^T beta_b)[j]   (k <= n-1)
//            - Wout[j]                                                      (k = n, alpha_n = 1)
// (f of Sec. 4.1), the closed-form minimiser x*_m = u if f >= 0 else l (eqs. 7-8), and for
// m >= 1: g_m = beta0 uhat + beta1 lhat + sum_b beta_b kappa_b, z* = [g >= 0]. Writes the
// per-neuron bound terms of eq. (6). On addition iterations (mode 0) also records x*, z* into
// the new slot's snapshot bits: the oracle eq. (3) called at (x*, z*) (Alg. 1, Prop. 1).
// mode 0: iteration; mode 1: bound evaluation only.
__global__ void __launch_bounds__(CB_THREADS) k_as_colA(DNet net, DState st, DSched sc, Segs sg, int mode) {
    const int q = seg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    const DLayer& L = net.L[li];
    const int k = li + 1, m = k - 1;
    const int u = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    if (u < net.S * L.n_in) {
        const int s = u / L.n_in, j = u - s * L.n_in;
        const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
        const int cap_s = st.caps[s];
        const int nsl = min(sp.nadd_before, cap_s);
        const int bo = sp.nadd_before & 1;
        const bool add_iter = (mode == 0) && sp.b_new >= 0;
        const bool add = add_iter && sp.b_new < cap_s;
        const size_t NT = net.NT, NH = net.NH, cap = net.cap;
        const size_t xo = (size_t)s * NT + L.in_off + j;
        const float lo = st.lo[xo], hi = st.hi[xo];
        const unsigned xs = st.xsnap[bo][xo];
        float acc0 = 0.f, accM = 0.f;
        if (k <= net.n - 1) {
            const size_t rb = (size_t)s * NH + L.h_out;
            const float* al = st.alpha + rb;
            const float* b1 = st.beta1 + rb;
            const float* bsl = st.bs + (size_t)s * cap * NH + L.h_out;
            const uint8_t* zs = st.zsnap[bo] + rb;
            const bool fixed = lo == hi;
            col_walk(L, j, [&](int i, float w) {
                acc0 += w * (al[i] - b1[i]);
                if (nsl) {
                    const unsigned I = cb_slot_mask(zs[i], xs, fixed, w);
                    float sb = 0.f;
#pragma unroll
                    for (int b = 0; b < CB_MAXCUT; ++b)
                        if (b < nsl && ((I >> b) & 1u)) sb += bsl[(size_t)b * NH + i];
                    accM += w * sb;
                }
            });
        } else {
            acc0 = net.Wout[(size_t)s * L.n_in + j];
        }
        float f = accM - acc0;
        double term = 0.0;
        if (m >= 1) {
            const size_t h = (size_t)s * NH + L.h_in + j;
            const size_t hs = (size_t)s * cap * NH + L.h_in + j;
            float sb = 0.f, gk = st.beta0[h] * st.uhat[h] + st.beta1[h] * st.lhat[h];
            double cterm = 0.0;
#pragma unroll
            for (int b = 0; b < CB_MAXCUT; ++b)
                if (b < nsl) {
                    const float bb = st.bs[hs + (size_t)b * NH];
                    sb += bb;
                    gk += bb * st.kap[hs + (size_t)b * NH];
                    cterm += (double)bb * st.lam[hs + (size_t)b * NH];
                }
            f += st.alpha[h] - st.beta0[h] - st.beta1[h] - sb;
            const bool z = gk >= 0.f;
            st.zcur[h] = z;
            const float bm = net.L[m - 1].b[j];
            term = (double)bm * st.alpha[h] + (double)st.beta1[h] * ((double)st.lhat[h] - bm) + cterm
                   - (z ? (double)gk : 0.0);
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
}

// ------------------------------------------------------------- Big-M / Active Set: phase B
// Row pass over hidden layers. For (s, i) of layer k: xhat = W x* + b and, for every slot b,
// (W o I_b) x*; on addition iterations lambda and kappa of the new slot (mask row sums).
// Supergradient eq. (9), then the Adam ascent step and projection (Alg. 1 lines 10-11).
// The last block advances the iteration counter.
__global__ void __launch_bounds__(CB_THREADS) k_as_rowB(DNet net, DState st, DSched sc, Segs sg) {
    const int q = seg_of(sg, blockIdx.x);
    const DLayer& L = net.L[sg.layer[q]];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = (blockIdx.x - sg.start[q]) * CB_WARPS + wib;
    const int it = st.ctr[0];
    if (u < net.S * L.n_out) {
        const int s = u / L.n_out, i = u - s * L.n_out;
        const Step sp = cb_step(it, sc, st.lr_tab);
        const int cap_s = st.caps[s];
        const int newb = (sp.b_new >= 0 && sp.b_new < cap_s) ? sp.b_new : -1;
        const int nsl = min(sp.nadd_before + (sp.b_new >= 0 ? 1 : 0), cap_s);
        const int bn = (sp.nadd_before + (sp.b_new >= 0 ? 1 : 0)) & 1;
        const size_t NT = net.NT, NH = net.NH, cap = net.cap;
        const size_t h = (size_t)s * NH + L.h_out + i;
        const unsigned zs = st.zsnap[bn][h];
        const float* xv = st.xval + (size_t)s * NT + L.in_off;
        const float* lo = st.lo + (size_t)s * NT + L.in_off;
        const float* hi = st.hi + (size_t)s * NT + L.in_off;
        const uint8_t* xsn = st.xsnap[bn] + (size_t)s * NT + L.in_off;
        float acc0 = 0.f, lamN = 0.f, muN = 0.f;
        float acc[CB_MAXCUT];
#pragma unroll
        for (int b = 0; b < CB_MAXCUT; ++b) acc[b] = 0.f;
        row_walk(L, i, lane, [&](int j, float w) {
            const float x = xv[j];
            const float wx = w * x;
            acc0 += wx;
            if (nsl) {
                const float l = lo[j], uu = hi[j];
                const unsigned I = cb_slot_mask(zs, xsn[j], l == uu, w);
#pragma unroll
                for (int b = 0; b < CB_MAXCUT; ++b)
                    if (b < nsl && ((I >> b) & 1u)) acc[b] += wx;
                if (newb >= 0) {
                    if ((I >> newb) & 1u) lamN += w * (w >= 0.f ? l : uu);
                    else muN += w * (w >= 0.f ? uu : l);
                }
            }
        });
        acc0 = warp_sum(acc0);
#pragma unroll
        for (int b = 0; b < CB_MAXCUT; ++b)
            if (b < nsl) acc[b] = warp_sum(acc[b]);
        if (newb >= 0) { lamN = warp_sum(lamN); muN = warp_sum(muN); }
        const float bi = L.b[i];
        const float xhat = acc0 + bi;
        const float x = st.xval[(size_t)s * NT + L.out_off + i];
        const float z = st.zcur[h] ? 1.f : 0.f;
        const int step = it + 1;
        if (lane == 0) {
            const float bc1 = bias_corr(st.bc1_tab, sc.ntab, step, sc.b1);
            const float bc2 = bias_corr(st.bc2_tab, sc.ntab, step, sc.b2);
            const float ga = xhat - x;
            const float g0 = x - z * st.uhat[h];
            const float g1 = x - xhat + (1.f - z) * st.lhat[h];
            adam(st.alpha[h], st.ma[h], st.va[h], ga, sp.lr, bc1, bc2, sc);
            adam(st.beta0[h], st.m0[h], st.v0[h], g0, sp.lr, bc1, bc2, sc);
            adam(st.beta1[h], st.m1[h], st.v1[h], g1, sp.lr, bc1, bc2, sc);
        } else if (lane - 1 < nsl) {
            const int b = lane - 1;
            const size_t hs = (size_t)s * cap * NH + (size_t)b * NH + L.h_out + i;
            float lam, kap;
            if (b == newb) {
                lam = lamN;
                kap = lamN + muN + bi;
                st.lam[hs] = lam;
                st.kap[hs] = kap;
            } else {
                lam = st.lam[hs];
                kap = st.kap[hs];
            }
            float ab = 0.f;
#pragma unroll
            for (int bb = 0; bb < CB_MAXCUT; ++bb)
                if (bb == b) ab = acc[bb];
            const float gb = x - ab + lam * (1.f - z) - z * (kap - lam);
            const int sstep = sp.t - cb_slot_added_at(b, sc) + 1;
            const float bc1 = bias_corr(st.bc1_tab, sc.ntab, sstep, sc.b1);
            const float bc2 = bias_corr(st.bc2_tab, sc.ntab, sstep, sc.b2);
            adam(st.bs[hs], st.ms[hs], st.vs[hs], gb, sp.lr, bc1, bc2, sc);
        }
    }
    if (last_block(&st.done[0]) && threadIdx.x == 0) {
        st.ctr[0] = it + 1;
        st.done[0] = 0;
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

// P_k[j] = (W_k^T beta1_k)[j] + sum_b ((W_k o I_b)^T beta_b)[j] for hidden layers k (col pass).
__global__ void __launch_bounds__(CB_THREADS) k_sp_convert_P(DNet net, DState st, DSched sc, Segs sg) {
    const int q = seg_of(sg, blockIdx.x);
    const DLayer& L = net.L[sg.layer[q]];
    const int u = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    if (u >= net.S * L.n_in) return;
    const int s = u / L.n_in, j = u - s * L.n_in;
    const Step sp = cb_step(st.ctr[0], sc, st.lr_tab);
    const int nsl = min(sp.nadd_before, st.caps[s]);
    const int bo = sp.nadd_before & 1;
    const size_t NT = net.NT, NH = net.NH;
    const size_t xo = (size_t)s * NT + L.in_off + j;
    const unsigned xs = st.xsnap[bo][xo];
    const bool fixed = st.lo[xo] == st.hi[xo];
    const size_t rb = (size_t)s * NH + L.h_out;
    const float* b1 = st.beta1 + rb;
    const float* bsl = st.bs + (size_t)s * net.cap * NH + L.h_out;
    const uint8_t* zs = st.zsnap[bo] + rb;
    float acc = 0.f;
    col_walk(L, j, [&](int i, float w) {
        float sb = b1[i];
        if (nsl) {
            const unsigned I = cb_slot_mask(zs[i], xs, fixed, w);
            for (int b = 0; b < nsl; ++b)
                if ((I >> b) & 1u) sb += bsl[(size_t)b * NH + i];
        }
        acc += w * sb;
    });
    st.P[xo] = acc;
}

// --------------------------------------------------------------- Saddle Point: phase A
// Col pass over k = 1..n for neuron j of layer m = k-1 at the current (alpha, zeta):
// f_m = alpha_m - Sb_m - W_{m+1}^T alpha_{m+1} + P_{m+1} (Sec. 5.1), the primal conditional
// gradient x_bar, z_bar (eqs. 7-8 with B = E), the bound terms, and the oracle thresholds of
// neuron j at the current primal iterate. init != 0: also start the primal iterate there.
__global__ void __launch_bounds__(CB_THREADS) k_sp_colA(DNet net, DState st, Segs sg, int init) {
    const int q = seg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    const DLayer& L = net.L[li];
    const int k = li + 1, m = k - 1;
    const int u = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    if (u >= net.S * L.n_in) return;
    const int s = u / L.n_in, j = u - s * L.n_in;
    const int cur = st.ctr[1] & 1;
    const size_t NT = net.NT, NH = net.NH;
    const size_t xo = (size_t)s * NT + L.in_off + j;
    float acc = 0.f;
    if (k <= net.n - 1) {
        const float* al = st.alpha + (size_t)s * NH + L.h_out;
        col_walk(L, j, [&](int i, float w) { acc += w * al[i]; });
    } else {
        acc = net.Wout[(size_t)s * L.n_in + j];
    }
    float f = -acc;
    if (k <= net.n - 1) f += st.P[xo];
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
    const float x = init ? xb : st.spx[cur][xo];
    if (init) st.spx[cur][xo] = xb;
    if (lo == hi) {
        st.taup[xo] = -INFINITY;
        st.taun[xo] = -INFINITY;
    } else {
        const float den = __fsub_rn(hi, lo);
        st.taup[xo] = __fdiv_rn(__fsub_rn(x, lo), den);
        st.taun[xo] = __fdiv_rn(__fsub_rn(hi, x), den);
    }
}

// --------------------------------------------------------------- Saddle Point: phase B
// Row pass over hidden layers at the current primal iterate (x^t, z^t): the oracle mask I*
// (eq. 3), the gradients of beta_0, beta_1, beta_I* (eq. 9 with B = E), the dual conditional
// gradients alpha_bar (eq. 11) and beta_bar (eq. 12, ties to the lower index), and the convex
// combination of alpha and of the elementwise statistics Sb, G, C (Alg. 2).
__global__ void __launch_bounds__(CB_THREADS) k_sp_rowB(DNet net, DState st, DSched sc, Segs sg) {
    const int q = seg_of(sg, blockIdx.x);
    const DLayer& L = net.L[sg.layer[q]];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = (blockIdx.x - sg.start[q]) * CB_WARPS + wib;
    if (u >= net.S * L.n_out) return;
    const int s = u / L.n_out, i = u - s * L.n_out;
    const int t = st.ctr[1];
    const int cur = t & 1;
    const float gamma = 1.f / ((float)t + sc.gamma0);
    const size_t NT = net.NT, NH = net.NH;
    const size_t h = (size_t)s * NH + L.h_out + i;
    const float z = st.spz[cur][h];
    const size_t ib = (size_t)s * NT + L.in_off;
    const float* xv = st.spx[cur] + ib;
    const float* lo = st.lo + ib;
    const float* hi = st.hi + ib;
    const float* tp = st.taup + ib;
    const float* tn = st.taun + ib;
    float a0 = 0.f, A = 0.f, Lam = 0.f, Mu = 0.f;
    bool any_in = false, any_out = false;
    row_walk(L, i, lane, [&](int j, float w) {
        const float x = xv[j];
        const float wx = w * x;
        a0 += wx;
        const bool I = cb_sp_mask(z, tp[j], tn[j], w);
        const float l = lo[j], uu = hi[j];
        if (I) {
            A += wx;
            Lam += w * (w >= 0.f ? l : uu);
            any_in |= (w != 0.f) && (l != uu);
        } else {
            Mu += w * (w >= 0.f ? uu : l);
            any_out = true;   // I = 0 only for a nonzero weight on a free input
        }
    });
    // a row selecting none or all of its free inputs (nonzero weight, l < u; a fixed input adds the
    // same term selected or not) is the all-zero / all-ones constraint: a looser copy of the
    // beta_0 / beta_1 constraint, which does not compete in the choice of eq. (12)
    const bool degenerate = !__any_sync(0xffffffffu, any_in) || !__any_sync(0xffffffffu, any_out);
    a0 = warp_sum(a0);
    A = warp_sum(A);
    Lam = warp_sum(Lam);
    Mu = warp_sum(Mu);
    if (lane == 0) {
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
        st.alpha[h] = om * st.alpha[h] + gamma * abar;
        st.Sb[h] = om * st.Sb[h] + gamma * bb;
        st.G[h] = om * st.G[h] + gamma * (bb * gsel);
        st.C[h] = om * st.C[h] + gamma * (bb * csel);
        st.sel[h] = on ? (uint8_t)sel : (uint8_t)3;
    }
}

// --------------------------------------------------------------- Saddle Point: phase C
// Col pass over k = 1..n for neuron j of layer m = k-1: the masked backward product of the
// selected conditional-gradient masks, P_bar_k = (W_k o I_dagger)^T beta_bar (eq. 10's second
// statistic), and the convex combination of P_k and of the primal iterate (x_m, z_m) into the
// other buffer. The last block advances the iteration counter.
__global__ void __launch_bounds__(CB_THREADS) k_sp_colC(DNet net, DState st, DSched sc, Segs sg) {
    const int q = seg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    const DLayer& L = net.L[li];
    const int k = li + 1, m = k - 1;
    const int u = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    const int t = st.ctr[1];
    if (u < net.S * L.n_in) {
        const int s = u / L.n_in, j = u - s * L.n_in;
        const int cur = t & 1, nxt = cur ^ 1;
        const float gamma = 1.f / ((float)t + sc.gamma0);
        const float om = 1.f - gamma;
        const size_t NT = net.NT, NH = net.NH;
        const size_t xo = (size_t)s * NT + L.in_off + j;
        if (k <= net.n - 1) {
            const size_t rb = (size_t)s * NH + L.h_out;
            const uint8_t* sel = st.sel + rb;
            const float* mub = st.mub + rb;
            const float* zr = st.spz[cur] + rb;
            const float tp = st.taup[xo], tn = st.taun[xo];
            float acc = 0.f;
            col_walk(L, j, [&](int i, float w) {
                const int sl = sel[i];
                if (sl == 1 || (sl == 2 && cb_sp_mask(zr[i], tp, tn, w))) acc += w * mub[i];
            });
            st.P[xo] = om * st.P[xo] + gamma * acc;
        }
        st.spx[nxt][xo] = om * st.spx[cur][xo] + gamma * st.xbar[xo];
        if (m >= 1) {
            const size_t hh = (size_t)s * NH + L.h_in + j;
            st.spz[nxt][hh] = om * st.spz[cur][hh] + gamma * (st.zbar[hh] ? 1.f : 0.f);
        }
    }
    if (last_block(&st.done[1]) && threadIdx.x == 0) {
        st.ctr[1] = t + 1;
        st.done[1] = 0;
    }
}

// ------------------------------------------------------ Saddle Point: primal initialisation
// App. C.2, simplified to the Big-M variables. Row pass: inner maximisers at (x, z):
// alpha* = mu_alpha [xhat - x >= 0]; beta0*, beta1* = mu_beta on the larger of their gradients
// (ties to beta0) when it is >= 0.
__global__ void __launch_bounds__(CB_THREADS) k_spi_row(DNet net, DState st, Segs sg) {
    const int q = seg_of(sg, blockIdx.x);
    const DLayer& L = net.L[sg.layer[q]];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = (blockIdx.x - sg.start[q]) * CB_WARPS + wib;
    if (u >= net.S * L.n_out) return;
    const int s = u / L.n_out, i = u - s * L.n_out;
    const int cur = st.ctr[1] & 1;
    const size_t NT = net.NT, NH = net.NH;
    const float* xv = st.spx[cur] + (size_t)s * NT + L.in_off;
    float a0 = 0.f;
    row_walk(L, i, lane, [&](int j, float w) { a0 += w * xv[j]; });
    a0 = warp_sum(a0);
    if (lane == 0) {
        const size_t h = (size_t)s * NH + L.h_out + i;
        const float xhat = a0 + L.b[i];
        const float x = st.spx[cur][(size_t)s * NT + L.out_off + i];
        const float z = st.spz[cur][h];
        st.ab[h] = (xhat - x >= 0.f) ? st.mua[h] : 0.f;
        const float v0 = x - z * st.uhat[h];
        const float v1 = x - xhat + (1.f - z) * st.lhat[h];
        const bool on = fmaxf(v0, v1) >= 0.f;
        const bool p0 = v0 >= v1;
        st.b0i[h] = (on && p0) ? st.mub[h] : 0.f;
        st.b1i[h] = (on && !p0) ? st.mub[h] : 0.f;
    }
}

// Col pass: subgradient step x_m += eta f_m(alpha*, beta*), z_m += eta g_m(beta*), projected on
// the boxes. The primal view's subgradient in x_m is -f_m since L holds -f_m^T x_m.
__global__ void __launch_bounds__(CB_THREADS) k_spi_col(DNet net, DState st, DSched sc, Segs sg) {
    const int q = seg_of(sg, blockIdx.x);
    const int li = sg.layer[q];
    const DLayer& L = net.L[li];
    const int k = li + 1, m = k - 1;
    const int u = (blockIdx.x - sg.start[q]) * CB_THREADS + threadIdx.x;
    const int step = st.ctr[2];
    if (u < net.S * L.n_in) {
        const int s = u / L.n_in, j = u - s * L.n_in;
        const int cur = st.ctr[1] & 1;
        const size_t NT = net.NT, NH = net.NH;
        const float eta = sc.sp_lr0 + (sc.sp_lr1 - sc.sp_lr0) * (float)step /
                          (float)max(1, sc.sp_init_steps - 1);
        float acc = 0.f;
        if (k <= net.n - 1) {
            const size_t rb = (size_t)s * NH + L.h_out;
            const float* ab = st.ab + rb;
            const float* b1 = st.b1i + rb;
            col_walk(L, j, [&](int i, float w) { acc += w * (ab[i] - b1[i]); });
        } else {
            acc = net.Wout[(size_t)s * L.n_in + j];
        }
        float f = -acc;
        const size_t xo = (size_t)s * NT + L.in_off + j;
        if (m >= 1) {
            const size_t h = (size_t)s * NH + L.h_in + j;
            f += st.ab[h] - st.b0i[h] - st.b1i[h];
            const float g = st.b0i[h] * st.uhat[h] + st.b1i[h] * st.lhat[h];
            st.spz[cur][h] = fminf(fmaxf(st.spz[cur][h] + eta * g, 0.f), 1.f);
        }
        st.spx[cur][xo] = fminf(fmaxf(st.spx[cur][xo] + eta * f, st.lo[xo]), st.hi[xo]);
    }
    if (last_block(&st.done[2]) && threadIdx.x == 0) {
        st.ctr[2] = step + 1;
        st.done[2] = 0;
    }
}

}  // namespace cb

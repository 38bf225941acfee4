// Envelope gradient of the Active Set bound and the recomputation of mask row sums.
//
// At fixed duals alpha, beta and fixed masks, with the intermediate bounds and the signs of W held
// fixed, the bound d = min_{x,z} L has gradient dL/dtheta at the minimiser (x*, z*) (Danskin).
// With the constraint form of L (App. D of the paper), for hidden layer k and pair (i, j):
//   dL/dW[i,j] = (alpha - beta1)[i] x[j]
//                + sum_b beta_b[i] ( I_b ? (1 - z[i]) Lcheck[i,j] - x[j] : -z[i] Ucheck[i,j] )
//   dL/db[i]   = (alpha - beta1)[i] - z[i] sum_b beta_b[i]
// and for the input box, through x_0* and through Lcheck, Ucheck of layer 1:
//   dL/dl_0[j] = -f_0[j] [x_0* = l_0] + sum_i sum_b beta_b[i] (I ? (1-z) W [W >= 0] : -z W [W < 0])
//   dL/du_0[j] = -f_0[j] [x_0* = u_0] + sum_i sum_b beta_b[i] (I ? (1-z) W [W < 0]  : -z W [W >= 0])
// The output row C[s]^T W_n gives dW_n[o, j] = C[s, o] x*_{n-1}[j] and db_n[o] = C[s, o].
// Each output element is written by exactly one thread or block (no atomics): deterministic.
#pragma once
#include "cb_kernels.cuh"

namespace cb {

struct GradCtx {
    const double* gb;      // [S] upstream gradient of each subproblem's bound
    int nsl_before;        // slots before the current iteration (global)
    int bo;                // snapshot buffer parity
    const float* Ah = nullptr;   // [S][NH] adjoints of lhat, uhat (through interval propagation), or null
    const float* Uh = nullptr;
};

// Term of dL/dW for subproblem s and pair (i, j) of hidden layer L.
__device__ __forceinline__ float wgrad_term(const DNet& net, const DState& st, const DLayer& L, int s, int i,
                                            int j, float w, int nsl, int bo, const float* Ah, const float* Uh) {
    const size_t NT = net.NT, NH = net.NH;
    const size_t xo = (size_t)s * NT + L.in_off + j;
    const size_t h = (size_t)s * NH + L.h_out + i;
    const float x = st.xval[xo];
    float g = (st.alpha[h] - st.beta1[h]) * x;
    if (nsl) {
        const float lo = st.lo[xo], hi = st.hi[xo];
        const unsigned I = cb_slot_mask(st.zsnap[bo][h], st.xsnap[bo][xo], lo == hi, w, net.ball && L.in_off == 0);
        const float z = st.zcur[h] ? 1.f : 0.f;
        const float Lc = w >= 0.f ? lo : hi, Uc = w >= 0.f ? hi : lo;
        const size_t hs = (size_t)s * net.cap * NH + L.h_out + i;
        for (int b = 0; b < nsl; ++b) {
            const float bb = st.bs[hs + (size_t)b * NH];
            g += bb * (((I >> b) & 1u) ? (1.f - z) * Lc - x : -z * Uc);
        }
    }
    if (Ah) {   // interval propagation: lhat = W+ l + W- u + b, uhat = W+ u + W- l + b
        const float lo = st.lo[xo], hi = st.hi[xo];
        if (net.ball && L.in_off == 0) {   // over the ellipsoid: W c + b -+ |W_i o e|
            const float c = 0.5f * (lo + hi), e = 0.5f * (hi - lo), r = st.brad[h];
            g += (Ah[h] + Uh[h]) * c + (r > 0.f ? (Uh[h] - Ah[h]) * w * e * e / r : 0.f);
        } else {
            g += Ah[h] * (w >= 0.f ? lo : hi) + Uh[h] * (w >= 0.f ? hi : lo);
        }
    }
    return g;
}

// Linear hidden layer: one thread per (i, j), summing over subproblems.
__global__ void k_grad_W_linear(DNet net, DState st, int li, GradCtx gc, float* dW) {
    const DLayer& L = net.L[li];
    const size_t n = (size_t)L.n_out * L.n_in;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(u / L.n_in), j = (int)(u - (size_t)i * L.n_in);
        const float w = L.W[u];
        double acc = 0.0;
        for (int s = 0; s < net.S; ++s) {
            const int nsl = min(gc.nsl_before, st.caps[s]);
            acc += gc.gb[s] * (double)wgrad_term(net, st, L, s, i, j, w, nsl, gc.bo, gc.Ah, gc.Uh);
        }
        dW[u] += (float)acc;
    }
}

// Conv hidden layer: one block per filter entry, reducing over subproblems and positions.
__global__ void k_grad_W_conv(DNet net, DState st, int li, GradCtx gc, float* dW) {
    const DLayer& L = net.L[li];
    const int fi = blockIdx.x;
    const int kk = L.kh * L.kw;
    const int co = fi / (L.ci * kk), r = fi - co * L.ci * kk;
    const int c = r / kk, q = r - c * kk;
    const int ky = q / L.kw, kx = q - ky * L.kw;
    const float w = L.W[fi];
    const int P = L.ho * L.wo;
    double acc = 0.0;
    for (int u = threadIdx.x; u < net.S * P; u += blockDim.x) {
        const int s = u / P, p = u - s * P;
        const int oy = p / L.wo, ox = p - oy * L.wo;
        const int y = oy * L.st - L.pd + ky, x = ox * L.st - L.pd + kx;
        if (y < 0 || y >= L.hi || x < 0 || x >= L.wi) continue;
        const int i = co * P + p, j = (c * L.hi + y) * L.wi + x;
        const int nsl = min(gc.nsl_before, st.caps[s]);
        acc += gc.gb[s] * (double)wgrad_term(net, st, L, s, i, j, w, nsl, gc.bo, gc.Ah, gc.Uh);
    }
    __shared__ double red[CB_THREADS];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = CB_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) dW[fi] += (float)red[0];
}

// Hidden-layer bias: one block per bias entry (a neuron, or a conv channel's positions).
__global__ void k_grad_b(DNet net, DState st, int li, GradCtx gc, float* db) {
    const DLayer& L = net.L[li];
    const int e = blockIdx.x;
    const int per = L.kind == 0 ? 1 : L.ho * L.wo;
    double acc = 0.0;
    for (int u = threadIdx.x; u < net.S * per; u += blockDim.x) {
        const int s = u / per, p = u - s * per;
        const int i = e * per + p;
        const int nsl = min(gc.nsl_before, st.caps[s]);
        const size_t h = (size_t)s * net.NH + L.h_out + i;
        float g = st.alpha[h] - st.beta1[h];
        if (st.zcur[h]) {
            const size_t hs = (size_t)s * net.cap * net.NH + L.h_out + i;
            for (int b = 0; b < nsl; ++b) g -= st.bs[hs + (size_t)b * net.NH];
        }
        if (gc.Ah) g += gc.Ah[h] + gc.Uh[h];
        acc += gc.gb[s] * (double)g;
    }
    __shared__ double red[CB_THREADS];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = CB_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[e] += (float)red[0];
}

// Output layer through the property rows: dW_n[o, j] = sum_s gb[s] C[s, o] x*[s, j].
__global__ void k_grad_out(DNet net, DState st, GradCtx gc, const float* C, int n_out, float* dW, float* db) {
    const DLayer& L = net.L[net.n - 1];
    const size_t n = (size_t)n_out * (L.n_in + 1);
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += (size_t)gridDim.x * blockDim.x) {
        const int o = (int)(u / (L.n_in + 1)), j = (int)(u - (size_t)o * (L.n_in + 1));
        double acc = 0.0;
        for (int s = 0; s < net.S; ++s) {
            const double cs = C ? (double)C[(size_t)s * n_out + o] : 1.0;
            const double v = j < L.n_in ? (double)st.xval[(size_t)s * net.NT + L.in_off + j] : 1.0;
            acc += gc.gb[s] * cs * v;
        }
        if (j < L.n_in) {
            if (dW) dW[(size_t)o * L.n_in + j] += (float)acc;
        } else if (db) {
            db[o] += (float)acc;
        }
    }
}

// Input box: col pass over layer 1 for input j of subproblem s.
__global__ void k_grad_box(DNet net, DState st, GradCtx gc, float* dlo, float* dhi) {
    const DLayer& L = net.L[0];
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= net.S * L.n_in) return;
    const int s = u / L.n_in, j = u - s * L.n_in;
    const int nsl = min(gc.nsl_before, st.caps[s]);
    const size_t xo = (size_t)s * net.NT + L.in_off + j;
    const float lo = st.lo[xo], hi = st.hi[xo];
    const unsigned xs = st.xsnap[gc.bo][xo];
    float al = 0.f, ah = 0.f;
    if (nsl && net.n >= 2) {
        const size_t rb = (size_t)s * net.NH + L.h_out;
        const size_t sb = (size_t)s * net.cap * net.NH + L.h_out;
        col_walk(L, j, [&](int i, float w) {
            const unsigned I = cb_slot_mask(st.zsnap[gc.bo][rb + i], xs, lo == hi, w, net.ball != 0);
            const float z = st.zcur[rb + i] ? 1.f : 0.f;
            float bsum_in = 0.f, bsum_out = 0.f;
            for (int b = 0; b < nsl; ++b) {
                const float bb = st.bs[sb + (size_t)b * net.NH + i];
                if ((I >> b) & 1u) bsum_in += bb;
                else bsum_out += bb;
            }
            const float ti = (1.f - z) * w * bsum_in;   // through Lcheck
            const float to = -z * w * bsum_out;         // through Ucheck
            if (w >= 0.f) { al += ti; ah += to; }
            else { ah += ti; al += to; }
        });
    }
    const float f0 = st.fval[xo];
    const float x = st.xval[xo];
    if (net.ball) {   // value -f c - |e f| over the ellipsoid, c = (l + u) / 2, e = (u - l) / 2
        const double nrm = st.bnrm[s];
        const float d = nrm > 0.0 ? (float)(0.5 * (0.5 * ((double)hi - lo)) * f0 * f0 / nrm) : 0.f;
        al += -0.5f * f0 + d;
        ah += -0.5f * f0 - d;
    } else if (lo == hi) {
        al += -0.5f * f0;
        ah += -0.5f * f0;
    } else if (x == hi) {
        ah += -f0;
    } else {
        al += -f0;
    }
    if (dlo) dlo[u] += (float)(gc.gb[s] * (double)al);
    if (dhi) dhi[u] += (float)(gc.gb[s] * (double)ah);
}

// Through interval propagation (the chain form of the gradient). Per subproblem and unscaled:
// Lb, Ub [S][NT] are dd/dl_k, dd/du_k of the post-activation bounds, Ah, Uh [S][NH] dd/dlhat_k,
// dd/duhat_k of the pre-activation ones.
//
// Direct part for the inputs of layer li (post-activation layer li): x* at an end of its box, and
// Lcheck, Ucheck of layer li's masks (as k_grad_box, for any layer).
__global__ void k_post_adj(DNet net, DState st, int li, GradCtx gc, float* Lb, float* Ub) {
    const DLayer& L = net.L[li];
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= net.S * L.n_in) return;
    const int s = u / L.n_in, j = u - s * L.n_in;
    const int nsl = min(gc.nsl_before, st.caps[s]);
    const size_t xo = (size_t)s * net.NT + L.in_off + j;
    const float lo = st.lo[xo], hi = st.hi[xo];
    const unsigned xs = st.xsnap[gc.bo][xo];
    float al = 0.f, ah = 0.f;
    if (nsl && li <= net.n - 2) {
        const size_t rb = (size_t)s * net.NH + L.h_out;
        const size_t sb = (size_t)s * net.cap * net.NH + L.h_out;
        col_walk(L, j, [&](int i, float w) {
            const unsigned I = cb_slot_mask(st.zsnap[gc.bo][rb + i], xs, lo == hi, w, net.ball && li == 0);
            const float z = st.zcur[rb + i] ? 1.f : 0.f;
            float bsum_in = 0.f, bsum_out = 0.f;
            for (int b = 0; b < nsl; ++b) {
                const float bb = st.bs[sb + (size_t)b * net.NH + i];
                if ((I >> b) & 1u) bsum_in += bb;
                else bsum_out += bb;
            }
            const float ti = (1.f - z) * w * bsum_in, to = -z * w * bsum_out;
            if (w >= 0.f) { al += ti; ah += to; }
            else { ah += ti; al += to; }
        });
    }
    const float f = st.fval[xo], x = st.xval[xo];
    if (net.ball && li == 0) {   // value -f c - |e f| over the ellipsoid (as k_grad_box)
        const double nrm = st.bnrm[s];
        const float d = nrm > 0.0 ? (float)(0.5 * (0.5 * ((double)hi - lo)) * f * f / nrm) : 0.f;
        al += -0.5f * f + d;
        ah += -0.5f * f - d;
    } else if (lo == hi) {
        al += -0.5f * f;
        ah += -0.5f * f;
    } else if (x == hi) {
        ah += -f;
    } else {
        al += -f;
    }
    Lb[xo] = al;
    Ub[xo] = ah;
}

// Hidden layer li + 1 (outputs of layer li): the Big-M rows give dd/dlhat = beta_1 (1 - z) and
// dd/duhat = -beta_0 z; l = max(lhat, 0), u = max(uhat, 0) pass Lb, Ub where positive; a split
// clamp (+1 with lhat = 0, -1 with uhat = 0) makes the bound a constant.
__global__ void k_hat_adj(DNet net, DState st, int li, const signed char* splits, const float* Lb, const float* Ub,
                          float* Ah, float* Uh) {
    const DLayer& L = net.L[li];
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= net.S * L.n_out) return;
    const int s = u / L.n_out, i = u - s * L.n_out;
    const size_t h = (size_t)s * net.NH + L.h_out + i;
    const size_t xo = (size_t)s * net.NT + net.L[li + 1].in_off + i;
    const float z = st.zcur[h] ? 1.f : 0.f;
    const float lh = st.lhat[h], uh = st.uhat[h];
    float a = st.beta1[h] * (1.f - z) + (lh > 0.f ? Lb[xo] : 0.f);
    float b = -st.beta0[h] * z + (uh > 0.f ? Ub[xo] : 0.f);
    if (splits) {
        if (splits[h] > 0 && lh == 0.f) a = 0.f;
        if (splits[h] < 0 && uh == 0.f) b = 0.f;
    }
    Ah[h] = a;
    Uh[h] = b;
}

// Back through lhat = W+ l + W- u + b, uhat = W+ u + W- l + b of layer li: adds W+^T Ah + W-^T Uh
// to Lb and W-^T Ah + W+^T Uh to Ub of its inputs (one thread per input, no atomics).
__global__ void k_prop_adj(DNet net, DState st, int li, const float* Ah, const float* Uh, float* Lb, float* Ub) {
    const DLayer& L = net.L[li];
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= net.S * L.n_in) return;
    const int s = u / L.n_in, j = u - s * L.n_in;
    const size_t rb = (size_t)s * net.NH + L.h_out;
    float al = 0.f, au = 0.f;
    if (net.ball && li == 0) {
        // over the ellipsoid lhat, uhat = W c + b -+ r, r_i = |W_i o e|: d/dc = W, dr_i/de_j = W^2 e_j / r_i;
        // d/dl = (d/dc - d/de) / 2, d/du = (d/dc + d/de) / 2
        const size_t xo = (size_t)s * net.NT + L.in_off + j;
        const float e = 0.5f * (st.hi[xo] - st.lo[xo]);
        col_walk(L, j, [&](int i, float w) {
            const float a = Ah[rb + i], b = Uh[rb + i], r = st.brad[rb + i];
            const float dc = w * (a + b), de = r > 0.f ? w * w * e / r * (b - a) : 0.f;
            al += 0.5f * (dc - de);
            au += 0.5f * (dc + de);
        });
    } else
    col_walk(L, j, [&](int i, float w) {
        const float a = Ah[rb + i], b = Uh[rb + i];
        if (w >= 0.f) { al += w * a; au += w * b; }
        else { al += w * b; au += w * a; }
    });
    const size_t xo = (size_t)s * net.NT + L.in_off + j;
    Lb[xo] += al;
    Ub[xo] += au;
}

// dlo, dhi += gb[s] Lb, Ub of the input layer
__global__ void k_box_out(DNet net, GradCtx gc, const float* Lb, const float* Ub, float* dlo, float* dhi) {
    const DLayer& L = net.L[0];
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= net.S * L.n_in) return;
    const int s = u / L.n_in, j = u - s * L.n_in;
    const size_t xo = (size_t)s * net.NT + L.in_off + j;
    if (dlo) dlo[u] += (float)(gc.gb[s] * (double)Lb[xo]);
    if (dhi) dhi[u] += (float)(gc.gb[s] * (double)Ub[xo]);
}

}  // namespace cb

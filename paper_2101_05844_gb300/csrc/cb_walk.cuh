// Index walks over the fan-in / fan-out of one neuron of a linear or conv2d layer, and warp sums:
// inline device helpers shared by the library's translation units.
#pragma once
#include "cb_common.cuh"

namespace cb {

// ------------------------------------------------------------------------------------ walks
// Lane-strided walk over the fan-in of output neuron i of layer L: fn(j, w) for each input j, by a
// team of T lanes (lane = 0 .. T - 1). Conv layers: the lanes stride over (input channel, kernel
// row) pairs and each walks its row's kernel columns, the receptive field clipped to the image once
// per neuron, with no integer division inside the loop.
template <class Fn>
__device__ __forceinline__ void row_walk_team(const DLayer& L, int i, int lane, int T, Fn fn) {
    if (L.kind == 0) {
        const float* Wr = L.W + (size_t)i * L.n_in;
#pragma unroll 4
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
    int c = lane / L.kh, ky = lane - c * L.kh;
    const int cstep = T / L.kh, kstep = T - cstep * L.kh;
    while (c < L.ci) {
        if (ky >= ky0 && ky < ky1) {
            const float* Wk = Wc + (c * L.kh + ky) * L.kw;
            const int jrow = (c * L.hi + y0 + ky) * L.wi + x0;
#pragma unroll 4
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

// The same walk by a whole warp.
template <class Fn>
__device__ __forceinline__ void row_walk(const DLayer& L, int i, int lane, Fn fn) {
    row_walk_team(L, i, lane, 32, fn);
}

// Serial walk over the fan-out of input neuron j of layer L: fn(i, w) for each output i.
template <class Fn>
__device__ __forceinline__ void col_walk(const DLayer& L, int j, Fn fn) {
    if (L.kind == 0) {
        const float* Wc = L.W + j;
        for (int i = 0; i < L.n_out; ++i) fn(i, __ldg(Wc + (size_t)i * L.n_in));
    } else {
        const int hw = L.hi * L.wi;
        const int c = j / hw, rem = j - c * hw;
        const int y = rem / L.wi, x = rem - y * L.wi;
        const int kk = L.kh * L.kw;
        const size_t cstride = (size_t)L.ci * kk;
        for (int ky = 0; ky < L.kh; ++ky) {
            const int ty = y + L.pd - ky;
            if (ty < 0 || ty % L.st) continue;
            const int oy = ty / L.st;
            if (oy >= L.ho) continue;
            for (int kx = 0; kx < L.kw; ++kx) {
                const int tx = x + L.pd - kx;
                if (tx < 0 || tx % L.st) continue;
                const int ox = tx / L.st;
                if (ox >= L.wo) continue;
                const float* Wp = L.W + (size_t)c * kk + ky * L.kw + kx;
                const int ib = oy * L.wo + ox;
                for (int co = 0; co < L.co; ++co) fn(co * L.ho * L.wo + ib, __ldg(Wp + co * cstride));
            }
        }
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Compensated float32 sum of products (a lane's share of a row sum): every product is split
// exactly into p + pe (TwoProd by one fma) and added by TwoSum (Knuth), the rounding errors
// gathered in c, so that s + c holds the partial sum to about k 2^-48 of its sum of |terms| after k
// terms, the accuracy of a float64 accumulation, at float32 rates (float64 is a narrow pipe on this
// part). The _rn intrinsics keep the compiler from contracting the error-free steps into fmas.
struct CompSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_prod(float w, float x) {
        const float p = __fmul_rn(w, x);
        const float pe = __fmaf_rn(w, x, -p);
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(e, pe));
    }
    // the warp's row sum: the lanes' pairs combined in float64
    __device__ __forceinline__ double warp_total() const { return warp_sum((double)s + (double)c); }
};

}  // namespace cb

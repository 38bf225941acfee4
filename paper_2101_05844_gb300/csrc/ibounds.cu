// Intermediate bounds by batched dual solves over sub-networks (App. E): the pre-activation
// bounds of hidden layer k are the bounds of min x_hat_k[i] and max x_hat_k[i] over the
// relaxation of layers 1 .. k-1, solved by Big-M then Active Set (Alg. 1). Every neuron of the
// layer, both signs and every box make one batch of subproblems. Built on the library's own C
// ABI: each batch is one context over the sub-network of layers 1 .. k, whose last layer is
// layer k as a linear map (a conv layer as its dense operator) and whose property rows are
// +e_i and -e_i.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/convex_barrier.h"

namespace {

// dst[q][c] = src[((r0 + q) / per) * ld + c]: the row of the box that subproblem r0 + q belongs to
__global__ void k_box_rows(const float* src, long long ld, float* dst, long long rows, int cols, long long r0,
                           int per) {
    const long long n = rows * cols;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        const long long q = u / cols;
        const int c = (int)(u - q * cols);
        dst[u] = src[((r0 + q) / per) * ld + c];
    }
}

// C[q][c] = +1 / -1 where c is the neuron of subproblem r = r0 + q (neuron (r / 2) % n, sign r & 1)
__global__ void k_unit_rows(float* C, long long rows, int n, long long r0) {
    const long long tot = rows * n;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
        const long long q = u / n;
        const int c = (int)(u - q * n);
        const long long r = r0 + q;
        C[u] = c == (int)((r >> 1) % n) ? ((r & 1) ? -1.f : 1.f) : 0.f;
    }
}

// lhat = max(lhat, bound(+e_i)), uhat = min(uhat, -bound(-e_i)), rounded outward to float32. Splits
// need no clamp here: interval propagation clamped every split neuron whose interval straddles
// zero, and the tightened interval lies inside the clamped one.
__global__ void k_tighten(const double* b, float* lh, float* uh, int nk, int NH, int off, long long r0,
                          long long rn) {
    const long long pairs = rn >> 1;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < pairs; p += (long long)gridDim.x * blockDim.x) {
        const long long q = (r0 >> 1) + p;
        const long long s = q / nk;
        const int i = (int)(q - s * nk);
        const size_t h = (size_t)s * NH + off + i;
        float l = fmaxf(lh[h], __double2float_rd(b[2 * p]));
        float u = fminf(uh[h], __double2float_ru(-b[2 * p + 1]));
        if (l > u) {   // no point of the relaxation reaches this neuron's range: keep one value
            const float m = 0.5f * (l + u);
            l = u = m;
        }
        lh[h] = l;
        uh[h] = u;
    }
}

int grid_of(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16)); }

// The dense operator of a conv layer: W [out_c out_h out_w][in_c in_h in_w] (CHW order on both sides)
void conv_dense(const as_layer& L, const std::vector<float>& Wc, const std::vector<float>& bc, std::vector<float>& Wd,
                std::vector<float>& bd) {
    const int P = L.out_h * L.out_w, nin = L.in_c * L.in_h * L.in_w;
    Wd.assign((size_t)L.out_c * P * nin, 0.f);
    bd.assign((size_t)L.out_c * P, 0.f);
    for (int co = 0; co < L.out_c; ++co)
        for (int oy = 0; oy < L.out_h; ++oy)
            for (int ox = 0; ox < L.out_w; ++ox) {
                const size_t i = (size_t)co * P + oy * L.out_w + ox;
                bd[i] = bc[co];
                for (int ci = 0; ci < L.in_c; ++ci)
                    for (int ky = 0; ky < L.kh; ++ky)
                        for (int kx = 0; kx < L.kw; ++kx) {
                            const int y = oy * L.stride - L.pad + ky, x = ox * L.stride - L.pad + kx;
                            if (y < 0 || y >= L.in_h || x < 0 || x >= L.in_w) continue;
                            Wd[i * nin + ((size_t)ci * L.in_h + y) * L.in_w + x] +=
                                Wc[(((size_t)co * L.in_c + ci) * L.kh + ky) * L.kw + kx];
                        }
            }
}

struct DevBufs {
    std::vector<void*> p;
    template <class T>
    T* get(size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        p.push_back(q);
        return static_cast<T*>(q);
    }
    ~DevBufs() {
        for (void* q : p) cudaFree(q);
    }
};

}  // namespace

extern "C" int as_intermediate_bounds(const as_net* net, int S, const float* x_lo, const float* x_hi,
                                      const signed char* splits, const as_options* opt, long long max_batch,
                                      float* lhat, float* uhat, void* stream) {
    if (!net || !net->layers || S < 1 || !x_lo || !x_hi || !lhat || !uhat || max_batch < 0) return AS_ERR_ARG;
    const int n = net->n_layers;
    if (n < 2 || n > AS_MAX_LAYERS) return AS_ERR_SHAPE;
    if (max_batch == 0) max_batch = 1LL << 14;
    max_batch = std::max(2LL, max_batch & ~1LL);   // whole (+e_i, -e_i) pairs
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int> width(n);   // width[k]: inputs of layer k + 1 (width[0] = n_0)
    for (int k = 0; k < n; ++k) {
        const as_layer& L = net->layers[k];
        width[k] = L.kind == AS_LAYER_LINEAR ? L.in_c : L.in_c * L.in_h * L.in_w;
    }
    const int n0 = width[0];
    int NH = 0;
    std::vector<int> hoff(n, 0);   // hoff[k]: offset of hidden layer k in a hidden vector
    for (int k = 1; k < n; ++k) {
        hoff[k] = NH;
        NH += width[k];
    }
    as_options o;
    if (opt) o = *opt;
    else as_default_options(&o);
    int r = AS_OK;
    // interval bounds of every hidden layer (exact for layer 1, an affine map of the box), with
    // the split clamps, from a context of the whole network
    {
        as_ctx* c = nullptr;
        as_options oi;
        as_default_options(&oi);
        oi.input_l2 = o.input_l2;   // the same input set as the solves
        const int nout = net->layers[n - 1].out_c;
        std::vector<float> C1;
        if (nout != 1) {   // any property row serves: only the interval bounds are read
            C1.assign((size_t)S * nout, 0.f);
            for (int s = 0; s < S; ++s) C1[(size_t)s * nout] = 1.f;
        }
        r = as_init(&c, net, S, x_lo, x_hi, nout != 1 ? C1.data() : nullptr, nullptr, nullptr, splits, nullptr, &oi,
                    stream);
        if (r == AS_OK) r = as_get_state(c, AS_ST_LHAT, lhat);
        if (r == AS_OK) r = as_get_state(c, AS_ST_UHAT, uhat);
        if (c) as_destroy(c);
        if (r != AS_OK) return r;
    }
    DevBufs keep;
    float* dl = keep.get<float>((size_t)S * NH);
    float* du = keep.get<float>((size_t)S * NH);
    float* dlo = keep.get<float>((size_t)S * n0);
    float* dhi = keep.get<float>((size_t)S * n0);
    if (!dl || !du || !dlo || !dhi) return AS_ERR_OOM;
    if (cudaMemcpyAsync(dl, lhat, (size_t)S * NH * 4, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(du, uhat, (size_t)S * NH * 4, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(dlo, x_lo, (size_t)S * n0 * 4, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(dhi, x_hi, (size_t)S * n0 * 4, cudaMemcpyDefault, st) != cudaSuccess)
        return AS_ERR_CUDA;
    const int iters = o.bigm_iters + o.as_iters;
    for (int k = 2; k < n && r == AS_OK; ++k) {   // hidden layer k is the output of net->layers[k - 1]
        const as_layer& Lk = net->layers[k - 1];
        const int nk = width[k];
        std::vector<as_layer> sub(net->layers, net->layers + k);
        std::vector<float> Wd, bd;
        if (Lk.kind == AS_LAYER_CONV2D) {
            std::vector<float> Wc((size_t)Lk.out_c * Lk.in_c * Lk.kh * Lk.kw), bc(Lk.out_c);
            if (cudaMemcpy(Wc.data(), Lk.W, Wc.size() * 4, cudaMemcpyDefault) != cudaSuccess ||
                cudaMemcpy(bc.data(), Lk.b, bc.size() * 4, cudaMemcpyDefault) != cudaSuccess)
                return AS_ERR_CUDA;
            conv_dense(Lk, Wc, bc, Wd, bd);
            as_layer lin{};
            lin.kind = AS_LAYER_LINEAR;
            lin.in_c = width[k - 1];
            lin.out_c = nk;
            lin.W = Wd.data();
            lin.b = bd.data();
            sub[k - 1] = lin;
        }
        const as_net sn{k, sub.data()};
        const int hsub = hoff[k];   // hidden neurons of layers 1 .. k-1 (>= n_1 > 0)
        const int per = 2 * nk;     // subproblems per box
        const long long rows = (long long)S * per;
        const long long cap = std::min(max_batch, rows);
        DevBufs chunk;
        float* blo = chunk.get<float>(cap * n0);
        float* bhi = chunk.get<float>(cap * n0);
        float* bl = chunk.get<float>(cap * hsub);
        float* bu = chunk.get<float>(cap * hsub);
        float* bC = chunk.get<float>(cap * nk);
        double* bout = chunk.get<double>(cap);
        if (!blo || !bhi || !bl || !bu || !bC || !bout) return AS_ERR_OOM;
        as_ctx* c = nullptr;
        for (long long r0 = 0; r0 < rows && r == AS_OK; r0 += cap) {
            const long long rn = std::min(cap, rows - r0);
            k_box_rows<<<grid_of(rn * n0), 256, 0, st>>>(dlo, n0, blo, rn, n0, r0, per);
            k_box_rows<<<grid_of(rn * n0), 256, 0, st>>>(dhi, n0, bhi, rn, n0, r0, per);
            k_box_rows<<<grid_of(rn * hsub), 256, 0, st>>>(dl, NH, bl, rn, hsub, r0, per);
            k_box_rows<<<grid_of(rn * hsub), 256, 0, st>>>(du, NH, bu, rn, hsub, r0, per);
            k_unit_rows<<<grid_of(rn * nk), 256, 0, st>>>(bC, rn, nk, r0);
            if (cudaGetLastError() != cudaSuccess) r = AS_ERR_CUDA;
            // the bounds of layers 1 .. k-1 carry their split clamps already
            if (r == AS_OK) {
                if (c && rn == cap) r = as_reset(c, blo, bhi, bC, bl, bu, nullptr, nullptr);
                else {
                    if (c) as_destroy(c);
                    c = nullptr;
                    r = as_init(&c, &sn, (int)rn, blo, bhi, bC, bl, bu, nullptr, nullptr, &o, stream);
                }
            }
            if (r == AS_OK) r = as_step(c, iters);
            if (r == AS_OK) r = as_bound(c, 64, bout, nullptr);
            if (r == AS_OK) {
                k_tighten<<<grid_of(rn / 2), 256, 0, st>>>(bout, dl, du, nk, NH, hoff[k], r0, rn);
                if (cudaGetLastError() != cudaSuccess) r = AS_ERR_CUDA;
            }
        }
        if (c) as_destroy(c);
        if (cudaStreamSynchronize(st) != cudaSuccess && r == AS_OK) r = AS_ERR_CUDA;
    }
    if (r != AS_OK) return r;
    if (cudaMemcpyAsync(lhat, dl, (size_t)S * NH * 4, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(uhat, du, (size_t)S * NH * 4, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return AS_ERR_CUDA;
    return AS_OK;
}

// as_ibp_noalloc: interval bounds of every hidden layer for callers that cannot allocate device
// memory. It runs the same per-layer computation as the bounds that as_init derives, but keeps the
// post-activation bounds passed from one layer to the next in a fixed, file-scope device array
// instead of context buffers, so the call itself allocates nothing.
#include <cstdio>

#include "../../include/convex_barrier.h"
#include "cb_walk.cuh"

namespace {

// Scratch shared by every call on a device: four regions (lower and upper post-activation bounds
// of the layer being read and of the layer being written) of up to S x (widest hidden layer)
// floats each. Every GPU that loads the library holds it until the process exits.
constexpr size_t kScratchFloats = AS_NOALLOC_SCRATCH_FLOATS;
static __device__ __align__(256) float g_ibp_scratch[kScratchFloats];

// Device address of g_ibp_scratch on the current device. In host code the array's name only stands
// for the symbol; a kernel must be given this address instead. It is looked up on every call (a
// lookup, not an allocation, once the module is loaded on the device), so that a device reset or a
// new primary context, after which the module is loaded again at a possibly different address,
// never leaves a stale address behind.
int scratch_address(float** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ibp_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return AS_ERR_CUDA;
    }
    *out = (float*)p;
    return AS_OK;
}

// Device memory of the current device (or managed memory): the only memory the kernels may read and
// write without peer access.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// One hidden layer of interval propagation (App. E): W+ l + W- u + b and W+ u + W- l + b to float64
// accuracy (the context's compensated float32 sums, in the same order), outward rounding to float32, split clamps of straddling neurons, then the
// post-activation box written to the next region of the scratch.
__global__ void k_ibp_noalloc(DLayer L, int S, int bias_per, const float* in_lo, const float* in_hi,
                              int in_stride, const signed char* splits, int NH, int h_off, float* lhat,
                              float* uhat, float* out_lo, float* out_hi, int out_stride) {
    const int warp = (blockIdx.x * CB_THREADS + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= S * L.n_out) return;
    const int s = warp / L.n_out, i = warp - s * L.n_out;
    const float* lo = in_lo + (size_t)s * in_stride;
    const float* hi = in_hi + (size_t)s * in_stride;
    cb::CompSum ca, cc;
    cb::row_walk(L, i, lane, [&](int j, float w) {
        const float l = lo[j], u = hi[j];
        ca.add_prod(w, w >= 0.f ? l : u);
        cc.add_prod(w, w >= 0.f ? u : l);
    });
    double a = ca.warp_total(), c = cc.warp_total();
    if (lane == 0) {
        const double bi = (double)L.b[i / bias_per];
        a += bi;
        c += bi;
        const size_t h = (size_t)s * NH + h_off + i;
        if (splits && a < 0.0 && c > 0.0) {
            if (splits[h] > 0) a = 0.0;
            if (splits[h] < 0) c = 0.0;
        }
        const float lh = __double2float_rd(a), uh = __double2float_ru(c);
        lhat[h] = lh;
        uhat[h] = uh;
        out_lo[(size_t)s * out_stride + i] = fmaxf(lh, 0.f);
        out_hi[(size_t)s * out_stride + i] = fmaxf(uh, 0.f);
    }
}

}  // namespace

extern "C" int as_ibp_noalloc(const as_net* net, int S, const float* x_lo, const float* x_hi,
                              const signed char* splits, float* lhat, float* uhat, void* stream) {
    if (!net || !net->layers || S < 1 || !x_lo || !x_hi || !lhat || !uhat) return AS_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return AS_ERR_CUDA;
    const int n = net->n_layers;
    if (n < 2 || n > AS_MAX_LAYERS) return AS_ERR_SHAPE;
    DLayer Ls[AS_MAX_LAYERS];
    int bias_per[AS_MAX_LAYERS];
    int NH = 0, widest = 0, prev = -1;
    for (int k = 0; k < n - 1; ++k) {  // the hidden layers; the output layer needs no bounds
        const as_layer& A = net->layers[k];
        DLayer& L = Ls[k];
        L = DLayer{};
        if (!A.W || !A.b || !on_device(A.W, dev) || !on_device(A.b, dev)) return AS_ERR_ARG;
        L.kind = A.kind;
        if (A.kind == AS_LAYER_LINEAR) {
            if (A.in_c < 1 || A.out_c < 1) return AS_ERR_SHAPE;
            L.n_in = A.in_c; L.n_out = A.out_c;
            L.ci = A.in_c; L.hi = L.wi = 1; L.co = A.out_c; L.ho = L.wo = 1;
            L.kh = L.kw = L.st = 1; L.pd = 0;
            bias_per[k] = 1;
        } else if (A.kind == AS_LAYER_CONV2D) {
            if (A.in_c < 1 || A.in_h < 1 || A.in_w < 1 || A.out_c < 1 || A.kh < 1 || A.kw < 1 || A.stride < 1 ||
                A.pad < 0)
                return AS_ERR_SHAPE;
            const int oh = (A.in_h + 2 * A.pad - A.kh) / A.stride + 1, ow = (A.in_w + 2 * A.pad - A.kw) / A.stride + 1;
            if (oh != A.out_h || ow != A.out_w || oh < 1 || ow < 1) return AS_ERR_SHAPE;
            L.ci = A.in_c; L.hi = A.in_h; L.wi = A.in_w; L.co = A.out_c; L.ho = oh; L.wo = ow;
            L.kh = A.kh; L.kw = A.kw; L.st = A.stride; L.pd = A.pad;
            L.n_in = L.ci * L.hi * L.wi;
            L.n_out = L.co * oh * ow;
            bias_per[k] = oh * ow;
        } else {
            return AS_ERR_ARG;
        }
        if (prev >= 0 && L.n_in != prev) return AS_ERR_SHAPE;
        prev = L.n_out;
        L.W = A.W;
        L.b = A.b;
        NH += L.n_out;
        if (L.n_out > widest) widest = L.n_out;
    }
    if (!on_device(x_lo, dev) || !on_device(x_hi, dev) || !on_device(lhat, dev) || !on_device(uhat, dev) ||
        (splits && !on_device(splits, dev)))
        return AS_ERR_ARG;
    // four scratch regions of S x widest floats
    if ((size_t)S * (size_t)widest * 4 > kScratchFloats) return AS_ERR_SCRATCH;
    float* scratch = nullptr;
    if (scratch_address(&scratch) != AS_OK) return AS_ERR_CUDA;
    const size_t region = (size_t)S * widest;
    float* lo_buf[2] = {scratch, scratch + 2 * region};
    float* hi_buf[2] = {scratch + region, scratch + 3 * region};
    cudaStream_t st = (cudaStream_t)stream;
    const float* in_lo = x_lo;
    const float* in_hi = x_hi;
    int in_stride = Ls[0].n_in, h_off = 0;
    for (int k = 0; k < n - 1; ++k) {
        const DLayer& L = Ls[k];
        float* out_lo = lo_buf[k & 1];
        float* out_hi = hi_buf[k & 1];
        const long long warps = (long long)S * L.n_out;
        k_ibp_noalloc<<<(int)((warps + CB_WARPS - 1) / CB_WARPS), CB_THREADS, 0, st>>>(
            L, S, bias_per[k], in_lo, in_hi, in_stride, splits, NH, h_off, lhat, uhat, out_lo, out_hi, L.n_out);
        if (cudaGetLastError() != cudaSuccess) return AS_ERR_CUDA;
        in_lo = out_lo;
        in_hi = out_hi;
        in_stride = L.n_out;
        h_off += L.n_out;
    }
    return AS_OK;
}

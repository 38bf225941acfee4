// Branch and bound with stratified bounding (Sec. 6.2) and parent warm starts (Sec. 8.2), on the
// library's own C ABI. The bounding of a batch of domains is one as_reset / as_step / as_bound of
// a context; the driver adds the per-domain bookkeeping: best-first selection, branching on the
// ambiguous neuron with the largest relaxation gap, the stratification estimate, the dual arena
// for warm starts and the upper bound from each solve's x_0*.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <queue>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/convex_barrier.h"

namespace {

constexpr int kThreads = 256;

// argmax over the ambiguous unsplit neurons of row b of -l u / (u - l); lowest index on ties; -1
__global__ void k_branch(const float* lh, const float* uh, const signed char* splits, int NH, int* out) {
    const int b = blockIdx.x;
    const float* l = lh + (size_t)b * NH;
    const float* u = uh + (size_t)b * NH;
    const signed char* sp = splits + (size_t)b * NH;
    float best = -1.f;
    int bi = -1;
    for (int j = threadIdx.x; j < NH; j += blockDim.x) {
        const float lj = l[j], uj = u[j];
        if (lj < 0.f && uj > 0.f && sp[j] == 0) {
            const float sc = -lj * uj / (uj - lj);
            if (sc > best) best = sc, bi = j;   // j rises within a thread: first of equals kept
        }
    }
    __shared__ float sb[kThreads];
    __shared__ int si[kThreads];
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            const float o = sb[threadIdx.x + h];
            const int oi = si[threadIdx.x + h];
            if (oi >= 0 && (si[threadIdx.x] < 0 || o > sb[threadIdx.x] || (o == sb[threadIdx.x] && oi < si[threadIdx.x]))) {
                sb[threadIdx.x] = o;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = si[0];
}

// lh = max(lh, rl), uh = min(uh, ru) with the root's bounds broadcast over the rows
__global__ void k_intersect(float* lh, float* uh, const float* rl, const float* ru, long long n, int NH) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(u % NH);
        lh[u] = fmaxf(lh[u], rl[j]);
        uh[u] = fminf(uh[u], ru[j]);
    }
}

// rows of (alpha, beta_0, beta_1) from / to the dual arena ([slot][3][NH]); slot < 0: zeros
__global__ void k_gather(const float* arena, const int* slot, float* a, float* b0, float* b1, int rows, int NH) {
    const long long n = (long long)rows * NH;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(u / NH), j = (int)(u - (long long)r * NH);
        const int s = slot[r];
        const float* src = arena + (size_t)(s < 0 ? 0 : s) * 3 * NH;
        a[u] = s < 0 ? 0.f : src[j];
        b0[u] = s < 0 ? 0.f : src[NH + j];
        b1[u] = s < 0 ? 0.f : src[2 * NH + j];
    }
}

__global__ void k_scatter(float* arena, const int* slot, const float* a, const float* b0, const float* b1, int rows,
                          int NH) {
    const long long n = (long long)rows * NH;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(u / NH), j = (int)(u - (long long)r * NH);
        float* dst = arena + (size_t)slot[r] * 3 * NH;
        dst[j] = a[u];
        dst[NH + j] = b0[u];
        dst[2 * NH + j] = b1[u];
    }
}

int grid_of(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 8)); }

struct Domain {
    std::vector<signed char> splits;
    double lb = 0, v = 0;
    bool hard = false, again = false;
    int alg = 0;   // 0: a_l, 1: a_t
    int branch = -1, rebounds = 0, slot = -1, depth = 0;
    long long seq = 0;
};

struct Entry {
    double lb;
    long long seq;
    int idx;
    bool operator<(const Entry& o) const { return lb != o.lb ? lb > o.lb : seq > o.seq; }   // min-heap
};

// float64 forward pass on the host (the confirmation of a counterexample)
struct HostNet {
    std::vector<as_layer> L;
    std::vector<std::vector<double>> W, b;
    int init(const as_net* net) {
        L.assign(net->layers, net->layers + net->n_layers);
        for (auto& l : L) {
            const size_t nw = l.kind == AS_LAYER_LINEAR ? (size_t)l.out_c * l.in_c : (size_t)l.out_c * l.in_c * l.kh * l.kw;
            std::vector<float> wf(nw), bf(l.out_c);
            if (cudaMemcpy(wf.data(), l.W, nw * 4, cudaMemcpyDefault) != cudaSuccess ||
                cudaMemcpy(bf.data(), l.b, bf.size() * 4, cudaMemcpyDefault) != cudaSuccess)
                return AS_ERR_CUDA;
            W.emplace_back(wf.begin(), wf.end());
            b.emplace_back(bf.begin(), bf.end());
        }
        return AS_OK;
    }
    double value(const float* x0, const std::vector<double>& c) const {
        std::vector<double> h(x0, x0 + (L[0].kind == AS_LAYER_LINEAR ? L[0].in_c : L[0].in_c * L[0].in_h * L[0].in_w));
        for (size_t k = 0; k < L.size(); ++k) {
            const as_layer& l = L[k];
            std::vector<double> o;
            if (l.kind == AS_LAYER_LINEAR) {
                o.assign(l.out_c, 0.0);
                for (int i = 0; i < l.out_c; ++i) {
                    double s = b[k][i];
                    for (int j = 0; j < l.in_c; ++j) s += W[k][(size_t)i * l.in_c + j] * h[j];
                    o[i] = s;
                }
            } else {
                o.assign((size_t)l.out_c * l.out_h * l.out_w, 0.0);
                for (int co = 0; co < l.out_c; ++co)
                    for (int oy = 0; oy < l.out_h; ++oy)
                        for (int ox = 0; ox < l.out_w; ++ox) {
                            double s = b[k][co];
                            for (int ci = 0; ci < l.in_c; ++ci)
                                for (int ky = 0; ky < l.kh; ++ky)
                                    for (int kx = 0; kx < l.kw; ++kx) {
                                        const int y = oy * l.stride - l.pad + ky, x = ox * l.stride - l.pad + kx;
                                        if (y < 0 || y >= l.in_h || x < 0 || x >= l.in_w) continue;
                                        s += W[k][(((size_t)co * l.in_c + ci) * l.kh + ky) * l.kw + kx] *
                                             h[((size_t)ci * l.in_h + y) * l.in_w + x];
                                    }
                            o[((size_t)co * l.out_h + oy) * l.out_w + ox] = s;
                        }
            }
            if (k + 1 < L.size())
                for (auto& v : o) v = std::max(v, 0.0);
            h.swap(o);
        }
        double s = 0;
        for (size_t i = 0; i < c.size(); ++i) s += c[i] * h[i];
        return s;
    }
};

bool subtree_hard(double lp, double delta, bool have_ema, double i, double c) {
    if (!have_ema) return false;
    if (i <= 0.0) return delta > 0.0;
    const double a = -lp / i + 1.0, bb = -(lp + delta) / i + 1.0;
    if (a > 60.0 && bb > 60.0) return std::exp2(a - bb) > c;
    const double sl = std::exp2(a) - 1.0, st = std::exp2(bb) - 1.0;
    if (st <= 0.0) return sl > 0.0;
    return sl / st > c;
}

struct Bab {
    const as_net* net;
    as_bab_options o;
    cudaStream_t st;
    int n0 = 0, NH = 0, NT = 0, nout = 0, B = 0;
    as_ctx* ctx[2] = {nullptr, nullptr};
    as_ctx* ev = nullptr;
    std::vector<void*> bufs;
    float *lo_d = nullptr, *hi_d = nullptr, *C_d = nullptr, *lh_d = nullptr, *uh_d = nullptr, *rl_d = nullptr,
          *ru_d = nullptr, *al_d = nullptr, *b0_d = nullptr, *b1_d = nullptr, *xs_d = nullptr, *x0_d = nullptr;
    signed char* sp_d = nullptr;
    double *bd_d = nullptr, *ev_d = nullptr;
    int *br_d = nullptr, *slot_d = nullptr;
    float* arena = nullptr;
    long long arena_cap = 0;
    std::vector<int> free_slots;
    int next_slot = 0;
    std::vector<signed char> sp_h;
    std::vector<double> crow;
    HostNet hn;
    double ub = std::numeric_limits<double>::infinity();
    std::vector<float> x_ub;
    long long bounded = 0, hard_bounded = 0, batches = 0;

    template <class T>
    T* dev(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return static_cast<T*>(p);
    }
    ~Bab() {
        for (auto* c : ctx)
            if (c) as_destroy(c);
        if (ev) as_destroy(ev);
        for (void* p : bufs) cudaFree(p);
        cudaFree(arena);
    }

    int alloc_slot(int* out) {
        if (!free_slots.empty()) {
            *out = free_slots.back();
            free_slots.pop_back();
            return AS_OK;
        }
        if (next_slot == arena_cap) {   // grow the arena, keeping the stored rows
            const long long ncap = std::max<long long>(2 * arena_cap, 4LL * B);
            float* na = nullptr;
            if (cudaMalloc(&na, (size_t)ncap * 3 * NH * 4) != cudaSuccess) return AS_ERR_OOM;
            if (arena && cudaMemcpyAsync(na, arena, (size_t)arena_cap * 3 * NH * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return AS_ERR_CUDA;
            if (cudaStreamSynchronize(st) != cudaSuccess) return AS_ERR_CUDA;
            cudaFree(arena);
            arena = na;
            arena_cap = ncap;
        }
        *out = next_slot++;
        return AS_OK;
    }

    // bounds the domains of `jobs` with algorithm alg; parents[r]: arena slot of the warm start or -1
    int bound(std::vector<Domain*>& jobs, const std::vector<int>& parents, int alg) {
        const int m = (int)jobs.size();
        if (m == 0) return AS_OK;
        as_ctx* c = ctx[alg];
        for (int r = 0; r < B; ++r)
            std::memcpy(&sp_h[(size_t)r * NH], jobs[r < m ? r : 0]->splits.data(), NH);
        if (cudaMemcpyAsync(sp_d, sp_h.data(), (size_t)B * NH, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return AS_ERR_CUDA;
        int r = as_reset(c, lo_d, hi_d, C_d, nullptr, nullptr, sp_d, nullptr);
        if (r != AS_OK) return r;
        if (o.root_intermediate) {
            if ((r = as_get_state(c, AS_ST_LHAT, lh_d)) != AS_OK || (r = as_get_state(c, AS_ST_UHAT, uh_d)) != AS_OK)
                return r;
            k_intersect<<<grid_of((long long)B * NH), kThreads, 0, st>>>(lh_d, uh_d, rl_d, ru_d, (long long)B * NH, NH);
            if ((r = as_reset(c, lo_d, hi_d, C_d, lh_d, uh_d, nullptr, nullptr)) != AS_OK) return r;
        }
        if (o.warm_start) {
            std::vector<int> ps(B, -1);
            for (int q = 0; q < m; ++q) ps[q] = parents[q];
            bool any = false;
            for (int q = 0; q < m; ++q) any |= ps[q] >= 0;
            if (any) {
                if (cudaMemcpyAsync(slot_d, ps.data(), B * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
                    return AS_ERR_CUDA;
                k_gather<<<grid_of((long long)B * NH), kThreads, 0, st>>>(arena, slot_d, al_d, b0_d, b1_d, B, NH);
                if ((r = as_set_state(c, AS_ST_ALPHA, al_d)) != AS_OK || (r = as_set_state(c, AS_ST_BETA0, b0_d)) != AS_OK ||
                    (r = as_set_state(c, AS_ST_BETA1, b1_d)) != AS_OK)
                    return r;
            }
        }
        const as_options& ao = alg ? o.tight : o.loose;
        if ((r = as_step(c, ao.bigm_iters + ao.as_iters)) != AS_OK) return r;
        if ((r = as_bound(c, 64, bd_d, nullptr)) != AS_OK) return r;
        // branching choice from the bounds the solve used
        if ((r = as_get_state(c, AS_ST_LHAT, lh_d)) != AS_OK || (r = as_get_state(c, AS_ST_UHAT, uh_d)) != AS_OK)
            return r;
        k_branch<<<m, kThreads, 0, st>>>(lh_d, uh_d, sp_d, NH, br_d);
        // the network at each solve's x_0*
        if ((r = as_get_state(c, AS_ST_XSTAR, xs_d)) != AS_OK) return r;
        if (cudaMemcpy2DAsync(x0_d, (size_t)n0 * 4, xs_d, (size_t)NT * 4, (size_t)n0 * 4, B, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return AS_ERR_CUDA;
        if ((r = as_reset(ev, x0_d, x0_d, C_d, nullptr, nullptr, nullptr, nullptr)) != AS_OK) return r;
        if ((r = as_bound(ev, 64, ev_d, nullptr)) != AS_OK) return r;
        // the duals of every solved domain into its arena slot
        std::vector<int> slots(B, 0);
        for (int q = 0; q < m; ++q) {
            if (jobs[q]->slot < 0 && (r = alloc_slot(&jobs[q]->slot)) != AS_OK) return r;
            slots[q] = jobs[q]->slot;
        }
        if ((r = as_get_state(c, AS_ST_ALPHA, al_d)) != AS_OK || (r = as_get_state(c, AS_ST_BETA0, b0_d)) != AS_OK ||
            (r = as_get_state(c, AS_ST_BETA1, b1_d)) != AS_OK)
            return r;
        if (cudaMemcpyAsync(slot_d, slots.data(), B * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return AS_ERR_CUDA;
        k_scatter<<<grid_of((long long)m * NH), kThreads, 0, st>>>(arena, slot_d, al_d, b0_d, b1_d, m, NH);
        if (cudaGetLastError() != cudaSuccess) return AS_ERR_CUDA;
        std::vector<double> bd(m), evh(m);
        std::vector<int> br(m);
        if (cudaMemcpyAsync(bd.data(), bd_d, m * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(evh.data(), ev_d, m * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(br.data(), br_d, m * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return AS_ERR_CUDA;
        for (int q = 0; q < m; ++q) {
            jobs[q]->v = bd[q];
            jobs[q]->branch = br[q];
            if (evh[q] < ub) {   // a candidate: its float64 value decides
                std::vector<float> x(n0);
                if (cudaMemcpy(x.data(), x0_d + (size_t)q * n0, n0 * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
                    return AS_ERR_CUDA;
                const double v = hn.value(x.data(), crow);
                if (v < ub) {
                    ub = v;
                    x_ub = x;
                }
            }
        }
        bounded += m;
        if (alg) hard_bounded += m;
        ++batches;
        return AS_OK;
    }
};

}  // namespace

extern "C" void as_bab_default_options(as_bab_options* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    as_default_options(&p->loose);
    p->loose.bigm_iters = 180;
    p->loose.as_iters = 0;
    p->loose.graph_chunk = 0;
    as_default_options(&p->tight);
    p->tight.bigm_iters = 180;   // a_t = a_l followed by Active Set: Big-M initialises it (App. B)
    p->tight.as_iters = 100;
    p->tight.omega = 40;
    p->tight.max_cuts = 3;
    p->tight.graph_chunk = 0;
    p->stratify = 1;
    p->cost_ratio = 0.0;
    p->ema_weight = 0.3;
    p->batch = 256;
    p->max_domains = 100000;
    p->time_limit = 0.0;
    p->warm_start = 1;
    p->leaf_rebounds = 8;
    p->root_intermediate = 0;
    as_default_options(&p->intermediate);
    p->intermediate.bigm_iters = 100;
    p->intermediate.as_iters = 0;
}

extern "C" int as_bab(const as_net* net, const float* x_lo, const float* x_hi, const float* cvec,
                      const as_bab_options* opt, as_bab_result* res, float* x_best, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!net || !net->layers || !x_lo || !x_hi || !res || net->n_layers < 2 || net->n_layers > AS_MAX_LAYERS)
        return AS_ERR_ARG;
    Bab b;
    b.net = net;
    if (opt) b.o = *opt;
    else as_bab_default_options(&b.o);
    if (b.o.batch < 2 || (b.o.batch & 1) || b.o.ema_weight < 0 || b.o.ema_weight > 1 || b.o.leaf_rebounds < 0)
        return AS_ERR_ARG;
    if (b.o.loose.input_l2 != b.o.tight.input_l2) return AS_ERR_ARG;   // one input set for the search
    b.o.intermediate.input_l2 = b.o.tight.input_l2;
    b.st = static_cast<cudaStream_t>(stream);
    const int n = net->n_layers;
    const as_layer& L0 = net->layers[0];
    b.n0 = L0.kind == AS_LAYER_LINEAR ? L0.in_c : L0.in_c * L0.in_h * L0.in_w;
    for (int k = 1; k < n; ++k) {
        const as_layer& l = net->layers[k];
        b.NH += l.kind == AS_LAYER_LINEAR ? l.in_c : l.in_c * l.in_h * l.in_w;
    }
    b.NT = b.n0 + b.NH;
    b.nout = net->layers[n - 1].out_c;
    if (!cvec && b.nout != 1) return AS_ERR_ARG;
    b.crow.assign(b.nout, 1.0);
    if (cvec)
        for (int i = 0; i < b.nout; ++i) b.crow[i] = cvec[i];
    for (int j = 0; j < b.n0; ++j)
        if (!(x_lo[j] <= x_hi[j])) return AS_ERR_ARG;
    int r = b.hn.init(net);
    if (r != AS_OK) return r;
    const int B = b.B = b.o.batch;
    const int NH = b.NH, n0 = b.n0;
    // the box and the property row repeated over the batch
    std::vector<float> lo((size_t)B * n0), hi((size_t)B * n0), C((size_t)B * b.nout);
    for (int q = 0; q < B; ++q) {
        std::memcpy(&lo[(size_t)q * n0], x_lo, n0 * 4);
        std::memcpy(&hi[(size_t)q * n0], x_hi, n0 * 4);
        for (int i = 0; i < b.nout; ++i) C[(size_t)q * b.nout + i] = (float)b.crow[i];
    }
    b.lo_d = b.dev<float>((size_t)B * n0);
    b.hi_d = b.dev<float>((size_t)B * n0);
    b.C_d = b.dev<float>((size_t)B * b.nout);
    b.lh_d = b.dev<float>((size_t)B * NH);
    b.uh_d = b.dev<float>((size_t)B * NH);
    b.al_d = b.dev<float>((size_t)B * NH);
    b.b0_d = b.dev<float>((size_t)B * NH);
    b.b1_d = b.dev<float>((size_t)B * NH);
    b.xs_d = b.dev<float>((size_t)B * b.NT);
    b.x0_d = b.dev<float>((size_t)B * n0);
    b.sp_d = b.dev<signed char>((size_t)B * NH);
    b.bd_d = b.dev<double>(B);
    b.ev_d = b.dev<double>(B);
    b.br_d = b.dev<int>(B);
    b.slot_d = b.dev<int>(B);
    if (!b.lo_d || !b.hi_d || !b.C_d || !b.lh_d || !b.uh_d || !b.al_d || !b.b0_d || !b.b1_d || !b.xs_d || !b.x0_d ||
        !b.sp_d || !b.bd_d || !b.ev_d || !b.br_d || !b.slot_d)
        return AS_ERR_OOM;
    if (cudaMemcpyAsync(b.lo_d, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice, b.st) != cudaSuccess ||
        cudaMemcpyAsync(b.hi_d, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice, b.st) != cudaSuccess ||
        cudaMemcpyAsync(b.C_d, C.data(), C.size() * 4, cudaMemcpyHostToDevice, b.st) != cudaSuccess)
        return AS_ERR_CUDA;
    b.sp_h.assign((size_t)B * NH, 0);
    if (b.o.root_intermediate) {
        std::vector<float> rl(NH), ru(NH);
        if ((r = as_intermediate_bounds(net, 1, x_lo, x_hi, nullptr, &b.o.intermediate, 0, rl.data(), ru.data(),
                                        stream)) != AS_OK)
            return r;
        b.rl_d = b.dev<float>(NH);
        b.ru_d = b.dev<float>(NH);
        if (!b.rl_d || !b.ru_d) return AS_ERR_OOM;
        if (cudaMemcpyAsync(b.rl_d, rl.data(), NH * 4, cudaMemcpyHostToDevice, b.st) != cudaSuccess ||
            cudaMemcpyAsync(b.ru_d, ru.data(), NH * 4, cudaMemcpyHostToDevice, b.st) != cudaSuccess)
            return AS_ERR_CUDA;
    }
    const bool strat = b.o.stratify != 0;
    as_options eo;
    as_default_options(&eo);
    eo.bigm_iters = eo.as_iters = 0;
    eo.graph_chunk = 0;
    if ((r = as_init(&b.ctx[1], net, B, b.lo_d, b.hi_d, b.C_d, nullptr, nullptr, nullptr, nullptr, &b.o.tight, stream)) !=
            AS_OK ||
        (strat && (r = as_init(&b.ctx[0], net, B, b.lo_d, b.hi_d, b.C_d, nullptr, nullptr, nullptr, nullptr, &b.o.loose,
                               stream)) != AS_OK) ||
        (r = as_init(&b.ev, net, B, b.lo_d, b.hi_d, b.C_d, nullptr, nullptr, nullptr, nullptr, &eo, stream)) != AS_OK)
        return r;

    std::vector<Domain> dom;
    dom.reserve(1024);
    dom.emplace_back();
    dom[0].splits.assign(NH, 0);
    std::vector<Domain*> jobs{&dom[0]};
    std::vector<int> none{-1};
    // the root: a_t, then a_l (whose duals the root keeps), timed for the cost ratio
    auto wall = [] { return std::chrono::steady_clock::now(); };
    auto t_a = wall();
    if ((r = b.bound(jobs, none, 1)) != AS_OK) return r;
    const double vt = dom[0].v;
    const double tt = std::chrono::duration<double>(wall() - t_a).count();
    double vl = vt, delta = 0.0, ratio = b.o.cost_ratio;
    if (strat) {
        t_a = wall();
        if ((r = b.bound(jobs, none, 0)) != AS_OK) return r;
        const double tl = std::chrono::duration<double>(wall() - t_a).count();
        vl = dom[0].v;
        delta = vt - vl;
        if (ratio <= 0) ratio = tl > 0 ? tt / tl : 1.0;
    }
    dom[0].v = vl;
    dom[0].lb = std::max(vl, vt);
    dom[0].alg = strat ? 0 : 1;
    dom[0].seq = 0;
    long long seq = 1;
    double lower_pruned = std::numeric_limits<double>::infinity();
    std::priority_queue<Entry> pool;
    std::vector<int> leaves;
    if (dom[0].lb > 0) lower_pruned = dom[0].lb;
    else pool.push({dom[0].lb, 0, 0});
    bool have_ema = false;
    double ema = 0.0;
    long long max_depth = 0;
    int status = AS_BAB_UNKNOWN;
    auto free_domain = [&](Domain& d) {
        if (d.slot >= 0) b.free_slots.push_back(d.slot);
        d.slot = -1;
        std::vector<signed char>().swap(d.splits);
    };
    while (true) {
        if (b.ub < 0) {
            status = AS_BAB_FALSIFIED;
            break;
        }
        if (pool.empty()) {
            status = leaves.empty() ? AS_BAB_VERIFIED : AS_BAB_UNKNOWN;
            break;
        }
        if (b.bounded >= b.o.max_domains) break;
        if (b.o.time_limit > 0 && std::chrono::duration<double>(wall() - t0).count() > b.o.time_limit) break;
        std::vector<int> parents;
        while (!pool.empty() && (int)parents.size() < B / 2) {
            parents.push_back(pool.top().idx);
            pool.pop();
        }
        struct Kid {
            int parent, idx;
        };
        std::vector<Kid> kids;
        for (int p : parents) {
            if (dom[p].branch < 0) {
                if (dom[p].rebounds < b.o.leaf_rebounds) {
                    Domain d;
                    d.splits = dom[p].splits;
                    d.hard = dom[p].hard;
                    d.alg = dom[p].alg;
                    d.rebounds = dom[p].rebounds + 1;
                    d.again = true;
                    d.depth = dom[p].depth;
                    d.seq = seq++;
                    dom.push_back(std::move(d));
                    kids.push_back({p, (int)dom.size() - 1});
                } else {
                    leaves.push_back(p);
                }
                continue;
            }
            for (int sgn : {1, -1}) {
                Domain d;
                d.splits = dom[p].splits;
                d.splits[dom[p].branch] = (signed char)sgn;
                d.hard = !strat || dom[p].hard || subtree_hard(dom[p].v, delta, have_ema, ema, ratio);
                d.alg = d.hard ? 1 : 0;
                d.depth = dom[p].depth + 1;
                d.seq = seq++;
                max_depth = std::max<long long>(max_depth, d.depth);
                dom.push_back(std::move(d));
                kids.push_back({p, (int)dom.size() - 1});
            }
        }
        for (int alg = 0; alg < 2; ++alg) {   // the easy batch, then the hard one
            std::vector<Domain*> js;
            std::vector<int> ps;
            for (auto& k : kids)
                if (dom[k.idx].alg == alg) {
                    js.push_back(&dom[k.idx]);
                    ps.push_back(dom[k.parent].slot);
                }
            if ((r = b.bound(js, ps, alg)) != AS_OK) return r;
        }
        for (auto& k : kids) {
            Domain& c = dom[k.idx];
            const Domain& p = dom[k.parent];
            c.lb = std::max(c.v, p.lb);
            if (c.alg == p.alg && !c.again) {
                const double d = c.v - p.v;
                ema = have_ema ? (1 - b.o.ema_weight) * ema + b.o.ema_weight * d : d;
                have_ema = true;
            }
            if (c.lb > 0) {
                lower_pruned = std::min(lower_pruned, c.lb);
                free_domain(c);
            } else {
                pool.push({c.lb, c.seq, k.idx});
            }
        }
        for (int p : parents)
            if (std::find(leaves.begin(), leaves.end(), p) == leaves.end()) free_domain(dom[p]);
    }
    double lower = std::numeric_limits<double>::infinity();
    long long frontier = 0;
    while (!pool.empty()) {
        lower = std::min(lower, pool.top().lb);
        pool.pop();
        ++frontier;
    }
    for (int p : leaves) lower = std::min(lower, dom[p].lb), ++frontier;
    if (frontier == 0) lower = lower_pruned;
    res->status = status;
    res->lower = lower;
    res->upper = b.ub;
    res->bounded = b.bounded;
    res->hard_bounded = b.hard_bounded;
    res->batches = b.batches;
    res->max_depth = max_depth;
    res->frontier = frontier;
    res->cost_ratio = strat ? ratio : 0.0;
    res->seconds = std::chrono::duration<double>(wall() - t0).count();
    if (x_best && !b.x_ub.empty()) std::memcpy(x_best, b.x_ub.data(), n0 * 4);
    return AS_OK;
}

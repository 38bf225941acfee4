// Host side of the convex-barrier C ABI (include/convex_barrier.h): context creation, buffer
// layout in device memory, the Big-M / Active Set and Saddle Point iteration loops (optionally
// captured as CUDA graphs), bound evaluation and state access.
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/convex_barrier.h"
#include "cb_kernels.cuh"
#include "cb_backward.cuh"
#include "cb_team.cuh"
#include "cb_tc.cuh"

using namespace cb;

struct as_ctx {
    DNet net{};
    DState st{};
    DSched sc{};
    as_options opt{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<void*> allocs;
    std::string err;
    int n_out = 0;                 // outputs of the last layer (before the property rows)
    std::vector<as_layer> layers;  // shapes (pointers not kept)
    std::vector<int> widths;       // neuron layers 0..n-1
    bool sp_started = false;
    bool bounds_ibp = true;        // lhat, uhat of the batch came from interval propagation
    bool have_splits = false;      // ... with the split clamps of splits_dev
    bool sp_need_phaseA = true;    // the next Saddle Point iteration starts with a separate phase A
    long long launches = 0;
    Segs segA{}, segB{};
    int blocksA = 0, blocksB = 0;
    TSegs tA{}, tB{};                // lane-team launch geometry of the Active Set passes
    int blocksTA = 0, blocksTB = 0;
    cudaGraphExec_t g_as = nullptr, g_sp = nullptr;
    int g_as_len = 0, g_sp_len = 0, g_as_nodes = 0, g_sp_nodes = 0;
    float* Wlast = nullptr;        // original last layer [n_out][n_{n-1}] and bias
    float* blast = nullptr;
    float* C = nullptr;            // property rows [S][n_out]
    int* caps_dev = nullptr;
    signed char* splits_dev = nullptr;
    double* bound_out = nullptr;   // [S] device result of the last as_bound
    char* zero_arena = nullptr;
    char* work_arena = nullptr;
    size_t zero_bytes = 0;
    // per-kernel CUDA-event timing (as_options.profile)
    struct Rec { int id; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double prof_ms[CB_NPROF] = {};
    long long prof_n[CB_NPROF] = {};
    // BF16 form (as_options.precision = 16)
    struct TcGemm {
        tc::GemmGroup g;
        int ng, maxM, bn;
        int win = 0, mt = 1, smem = 0;   // window operands (k_gemm_wgroup_bf16): row blocks per CTA, bytes
    };
    std::vector<TcGemm> tc_row, tc_col;           // per hidden-output layer
    std::vector<TcGemm> tc_row_alt, tc_col_alt;   // gathered-operand plans beside window ones (autotune)
    std::vector<std::pair<void*, size_t>> planes; // bf16 operand planes, cleared with each batch
    int* tc_status = nullptr;                     // set by a tensor-core kernel whose wait ran out
    TSegs tA1{}, tB1{};                           // one lane per unit
    int blocksTA1 = 0, blocksTB1 = 0;
    long long team_row = 40000, team_col = 40000; // team-size targets of the float32 passes
    uint32_t tc_stage_limit = tc::TC_WAIT_LIMIT;  // try_wait rounds of the GEMMs' stage waits
    // conv products of the BF16 form by window operands where their taps are shifts of one grid
    // (environment CB_TC_WINDOWS = 0: the gathered operands everywhere, to compare the two)
    bool tc_windows = true;
    // host-side fault injection for tests (environment CB_FAIL_ALLOC_AT = n): the n-th device
    // allocation of the context is refused as if the device were out of memory
    long long fail_alloc_at = 0, alloc_calls = 0;
};

static int fail(as_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CUDA_TRY(c, call)                                                                    \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((c), e_ == cudaErrorMemoryAllocation ? AS_ERR_OOM : AS_ERR_CUDA,     \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                     \
    } while (0)

template <class T>
static int dalloc(as_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    if (++c->alloc_calls == c->fail_alloc_at)
        return fail(c, AS_ERR_OOM, "device allocation %lld (%zu bytes) refused by CB_FAIL_ALLOC_AT", c->alloc_calls,
                    bytes);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess)
        return fail(c, e == cudaErrorMemoryAllocation ? AS_ERR_OOM : AS_ERR_CUDA,
                    "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    c->allocs.push_back(q);
    *p = (T*)q;
    return AS_OK;
}

#define TRY(x)                    \
    do {                          \
        int r_ = (x);             \
        if (r_ != AS_OK) return r_; \
    } while (0)

// defined further down (cb_bf16.inc, cb_host_extra.inc)
static int clear_planes(as_ctx* c);
static int build_bf16(as_ctx* c, const std::vector<std::vector<float>>& Wh);
static int autotune_tc(as_ctx* c);
static int recompute_slot_sums(as_ctx* c);

extern "C" void as_default_options(as_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->bigm_iters = 500;
    o->as_iters = 1000;
    o->bigm_lr0 = 1e-2;
    o->bigm_lr1 = 1e-4;
    o->as_lr0 = 1e-3;
    o->as_lr1 = 1e-6;
    o->omega = 450;
    o->vars_per_add = 2;
    o->max_cuts = 7;
    o->adam_b1 = 0.9;
    o->adam_b2 = 0.999;
    o->adam_eps = 1e-8;
    o->sp_gamma0 = 10.0;
    o->sp_c_alpha = 1e-3;
    o->sp_c_beta = 1e-3;
    o->sp_init_steps = 100;
    o->sp_init_lr0 = 1e-2;
    o->sp_init_lr1 = 1e-5;
    o->track_best = 0;
    o->graph_chunk = 16;
    o->precision = 32;
    o->input_l2 = 0;
}

extern "C" const char* as_last_error(as_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" int as_team_targets(as_ctx* c, long long* row, long long* col) {
    if (!c || !row || !col) return AS_ERR_ARG;
    *row = c->team_row;
    *col = c->team_col;
    return AS_OK;
}
extern "C" long long as_launch_count(as_ctx* c) { return c ? c->launches : -1; }

static int check_launch(as_ctx* c, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, AS_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return AS_OK;
}

// Segment tables: one launch covers several layers, each layer a contiguous block range.
static void make_segs(Segs& sg, int& blocks, const std::vector<int>& layer_ids,
                      const std::vector<long long>& units, int units_per_block) {
    sg.n = (int)layer_ids.size();
    int b = 0;
    for (int q = 0; q < sg.n; ++q) {
        sg.layer[q] = layer_ids[q];
        sg.start[q] = b;
        b += (int)((units[q] + units_per_block - 1) / units_per_block);
    }
    sg.start[sg.n] = b;
    blocks = b;
}

static int validate_net(as_ctx* c, const as_net* net) {
    if (!net || !net->layers) return fail(c, AS_ERR_ARG, "net is null");
    const int n = net->n_layers;
    if (n < 2 || n > AS_MAX_LAYERS) return fail(c, AS_ERR_SHAPE, "n_layers = %d not in [2, %d]", n, AS_MAX_LAYERS);
    int prev = -1;
    for (int k = 0; k < n; ++k) {
        const as_layer& L = net->layers[k];
        if (!L.W || !L.b) return fail(c, AS_ERR_ARG, "layer %d: null W or b", k + 1);
        int nin, nout;
        if (L.kind == AS_LAYER_LINEAR) {
            nin = L.in_c;
            nout = L.out_c;
            if (nin < 1 || nout < 1) return fail(c, AS_ERR_SHAPE, "layer %d: bad linear shape", k + 1);
        } else if (L.kind == AS_LAYER_CONV2D) {
            if (k == n - 1) return fail(c, AS_ERR_SHAPE, "the last layer must be linear");
            if (L.in_c < 1 || L.in_h < 1 || L.in_w < 1 || L.out_c < 1 || L.kh < 1 || L.kw < 1 ||
                L.stride < 1 || L.pad < 0)
                return fail(c, AS_ERR_SHAPE, "layer %d: bad conv shape", k + 1);
            const int oh = (L.in_h + 2 * L.pad - L.kh) / L.stride + 1;
            const int ow = (L.in_w + 2 * L.pad - L.kw) / L.stride + 1;
            if (oh < 1 || ow < 1 || oh != L.out_h || ow != L.out_w)
                return fail(c, AS_ERR_SHAPE, "layer %d: conv output %dx%d, given %dx%d", k + 1, oh, ow,
                            L.out_h, L.out_w);
            nin = L.in_c * L.in_h * L.in_w;
            nout = L.out_c * oh * ow;
        } else {
            return fail(c, AS_ERR_ARG, "layer %d: unknown kind %d", k + 1, L.kind);
        }
        if (prev >= 0 && nin != prev)
            return fail(c, AS_ERR_SHAPE, "layer %d takes %d inputs, previous layer gives %d", k + 1, nin, prev);
        prev = nout;
        c->layers.push_back(L);
        if (k == 0) c->widths.push_back(nin);
        if (k < n - 1) c->widths.push_back(nout);
    }
    c->n_out = prev;
    return AS_OK;
}

static int validate_opt(as_ctx* c, const as_options& o) {
    if (o.bigm_iters < 0 || o.as_iters < 0) return fail(c, AS_ERR_ARG, "negative iteration counts");
    if (o.max_cuts < 0 || o.max_cuts > AS_MAX_CUTS) return fail(c, AS_ERR_ARG, "max_cuts not in [0, %d]", AS_MAX_CUTS);
    if (o.vars_per_add < 1) return fail(c, AS_ERR_ARG, "vars_per_add < 1");
    if (o.omega > 0 && o.omega < o.vars_per_add) return fail(c, AS_ERR_ARG, "omega < vars_per_add");
    if (!(o.adam_b1 >= 0 && o.adam_b1 < 1 && o.adam_b2 >= 0 && o.adam_b2 < 1 && o.adam_eps > 0))
        return fail(c, AS_ERR_ARG, "bad Adam parameters");
    if (!(o.sp_gamma0 >= 1)) return fail(c, AS_ERR_ARG, "sp_gamma0 < 1");
    if (!(o.sp_c_alpha > 0 && o.sp_c_beta > 0)) return fail(c, AS_ERR_ARG, "price-cap constants must be > 0");
    if (o.sp_init_steps < 0 || o.graph_chunk < 0) return fail(c, AS_ERR_ARG, "negative step counts");
    if (o.precision != 32 && o.precision != 16) return fail(c, AS_ERR_ARG, "precision must be 32 or 16");
    if (o.input_l2 != 0 && o.input_l2 != 1) return fail(c, AS_ERR_ARG, "input_l2 must be 0 or 1");
    return AS_OK;
}

static int build_tables(as_ctx* c) {
    const as_options& o = c->opt;
    const int ntab = o.bigm_iters + o.as_iters + 2;
    std::vector<float> lr(ntab), b1(ntab), b2(ntab);
    const double lr_end = o.as_iters > 0 ? o.as_lr1 : o.bigm_lr1;
    for (int it = 0; it < ntab; ++it) {
        double v;
        if (it < o.bigm_iters) v = o.bigm_lr0 + (o.bigm_lr1 - o.bigm_lr0) * it / std::max(1, o.bigm_iters - 1);
        else if (it - o.bigm_iters < o.as_iters)
            v = o.as_lr0 + (o.as_lr1 - o.as_lr0) * (it - o.bigm_iters) / std::max(1, o.as_iters - 1);
        else v = lr_end;
        lr[it] = (float)v;
        // reciprocal bias corrections 1 / (1 - beta^step); entry 0 is never used
        b1[it] = it ? (float)(1.0 / (1.0 - std::pow(o.adam_b1, (double)it))) : 1.f;
        b2[it] = it ? (float)(1.0 / (1.0 - std::pow(o.adam_b2, (double)it))) : 1.f;
    }
    float *dlr, *db1, *db2;
    TRY(dalloc(c, &dlr, ntab));
    TRY(dalloc(c, &db1, ntab));
    TRY(dalloc(c, &db2, ntab));
    CUDA_TRY(c, cudaMemcpyAsync(dlr, lr.data(), ntab * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(db1, b1.data(), ntab * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(db2, b2.data(), ntab * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // host vectors go out of scope
    c->st.lr_tab = dlr;
    c->st.bc1_tab = db1;
    c->st.bc2_tab = db2;
    DSched& d = c->sc;
    d.TM = o.bigm_iters;
    d.TA = o.as_iters;
    d.omega = o.omega;
    d.vpa = o.vars_per_add;
    d.maxcut = o.max_cuts;
    d.ntab = ntab;
    d.b1 = (float)o.adam_b1;
    d.omb1 = (float)(1.0 - o.adam_b1);
    d.b2 = (float)o.adam_b2;
    d.omb2 = (float)(1.0 - o.adam_b2);
    d.eps = (float)o.adam_eps;
    d.lr_as_end = (float)lr_end;
    d.gamma0 = (float)o.sp_gamma0;
    d.sp_init_steps = o.sp_init_steps;
    d.sp_lr0 = (float)o.sp_init_lr0;
    d.sp_lr1 = (float)o.sp_init_lr1;
    return AS_OK;
}

static int grid_for(size_t n) { return (int)std::min<size_t>((n + CB_THREADS - 1) / CB_THREADS, 152 * 16); }


// Device state in two arenas: the "zeroed" arena holds everything a new batch starts from zero
// (duals, Adam moments, slots, snapshots, Saddle Point statistics, counters), so that a reset is
// one memset; the other arena holds buffers each batch overwrites before reading.
struct Bump {
    char* base;
    size_t off;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base + off);
        off += count * sizeof(T);
        return p;
    }
};

// Sign-partitioned tap lists and record layouts of the Active Set walks (DLayer fields) for the
// hidden-output layers. Taps index record positions: the input records (one float2 each) for the
// row pass, the output records (RS / 4 float4 planes) for the col pass.
static int build_walks(as_ctx* c, const std::vector<std::vector<float>>& Wh) {
    DNet& D = c->net;
    const int RS = D.RS;
    int xo = 0, ao = 0;
    for (int k = 0; k + 1 < D.n; ++k) {
        DLayer& L = D.L[k];
        const std::vector<float>& W = Wh[k];
        std::vector<int2> rt, ct, pos, neg;
        std::vector<int> rg, cg;
        auto close_group = [&](std::vector<int2>& taps, std::vector<int>& grp) {
            grp.push_back((int)taps.size());
            taps.insert(taps.end(), pos.begin(), pos.end());
            grp.push_back((int)taps.size());
            taps.insert(taps.end(), neg.begin(), neg.end());
            pos.clear();
            neg.clear();
        };
        auto add = [&](int off, float w) {
            int2 e;
            e.x = off;
            std::memcpy(&e.y, &w, sizeof w);
            if (w > 0.f) pos.push_back(e);
            else if (w < 0.f) neg.push_back(e);
        };
        int xpos, apos;
        if (L.kind == 0) {
            L.Hp = L.Wp = L.Hpo = L.Wpo = 1;
            L.hl = L.wl = 0;
            for (int i = 0; i < L.n_out; ++i) {
                for (int j = 0; j < L.n_in; ++j) add(j, W[(size_t)i * L.n_in + j]);
                close_group(rt, rg);
            }
            for (int j = 0; j < L.n_in; ++j) {
                for (int i = 0; i < L.n_out; ++i) add(i, W[(size_t)i * L.n_in + j]);
                close_group(ct, cg);
            }
            xpos = L.n_in;
            apos = L.n_out;
        } else {
            L.Hp = L.hi + 2 * L.pd;
            L.Wp = L.wi + 2 * L.pd;
            // col pass: input (y, x) of stride phase (py, px) reaches outputs (Y0 - dky, X0 - dkx),
            // Y0 = (y + pad) / stride, kernel row py + stride dky; the halo holds the out-of-range ones
            const int nky = (L.kh + L.st - 1) / L.st, nkx = (L.kw + L.st - 1) / L.st;
            const int maxY0 = (L.hi - 1 + L.pd) / L.st, maxX0 = (L.wi - 1 + L.pd) / L.st;
            L.hl = nky - 1;
            L.wl = nkx - 1;
            L.Hpo = L.hl + std::max(L.ho, maxY0 + 1);
            L.Wpo = L.wl + std::max(L.wo, maxX0 + 1);
            const size_t kk = (size_t)L.kh * L.kw;
            for (int co = 0; co < L.co; ++co) {
                for (int ci = 0; ci < L.ci; ++ci)
                    for (int ky = 0; ky < L.kh; ++ky)
                        for (int kx = 0; kx < L.kw; ++kx)
                            add((ci * L.Hp + ky) * L.Wp + kx,
                                W[((size_t)co * L.ci + ci) * kk + ky * L.kw + kx]);
                close_group(rt, rg);
            }
            for (int ci = 0; ci < L.ci; ++ci)
                for (int py = 0; py < L.st; ++py)
                    for (int px = 0; px < L.st; ++px) {
                        for (int co = 0; co < L.co; ++co)
                            for (int ky = py, dky = 0; ky < L.kh; ky += L.st, ++dky)
                                for (int kx = px, dkx = 0; kx < L.kw; kx += L.st, ++dkx)
                                    add(co * L.Hpo * L.Wpo - dky * L.Wpo - dkx,
                                        W[((size_t)co * L.ci + ci) * kk + ky * L.kw + kx]);
                        close_group(ct, cg);
                    }
            xpos = L.ci * L.Hp * L.Wp;
            apos = L.co * L.Hpo * L.Wpo;
        }
        rg.push_back((int)rt.size());
        cg.push_back((int)ct.size());
        int2 *drt, *dct;
        int *drg, *dcg;
        TRY(dalloc(c, &drt, rt.size()));
        TRY(dalloc(c, &dct, ct.size()));
        TRY(dalloc(c, &drg, rg.size()));
        TRY(dalloc(c, &dcg, cg.size()));
        CUDA_TRY(c, cudaMemcpy(drt, rt.data(), rt.size() * sizeof(int2), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(dct, ct.data(), ct.size() * sizeof(int2), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(drg, rg.data(), rg.size() * sizeof(int), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(dcg, cg.data(), cg.size() * sizeof(int), cudaMemcpyHostToDevice));
        L.rtap = drt;
        L.rgrp = drg;
        L.ctap = dct;
        L.cgrp = dcg;
        L.xo = xo;
        L.ao = ao;
        L.xpos = xpos;
        L.apos = apos;
        const long long xn = (long long)xo + (long long)xpos * 2, an = (long long)ao + (long long)apos * RS;
        if (xn > INT32_MAX / 2 || an > INT32_MAX / 2)
            return fail(c, AS_ERR_SHAPE, "layer %d: record offsets exceed 32 bits", k + 1);
        xo = (int)xn;
        ao = (int)an;
    }
    D.XT = xo;
    D.AT = ao;
    return AS_OK;
}

// Team size for a pass with `units` reductions of about `fan` terms each: enough lanes to fill the
// GPU (about 152 SMs x 1024 threads), at least 8 terms per lane, a power of two up to a warp.
static int team_size(long long units, long long fan, long long target) {
    int T = 1;
    while (T < 32 && units * T < target && fan / (2 * T) >= 8) T *= 2;
    return T;
}

// Threads a layer's segment aims for, row and col passes (as_options.autotune picks them per
// context; the default was measured on the Wide conv net with 9 subproblems: about a quarter of
// the threads the GPU holds at once, teams long enough to keep loads in flight, short enough not
// to replicate per-unit work). CB_TEAM_TARGET_ROW / CB_TEAM_TARGET_COL override them.
static int make_team_segs(as_ctx* c) {
    DNet& D = c->net;
    const int n = D.n, S = D.S;
    long long target_row = c->team_row, target_col = c->team_col;
    if (const char* e = getenv("CB_TEAM_TARGET_ROW")) target_row = atoll(e) > 0 ? atoll(e) : target_row;
    if (const char* e = getenv("CB_TEAM_TARGET_COL")) target_col = atoll(e) > 0 ? atoll(e) : target_col;
    c->team_row = target_row;   // the targets in effect (as_team_targets)
    c->team_col = target_col;
    auto build = [&](TSegs& sg, int& blocks, bool col) -> int {
        const int nseg = col ? n : n - 1;
        sg.n = nseg;
        int b = 0;
        for (int k = 0; k < nseg; ++k) {
            const DLayer& L = D.L[k];
            const long long units = (long long)S * (col ? L.n_in : L.n_out);
            long long fan;
            if (L.kind == 0) fan = col ? L.n_out : L.n_in;
            else fan = col ? (long long)L.co * ((L.kh + L.st - 1) / L.st) * ((L.kw + L.st - 1) / L.st)
                           : (long long)L.ci * L.kh * L.kw;
            int T = (col && k == n - 1) ? 1 : team_size(units, fan, col ? target_col : target_row);
            // conv row-pass lanes split (channel, kernel row) pairs; col-pass lanes split channels
            const long long split = L.kind == 0 ? fan : (col ? L.co : (long long)L.ci * L.kh);
            while (T > 1 && T > split) T >>= 1;
            sg.layer[k] = k;
            sg.T[k] = T;
            sg.start[k] = b;
            sg.perm[k] = nullptr;
            b += (int)((units * T + CB_THREADS - 1) / CB_THREADS);
            if (col && L.kind == 1 && L.st > 1) {
                std::vector<int> perm;
                perm.reserve(L.n_in);
                for (int py = 0; py < L.st; ++py)
                    for (int px = 0; px < L.st; ++px)
                        for (int ch = 0; ch < L.ci; ++ch)
                            for (int y = py; y < L.hi; y += L.st)
                                for (int x = px; x < L.wi; x += L.st) perm.push_back((ch * L.hi + y) * L.wi + x);
                int* dp;
                TRY(dalloc(c, &dp, perm.size()));
                CUDA_TRY(c, cudaMemcpy(dp, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice));
                sg.perm[k] = dp;
            }
        }
        sg.start[nseg] = b;
        blocks = b;
        return AS_OK;
    };
    TRY(build(c->tA, c->blocksTA, true));
    TRY(build(c->tB, c->blocksTB, false));
    return AS_OK;
}

static int alloc_state(as_ctx* c) {
    DNet& D = c->net;
    DState& st = c->st;
    const size_t S = D.S, NT = D.NT, NH = D.NH;
    const size_t NTS = S * NT, NHS = S * NH, SL = S * D.cap * NH;
    const int n = D.n;
    for (int pass = 0; pass < 2; ++pass) {
        Bump z{pass ? c->zero_arena : nullptr, 0};
        float** zf[] = {&st.alpha, &st.beta0, &st.beta1, &st.ma, &st.va, &st.m0, &st.v0, &st.m1, &st.v1,
                        &st.Sb, &st.G, &st.C, &st.mua, &st.mub, &st.ab, &st.b0i, &st.b1i};
        for (float** p : zf) *p = z.take<float>(NHS);
        float** zs[] = {&st.bs, &st.ms, &st.vs, &st.lam, &st.kap};
        for (float** p : zs) *p = z.take<float>(SL);
        st.P = z.take<float>(NTS);
        st.arec = z.take<float>(S * (size_t)D.AT);
        st.xin = z.take<float>(S * (size_t)D.XT);
        st.spin = z.take<float4>(S * (size_t)D.XT);
        for (int q = 0; q < 2; ++q) {
            st.xsnap[q] = z.take<uint8_t>(NTS);
            st.zsnap[q] = z.take<uint8_t>(NHS);
        }
        st.ctr = z.take<int>(4);
        st.status = z.take<int>(1);
        Bump o{pass ? c->work_arena : nullptr, 0};
        st.lo = o.take<float>(NTS);
        st.hi = o.take<float>(NTS);
        st.lhat = o.take<float>(NHS);
        st.uhat = o.take<float>(NHS);
        st.xval = o.take<float>(NTS);
        st.fval = o.take<float>(NTS);
        st.xbar = o.take<float>(NTS);
        for (int q = 0; q < 2; ++q) {
            st.spx[q] = o.take<float>(NTS);
            st.spz[q] = o.take<float>(NHS);
        }
        st.zcur = o.take<uint8_t>(NHS);
        st.lz = o.take<float>(NHS);
        st.uz = o.take<float>(NHS);
        st.brad = o.take<float>(NHS);
        st.bnrm = o.take<double>(S);
        st.efix = o.take<uint8_t>(NTS);
        st.arow = o.take<float>(NHS);
        st.nfree = o.take<int>(NHS);
        st.zbar = o.take<uint8_t>(NHS);
        st.sel = o.take<uint8_t>(NHS);
        st.terms = o.take<double>(NTS);
        st.best = o.take<double>(S);
        D.Wout = o.take<float>(S * c->widths[n - 1]);
        D.bout = o.take<float>(S);
        c->caps_dev = o.take<int>(S);
        c->C = o.take<float>(S * c->n_out);
        c->splits_dev = o.take<signed char>(NHS);
        c->bound_out = o.take<double>(S);
        st.caps = c->caps_dev;
        if (pass == 0) {
            c->zero_bytes = z.off;
            TRY(dalloc(c, &c->zero_arena, z.off));
            TRY(dalloc(c, &c->work_arena, o.off));
        }
    }
    CUDA_TRY(c, cudaMemsetAsync(c->st.terms, 0, NTS * sizeof(double), c->stream));
    return AS_OK;
}

// Per-kernel timing: with as_options.profile set, each launch is bracketed by CUDA events on its
// stream; as_kernel_times reads and accumulates them.
static cudaEvent_t prof_event(as_ctx* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

#define LAUNCH(c, s, id, ...)                                      \
    do {                                                           \
        if ((c)->opt.profile) {                                    \
            as_ctx::Rec r_{id, prof_event(c), prof_event(c)};      \
            cudaEventRecord(r_.a, s);                              \
            __VA_ARGS__;                                           \
            cudaEventRecord(r_.b, s);                              \
            (c)->pending.push_back(r_);                            \
        } else {                                                   \
            __VA_ARGS__;                                           \
        }                                                          \
        (c)->launches++;                                           \
    } while (0)

// Box, property rows, intermediate bounds, splits and caps of a batch; zeroes the duals.
static int load_batch(as_ctx* c, const float* x_lo, const float* x_hi, const float* C, const float* lhat,
                      const float* uhat, const signed char* splits, const int* caps, bool host_checks) {
    if (!x_lo || !x_hi) return fail(c, AS_ERR_ARG, "null input box");
    if ((lhat == nullptr) != (uhat == nullptr)) return fail(c, AS_ERR_ARG, "give both lhat and uhat or neither");
    if (!C && c->n_out != 1) return fail(c, AS_ERR_ARG, "C is null but the last layer has %d outputs", c->n_out);
    DNet& D = c->net;
    DState& st = c->st;
    const int S = D.S, n = D.n, n0 = c->widths[0];
    const size_t NT = D.NT, NHS = (size_t)S * D.NH;
    cudaStream_t s = c->stream;
    CUDA_TRY(c, cudaMemsetAsync(c->zero_arena, 0, c->zero_bytes, s));
    TRY(clear_planes(c));
    c->bounds_ibp = lhat == nullptr;
    c->have_splits = splits != nullptr && lhat == nullptr;
    LAUNCH(c, s, CB_K_BATCH, (k_fill<<<grid_for(S), CB_THREADS, 0, s>>>(st.best, (size_t)S, -INFINITY)));
    c->sp_started = false;
    if (host_checks) {
        std::vector<float> hl((size_t)S * n0), hh((size_t)S * n0);
        CUDA_TRY(c, cudaMemcpyAsync(hl.data(), x_lo, hl.size() * sizeof(float), cudaMemcpyDefault, s));
        CUDA_TRY(c, cudaMemcpyAsync(hh.data(), x_hi, hh.size() * sizeof(float), cudaMemcpyDefault, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        for (size_t q = 0; q < hl.size(); ++q)
            if (!(hl[q] <= hh[q]) || !std::isfinite(hl[q]) || !std::isfinite(hh[q]))
                return fail(c, AS_ERR_ARG, "input box entry %zu: lo = %g, hi = %g", q, hl[q], hh[q]);
        if (caps) {
            std::vector<int> hc(S);
            CUDA_TRY(c, cudaMemcpyAsync(hc.data(), caps, S * sizeof(int), cudaMemcpyDefault, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            for (int q = 0; q < S; ++q)
                if (hc[q] < 0 || hc[q] > c->opt.max_cuts)
                    return fail(c, AS_ERR_ARG, "caps[%d] = %d not in [0, max_cuts]", q, hc[q]);
        }
    }
    // box into the layer-0 part of the [S][NT] bound vectors
    CUDA_TRY(c, cudaMemcpy2DAsync(st.lo, NT * sizeof(float), x_lo, n0 * sizeof(float), n0 * sizeof(float), S,
                                  cudaMemcpyDefault, s));
    CUDA_TRY(c, cudaMemcpy2DAsync(st.hi, NT * sizeof(float), x_hi, n0 * sizeof(float), n0 * sizeof(float), S,
                                  cudaMemcpyDefault, s));
    if (!host_checks) {
        LAUNCH(c, s, CB_K_BATCH, (k_check_box<<<grid_for((size_t)S * n0), CB_THREADS, 0, s>>>(D, st)));
    }
    if (caps) CUDA_TRY(c, cudaMemcpyAsync(c->caps_dev, caps, S * sizeof(int), cudaMemcpyDefault, s));
    else {
        LAUNCH(c, s, CB_K_BATCH, (k_fill_int<<<grid_for(S), CB_THREADS, 0, s>>>(c->caps_dev, (size_t)S, c->opt.max_cuts)));
    }
    if (C) CUDA_TRY(c, cudaMemcpyAsync(c->C, C, (size_t)S * c->n_out * sizeof(float), cudaMemcpyDefault, s));
    LAUNCH(c, s, CB_K_BATCH, (k_fold<<<S, CB_THREADS, 0, s>>>(D, c->Wlast, c->blast, C ? c->C : nullptr, c->n_out,
                                                             (float*)D.Wout, (float*)D.bout)));
    TRY(check_launch(c, "k_fold"));
    if (lhat) {
        CUDA_TRY(c, cudaMemcpyAsync(st.lhat, lhat, NHS * sizeof(float), cudaMemcpyDefault, s));
        CUDA_TRY(c, cudaMemcpyAsync(st.uhat, uhat, NHS * sizeof(float), cudaMemcpyDefault, s));
        if (host_checks) {
            std::vector<float> a(NHS), b(NHS);
            CUDA_TRY(c, cudaMemcpyAsync(a.data(), st.lhat, NHS * sizeof(float), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(c, cudaMemcpyAsync(b.data(), st.uhat, NHS * sizeof(float), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            for (size_t q = 0; q < NHS; ++q)
                if (!(a[q] <= b[q])) return fail(c, AS_ERR_ARG, "lhat > uhat at hidden entry %zu", q);
        }
        LAUNCH(c, s, CB_K_BATCH, (k_post_from_pre<<<grid_for(NHS), CB_THREADS, 0, s>>>(D, st)));
        TRY(check_launch(c, "k_post_from_pre"));
    } else {
        const signed char* dsp = nullptr;
        if (splits) {
            CUDA_TRY(c, cudaMemcpyAsync(c->splits_dev, splits, NHS, cudaMemcpyDefault, s));
            dsp = c->splits_dev;
        }
        for (int k = 0; k < n - 1; ++k) {
            const long long warps = (long long)S * D.L[k].n_out;
            LAUNCH(c, s, CB_K_BATCH, (k_ibp<<<(int)((warps + CB_WARPS - 1) / CB_WARPS), CB_THREADS, 0, s>>>(D, st, k, dsp)));
            TRY(check_launch(c, "k_ibp"));
        }
    }
    LAUNCH(c, s, CB_K_BATCH, (k_efix<<<grid_for((size_t)S * NT), CB_THREADS, 0, s>>>(D, st)));
    TRY(check_launch(c, "k_efix"));
    // interval propagation computed lz, uz and the free counts with its own sums; caller-given bounds,
    // and layer 1 over an ellipsoid (whose interval comes from other sums), need k_lz
    for (int k = 0; k < n - 1; ++k) {
        if (!lhat && !(D.ball && k == 0)) continue;
        const long long warps = (long long)S * D.L[k].n_out;
        LAUNCH(c, s, CB_K_BATCH, (k_lz<<<(int)((warps + CB_WARPS - 1) / CB_WARPS), CB_THREADS, 0, s>>>(D, st, k)));
        TRY(check_launch(c, "k_lz"));
    }
    return AS_OK;
}

extern "C" int as_reset(as_ctx* c, const float* x_lo, const float* x_hi, const float* C, const float* lhat,
                        const float* uhat, const signed char* splits, const int* caps) {
    if (!c) return AS_ERR_ARG;
    if (!c->zero_arena) return fail(c, AS_ERR_STATE, "context was not initialised");
    return load_batch(c, x_lo, x_hi, C, lhat, uhat, splits, caps, false);
}

static int launch_as_iter(as_ctx* c, cudaStream_t s);

// Device time of `reps` float32 Active Set iterations at the last planned iteration (every slot in
// use: the walks' cost does not depend on the dual values), after one untimed iteration.
static int time_iters(as_ctx* c, int reps, float* ms);

// Device time per iteration, over at least `reps` iterations and about 2 ms (small workloads
// iterate in tens of microseconds: a few iterations alone would measure noise).
static int time_per_iter(as_ctx* c, float* ms_per) {
    float ms = 0.f;
    TRY(time_iters(c, 4, &ms));
    int reps = 4;
    if (ms < 2.f) {
        reps = (int)std::min(256.f, std::ceil(4.f * 2.f / std::max(ms, 1e-3f)));
        TRY(time_iters(c, reps, &ms));
    }
    *ms_per = ms / reps;
    return AS_OK;
}

static int time_iters(as_ctx* c, int reps, float* ms) {
    const int it = c->sc.ntab - 2 > 0 ? c->sc.ntab - 2 : 0;
    int w[3] = {it, 0, 0};
    CUDA_TRY(c, cudaMemcpyAsync(c->st.ctr, w, sizeof w, cudaMemcpyHostToDevice, c->stream));
    TRY(launch_as_iter(c, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->st.ctr, w, sizeof w, cudaMemcpyHostToDevice, c->stream));
    cudaEvent_t a, b;
    CUDA_TRY(c, cudaEventCreate(&a));
    CUDA_TRY(c, cudaEventCreate(&b));
    CUDA_TRY(c, cudaEventRecord(a, c->stream));
    int r = AS_OK;
    for (int q = 0; q < reps && r == AS_OK; ++q) r = launch_as_iter(c, c->stream);
    cudaEventRecord(b, c->stream);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r != AS_OK) return r;
    if (e != cudaSuccess) return fail(c, AS_ERR_CUDA, "autotune timing failed: %s", cudaGetErrorString(e));
    return AS_OK;
}

// as_options.autotune: the team-size targets of the col pass, then of the row pass, each the
// fastest of a doubling sequence on this context's own net and batch. The caller reloads the
// batch afterwards (the timing iterations move the duals).
static int autotune_teams(as_ctx* c) {
    static const long long cand[] = {5000, 10000, 20000, 40000, 80000, 160000, 320000};
    const bool prof = c->opt.profile != 0;
    c->opt.profile = 0;
    for (int pass = 0; pass < 2; ++pass) {
        // a target pinned by CB_TEAM_TARGET_COL / CB_TEAM_TARGET_ROW is not tuned
        if (getenv(pass ? "CB_TEAM_TARGET_ROW" : "CB_TEAM_TARGET_COL")) continue;
        long long best = pass ? c->team_row : c->team_col;
        float best_ms = 0.f;
        for (long long t : cand) {
            (pass ? c->team_row : c->team_col) = t;
            TRY(make_team_segs(c));
            float ms = 0.f;
            TRY(time_per_iter(c, &ms));
            if (best_ms == 0.f || ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
        (pass ? c->team_row : c->team_col) = best;
    }
    c->opt.profile = prof ? 1 : 0;
    return make_team_segs(c);
}

static int init_impl(as_ctx* c, const as_net* net, int S, const float* x_lo, const float* x_hi, const float* C,
                     const float* lhat, const float* uhat, const signed char* splits, const int* caps,
                     const as_options* opt) {
    if (S < 1) return fail(c, AS_ERR_ARG, "S = %d < 1", S);
    if (!x_lo || !x_hi) return fail(c, AS_ERR_ARG, "null input box");
    if ((lhat == nullptr) != (uhat == nullptr)) return fail(c, AS_ERR_ARG, "give both lhat and uhat or neither");
    if (opt) c->opt = *opt;
    else as_default_options(&c->opt);
    TRY(validate_opt(c, c->opt));
    TRY(validate_net(c, net));
    if (!C && c->n_out != 1) return fail(c, AS_ERR_ARG, "C is null but the last layer has %d outputs", c->n_out);
    const int n = net->n_layers;
    DNet& D = c->net;
    D.n = n;
    D.S = S;
    D.ball = c->opt.input_l2;
    D.cap = std::max(1, c->opt.max_cuts);
    D.RS = ((1 + D.cap) + 3) / 4 * 4;
    int NT = 0;
    std::vector<int> off(n);
    for (int m = 0; m < n; ++m) {
        off[m] = NT;
        NT += c->widths[m];
    }
    D.NT = NT;
    D.NH = NT - c->widths[0];
    std::vector<std::vector<float>> Wh(n);
    // weights
    for (int k = 0; k < n; ++k) {
        const as_layer& A = c->layers[k];
        DLayer& L = D.L[k];
        L.kind = A.kind;
        if (A.kind == AS_LAYER_LINEAR) {
            L.n_in = A.in_c;
            L.n_out = A.out_c;
            L.ci = A.in_c; L.hi = 1; L.wi = 1; L.co = A.out_c; L.ho = 1; L.wo = 1;
            L.kh = L.kw = L.st = 1; L.pd = 0;
        } else {
            L.ci = A.in_c; L.hi = A.in_h; L.wi = A.in_w; L.co = A.out_c; L.ho = A.out_h; L.wo = A.out_w;
            L.kh = A.kh; L.kw = A.kw; L.st = A.stride; L.pd = A.pad;
            L.n_in = L.ci * L.hi * L.wi;
            L.n_out = L.co * L.ho * L.wo;
        }
        const size_t wcount = A.kind == AS_LAYER_LINEAR ? (size_t)L.n_out * L.n_in
                                                         : (size_t)L.co * L.ci * L.kh * L.kw;
        const int bcount = A.kind == AS_LAYER_LINEAR ? L.n_out : L.co;
        float *W, *b;
        TRY(dalloc(c, &W, wcount));
        CUDA_TRY(c, cudaMemcpyAsync(W, A.W, wcount * sizeof(float), cudaMemcpyDefault, c->stream));
        Wh[k].resize(wcount);
        CUDA_TRY(c, cudaMemcpyAsync(Wh[k].data(), A.W, wcount * sizeof(float), cudaMemcpyDefault, c->stream));
        std::vector<float> hb(bcount), hbe(L.n_out);
        CUDA_TRY(c, cudaMemcpyAsync(hb.data(), A.b, bcount * sizeof(float), cudaMemcpyDefault, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        const int per = L.n_out / bcount;
        for (int i = 0; i < L.n_out; ++i) hbe[i] = hb[i / per];
        TRY(dalloc(c, &b, L.n_out));
        CUDA_TRY(c, cudaMemcpyAsync(b, hbe.data(), L.n_out * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        L.W = W;
        L.b = b;
        L.in_off = off[k];
        L.out_off = k + 1 < n ? off[k + 1] : -1;
        L.h_in = k >= 1 ? off[k] - c->widths[0] : -1;
        L.h_out = k + 1 < n ? off[k + 1] - c->widths[0] : -1;
        if (k == n - 1) {
            c->Wlast = W;
            c->blast = b;
        }
    }
    TRY(build_walks(c, Wh));
    // launch geometry
    {
        std::vector<int> ids;
        std::vector<long long> units;
        for (int k = 0; k < n; ++k) {
            ids.push_back(k);
            units.push_back((long long)S * D.L[k].n_in);
        }
        make_segs(c->segA, c->blocksA, ids, units, CB_THREADS);
        ids.clear();
        units.clear();
        for (int k = 0; k < n - 1; ++k) {
            ids.push_back(k);
            units.push_back((long long)S * D.L[k].n_out);
        }
        make_segs(c->segB, c->blocksB, ids, units, CB_WARPS);
    }
    TRY(make_team_segs(c));
    TRY(alloc_state(c));
    TRY(build_tables(c));
    if (c->opt.precision == 16) TRY(build_bf16(c, Wh));
    TRY(load_batch(c, x_lo, x_hi, C, lhat, uhat, splits, caps, true));
    if (c->opt.autotune && c->opt.precision == 32) {
        TRY(autotune_teams(c));
        TRY(load_batch(c, x_lo, x_hi, C, lhat, uhat, splits, caps, false));   // back to zero duals
    }
    if (c->opt.autotune && c->opt.precision == 16) {
        TRY(autotune_tc(c));
        TRY(load_batch(c, x_lo, x_hi, C, lhat, uhat, splits, caps, false));   // clean planes
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return AS_OK;
}

extern "C" int as_init(as_ctx** out, const as_net* net, int S, const float* x_lo, const float* x_hi, const float* C,
                       const float* lhat, const float* uhat, const signed char* splits, const int* caps,
                       const as_options* opt, void* stream) {
    if (!out) return AS_ERR_ARG;
    *out = nullptr;
    as_ctx* c = new (std::nothrow) as_ctx();
    if (!c) return AS_ERR_OOM;
    c->stream = (cudaStream_t)stream;
    if (const char* f = getenv("CB_FAIL_ALLOC_AT")) c->fail_alloc_at = atoll(f);
    if (const char* f = getenv("CB_TC_STAGE_WAIT_LIMIT")) c->tc_stage_limit = (uint32_t)strtoul(f, nullptr, 10);
    if (const char* f = getenv("CB_TC_WINDOWS")) c->tc_windows = atoi(f) != 0;
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return AS_ERR_CUDA;
    }
    int r = init_impl(c, net, S, x_lo, x_hi, C, lhat, uhat, splits, caps, opt);
    *out = c;  // returned even on failure so that as_last_error can explain; caller destroys it
    return r;
}

extern "C" void as_destroy(as_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->g_as) cudaGraphExecDestroy(c->g_as);
    if (c->g_sp) cudaGraphExecDestroy(c->g_sp);
    for (void* p : c->allocs) cudaFree(p);
    for (auto& r : c->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

// ------------------------------------------------------------------------------- iterations
static int launch_as_iter(as_ctx* c, cudaStream_t s) {
    // the per-neuron bound terms are only summed when the best bound is tracked
    const int mode = c->opt.track_best ? 0 : 2;
    LAUNCH(c, s, CB_K_AS_COLA, (k_as_colA_t<false><<<c->blocksTA, CB_THREADS, 0, s>>>(c->net, c->st, c->sc, c->tA, mode)));
    if (c->net.ball) LAUNCH(c, s, CB_K_BALL_X0, (k_ball_x0<<<c->net.S, CB_BALL_THREADS, 0, s>>>(c->net, c->st)));
    if (c->opt.track_best)
        LAUNCH(c, s, CB_K_REDUCE, (k_reduce<<<c->net.S, CB_THREADS, 0, s>>>(c->net, c->st, 64, nullptr, 1)));
    LAUNCH(c, s, CB_K_AS_ROWB, (k_as_rowB_t<false><<<c->blocksTB, CB_THREADS, 0, s>>>(c->net, c->st, c->sc, c->tB)));
    LAUNCH(c, s, CB_K_COUNTER, (k_advance<<<1, 1, 0, s>>>(c->st.ctr, 0)));
    return check_launch(c, "Active Set iteration");
}

// One Saddle Point iteration t: phase B, then phase C fused with phase A of iteration t + 1 (the
// loop's first phase A runs before it, k_sp_colA_t, whenever the state is new).
static int launch_sp_iter(as_ctx* c, cudaStream_t s) {
    LAUNCH(c, s, CB_K_SP_ROWB, (k_sp_rowB_t<<<c->blocksTB, CB_THREADS, 0, s>>>(c->net, c->st, c->sc, c->tB)));
    LAUNCH(c, s, CB_K_SP_COLC, (k_sp_colCA_t<<<c->blocksTA, CB_THREADS, 0, s>>>(c->net, c->st, c->sc, c->tA)));
    LAUNCH(c, s, CB_K_COUNTER, (k_advance<<<1, 1, 0, s>>>(c->st.ctr, 1)));
    if (c->net.ball) LAUNCH(c, s, CB_K_BALL_X0, (k_ball_sp<<<c->net.S, CB_BALL_THREADS, 0, s>>>(c->net, c->st, 0)));
    if (c->opt.track_best)
        LAUNCH(c, s, CB_K_REDUCE, (k_reduce<<<c->net.S, CB_THREADS, 0, s>>>(c->net, c->st, 64, nullptr, 1)));
    return check_launch(c, "Saddle Point iteration");
}

extern "C" int as_kernel_times(as_ctx* c, int kernel, double* total_ms, long long* launches) {
    if (!c || kernel < 0 || kernel >= CB_NPROF) return AS_ERR_ARG;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (auto& r : c->pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return fail(c, AS_ERR_CUDA, "event timing failed: %s", cudaGetErrorString(e));
        c->prof_ms[r.id] += ms;
        c->prof_n[r.id] += 1;
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->pending.clear();
    if (total_ms) *total_ms = c->prof_ms[kernel];
    if (launches) *launches = c->prof_n[kernel];
    return AS_OK;
}

#include "cb_bf16.inc"

typedef int (*iter_fn)(as_ctx*, cudaStream_t);

static int run_iters(as_ctx* c, int n_iters, iter_fn fn, cudaGraphExec_t* gexec, int* glen, int* gnodes) {
    const int G = c->opt.profile ? 0 : c->opt.graph_chunk;
    int done = 0;
    if (G > 1 && n_iters >= G) {
        if (!*gexec) {
            const long long before = c->launches;
            CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            int r = AS_OK;
            for (int q = 0; q < G && r == AS_OK; ++q) r = fn(c, c->cap_stream);
            cudaGraph_t g;
            cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
            if (r != AS_OK) return r;
            if (e != cudaSuccess) return fail(c, AS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(c, AS_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
            *glen = G;
            *gnodes = (int)(c->launches - before);
            c->launches = before;  // captured, not executed
        }
        for (; done + *glen <= n_iters; done += *glen) {
            CUDA_TRY(c, cudaGraphLaunch(*gexec, c->stream));
            c->launches += *gnodes;
        }
    }
    for (; done < n_iters; ++done) TRY(fn(c, c->stream));
    return AS_OK;
}

extern "C" int as_step(as_ctx* c, int n_iters) {
    if (!c) return AS_ERR_ARG;
    if (n_iters < 0) return fail(c, AS_ERR_ARG, "n_iters < 0");
    if (c->sp_started) return fail(c, AS_ERR_STATE, "Saddle Point has started on this context");
    return run_iters(c, n_iters, c->opt.precision == 16 ? launch_as_iter_bf16 : launch_as_iter, &c->g_as,
                     &c->g_as_len, &c->g_as_nodes);
}

static int sp_start(as_ctx* c) {
    cudaStream_t s = c->stream;
    if (c->opt.precision == 16) TRY(recompute_slot_sums(c));   // float32 lambda, kappa for the conversion
    const size_t NHS = (size_t)c->net.S * c->net.NH;
    LAUNCH(c, s, CB_K_SP_START, (k_sp_convert_elem<<<grid_for(NHS), CB_THREADS, 0, s>>>(c->net, c->st, c->sc,
                                                                                      (float)c->opt.sp_c_alpha,
                                                                                      (float)c->opt.sp_c_beta)));
    LAUNCH(c, s, CB_K_SP_START, (k_sp_convert_P_t<<<c->blocksTA, CB_THREADS, 0, s>>>(c->net, c->st, c->sc, c->tA)));
    LAUNCH(c, s, CB_K_SP_START, (k_sp_prep<<<grid_for(NHS), CB_THREADS, 0, s>>>(c->net, c->st)));
    LAUNCH(c, s, CB_K_SP_START, (k_sp_colA_t<<<c->blocksTA, CB_THREADS, 0, s>>>(c->net, c->st, c->tA, 1)));
    if (c->net.ball) LAUNCH(c, s, CB_K_BALL_X0, (k_ball_sp<<<c->net.S, CB_BALL_THREADS, 0, s>>>(c->net, c->st, 1)));
    TRY(check_launch(c, "Saddle Point conversion"));
    for (int t = 0; t < c->opt.sp_init_steps; ++t) {
        LAUNCH(c, s, CB_K_SPI_ROW, (k_spi_row_t<<<c->blocksTB, CB_THREADS, 0, s>>>(c->net, c->st, c->tB)));
        LAUNCH(c, s, CB_K_SPI_COL, (k_spi_col_t<<<c->blocksTA, CB_THREADS, 0, s>>>(c->net, c->st, c->sc, c->tA)));
        LAUNCH(c, s, CB_K_COUNTER, (k_advance<<<1, 1, 0, s>>>(c->st.ctr, 2)));
        if (c->net.ball)
            LAUNCH(c, s, CB_K_BALL_X0, (k_ball_retract<<<c->net.S, CB_BALL_THREADS, 0, s>>>(c->net, c->st)));
    }
    TRY(check_launch(c, "Saddle Point primal initialisation"));
    c->sp_started = true;
    c->sp_need_phaseA = true;
    return AS_OK;
}

extern "C" int sp_step(as_ctx* c, int n_iters) {
    if (!c) return AS_ERR_ARG;
    if (n_iters < 0) return fail(c, AS_ERR_ARG, "n_iters < 0");
    if (!c->sp_started) TRY(sp_start(c));
    if (n_iters == 0) return AS_OK;
    if (c->sp_need_phaseA) {
        cudaStream_t s = c->stream;
        LAUNCH(c, s, CB_K_SP_COLA, (k_sp_colA_t<<<c->blocksTA, CB_THREADS, 0, s>>>(c->net, c->st, c->tA, 0)));
        if (c->net.ball) LAUNCH(c, s, CB_K_BALL_X0, (k_ball_sp<<<c->net.S, CB_BALL_THREADS, 0, s>>>(c->net, c->st, 0)));
        TRY(check_launch(c, "Saddle Point phase A"));
        c->sp_need_phaseA = false;
    }
    return run_iters(c, n_iters, launch_sp_iter, &c->g_sp, &c->g_sp_len, &c->g_sp_nodes);
}

extern "C" int as_bound(as_ctx* c, int precision, double* out, double* best) {
    if (!c) return AS_ERR_ARG;
    if (precision != 32 && precision != 64) return fail(c, AS_ERR_ARG, "precision must be 32 or 64");
    const int S = c->net.S;
    cudaStream_t s = c->stream;
    if (c->sp_started) {
        LAUNCH(c, s, CB_K_SP_COLA, (k_sp_colA_t<<<c->blocksTA, CB_THREADS, 0, s>>>(c->net, c->st, c->tA, 0)));
        if (c->net.ball) LAUNCH(c, s, CB_K_BALL_X0, (k_ball_sp<<<S, CB_BALL_THREADS, 0, s>>>(c->net, c->st, 0)));
    } else {
        // the BF16 form's iterates give a bound through float32 lambda, kappa and records
        if (c->opt.precision == 16) TRY(recompute_slot_sums(c));
        LAUNCH(c, s, CB_K_AS_COLA, (k_as_colA_t<false><<<c->blocksTA, CB_THREADS, 0, s>>>(c->net, c->st, c->sc, c->tA, 1)));
        if (c->net.ball) LAUNCH(c, s, CB_K_BALL_X0, (k_ball_x0<<<S, CB_BALL_THREADS, 0, s>>>(c->net, c->st)));
    }
    double* dout = c->bound_out;
    LAUNCH(c, s, CB_K_REDUCE, (k_reduce<<<S, CB_THREADS, 0, s>>>(c->net, c->st, precision, dout, 1)));
    TRY(check_launch(c, "bound evaluation"));
    std::vector<double> h(S);
    int status = 0;
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), dout, S * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaMemcpyAsync(&status, c->st.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (out) CUDA_TRY(c, cudaMemcpyAsync(out, dout, S * sizeof(double), cudaMemcpyDefault, s));
    if (best) CUDA_TRY(c, cudaMemcpyAsync(best, c->st.best, S * sizeof(double), cudaMemcpyDefault, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (status) return fail(c, AS_ERR_ARG, "the batch's input box has lo > hi or a non-finite entry");
    if (c->tc_status) {
        int ts = 0;
        CUDA_TRY(c, cudaMemcpy(&ts, c->tc_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (ts) return fail(c, AS_ERR_TIMEOUT, "a tensor-core kernel's bounded wait ran out");
    }
    for (int q = 0; q < S; ++q)
        if (!std::isfinite(h[q])) return fail(c, AS_ERR_NUMERIC, "bound of subproblem %d is %g", q, h[q]);
    return AS_OK;
}

// ------------------------------------------------------------------------------ state access
struct StateBuf {
    void* p;
    size_t bytes;
};

static StateBuf state_buf(as_ctx* c, int which, int part = 0) {
    const size_t S = c->net.S, NT = c->net.NT, NH = c->net.NH, cap = c->net.cap;
    DState& st = c->st;
    const int bo = 0;
    (void)bo;
    switch (which) {
        case AS_ST_ALPHA: return {st.alpha, S * NH * 4};
        case AS_ST_BETA0: return {st.beta0, S * NH * 4};
        case AS_ST_BETA1: return {st.beta1, S * NH * 4};
        case AS_ST_SLOT_BETA: return {st.bs, S * cap * NH * 4};
        case AS_ST_LHAT: return {st.lhat, S * NH * 4};
        case AS_ST_UHAT: return {st.uhat, S * NH * 4};
        case AS_ST_XSTAR: return {st.xval, S * NT * 4};
        case AS_ST_ZSTAR: return {st.zcur, S * NH};
        case AS_ST_LAMBDA: return {st.lam, S * cap * NH * 4};
        case AS_ST_KAPPA: return {st.kap, S * cap * NH * 4};
        case AS_ST_LO: return {st.lo, S * NT * 4};
        case AS_ST_SP_SEL: return {st.sel, S * NH};
        case AS_ST_HI: return {st.hi, S * NT * 4};
        default: return {nullptr, 0};
    }
}

static int snap_parity(as_ctx* c, int* par) {
    int it = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&it, c->st.ctr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int nadd = 0;
    if (it >= c->sc.TM) nadd = cb_additions_before(it - c->sc.TM, c->sc);
    *par = nadd & 1;
    return AS_OK;
}

extern "C" int as_state_size(as_ctx* c, int which, long long* nbytes) {
    if (!c || !nbytes) return AS_ERR_ARG;
    const size_t S = c->net.S, NT = c->net.NT, NH = c->net.NH, cap = c->net.cap;
    size_t b;
    switch (which) {
        case AS_ST_XSNAP: b = S * NT; break;
        case AS_ST_ZSNAP: b = S * NH; break;
        case AS_ST_ITER: b = 3 * sizeof(int); break;
        case AS_ST_ADAM: b = 6 * S * NH * 4; break;
        case AS_ST_SLOT_ADAM: b = 2 * S * cap * NH * 4; break;
        case AS_ST_SP_X: b = S * NT * 4; break;
        case AS_ST_SP_Z: b = S * NH * 4; break;
        case AS_ST_SP_STATS: b = 4 * S * NT * 4; break;
        case AS_ST_SP_CAPS: b = 2 * S * NH * 4; break;
        default: {
            StateBuf sb = state_buf(c, which);
            if (!sb.p) return fail(c, AS_ERR_ARG, "unknown state buffer %d", which);
            b = sb.bytes;
        }
    }
    *nbytes = (long long)b;
    return AS_OK;
}

static int copy_pieces(as_ctx* c, void* dst, const void* src, bool out, std::vector<StateBuf> parts) {
    size_t o = 0;
    for (auto& p : parts) {
        if (out) CUDA_TRY(c, cudaMemcpyAsync((char*)dst + o, p.p, p.bytes, cudaMemcpyDefault, c->stream));
        else CUDA_TRY(c, cudaMemcpyAsync(p.p, (const char*)src + o, p.bytes, cudaMemcpyDefault, c->stream));
        o += p.bytes;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return AS_OK;
}

static std::vector<StateBuf> composite(as_ctx* c, int which, int par) {
    const size_t S = c->net.S, NT = c->net.NT, NH = c->net.NH, cap = c->net.cap;
    DState& st = c->st;
    int cur = 0;
    switch (which) {
        case AS_ST_XSNAP: return {{st.xsnap[par], S * NT}};
        case AS_ST_ZSNAP: return {{st.zsnap[par], S * NH}};
        case AS_ST_ITER: return {{st.ctr, 3 * sizeof(int)}};
        case AS_ST_ADAM:
            return {{st.ma, S * NH * 4}, {st.va, S * NH * 4}, {st.m0, S * NH * 4},
                    {st.v0, S * NH * 4}, {st.m1, S * NH * 4}, {st.v1, S * NH * 4}};
        case AS_ST_SLOT_ADAM: return {{st.ms, S * cap * NH * 4}, {st.vs, S * cap * NH * 4}};
        case AS_ST_SP_X: cur = par; return {{st.spx[cur], S * NT * 4}};
        case AS_ST_SP_Z: cur = par; return {{st.spz[cur], S * NH * 4}};
        case AS_ST_SP_CAPS: return {{st.mua, S * NH * 4}, {st.mub, S * NH * 4}};
        default: {
            StateBuf sb = state_buf(c, which);
            return {sb};
        }
    }
}

static int sp_parity(as_ctx* c, int* par) {
    int t = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&t, c->st.ctr + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *par = t & 1;
    return AS_OK;
}

extern "C" int as_get_state(as_ctx* c, int which, void* dst) {
    if (!c || !dst) return AS_ERR_ARG;
    if (which < 0 || which >= AS_ST_COUNT) return fail(c, AS_ERR_ARG, "unknown state buffer %d", which);
    int par = 0;
    if (which == AS_ST_XSNAP || which == AS_ST_ZSNAP) TRY(snap_parity(c, &par));
    if (which == AS_ST_SP_X || which == AS_ST_SP_Z) TRY(sp_parity(c, &par));
    if (which == AS_ST_ITER) {
        int v[3];
        CUDA_TRY(c, cudaMemcpyAsync(v, c->st.ctr, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        v[2] = c->sp_started ? 1 : 0;
        CUDA_TRY(c, cudaMemcpy(dst, v, sizeof v, cudaMemcpyDefault));
        return AS_OK;
    }
    if (which == AS_ST_SP_STATS) {
        const size_t S = c->net.S, NT = c->net.NT, NH = c->net.NH;
        // [4][S][NT]: Sb, G, C placed at the hidden part of each row, P as is
        std::vector<float> h(4 * S * NT, 0.f), t(S * NH);
        float* src[3] = {c->st.Sb, c->st.G, c->st.C};
        for (int q = 0; q < 3; ++q) {
            CUDA_TRY(c, cudaMemcpyAsync(t.data(), src[q], S * NH * 4, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            for (size_t s = 0; s < S; ++s)
                std::memcpy(&h[(q * S + s) * NT + (NT - NH)], &t[s * NH], NH * 4);
        }
        CUDA_TRY(c, cudaMemcpyAsync(&h[3 * S * NT], c->st.P, S * NT * 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        CUDA_TRY(c, cudaMemcpy(dst, h.data(), h.size() * 4, cudaMemcpyDefault));
        return AS_OK;
    }
    return copy_pieces(c, dst, nullptr, true, composite(c, which, par));
}

static int recompute_slot_sums(as_ctx* c);

extern "C" int as_set_state(as_ctx* c, int which, const void* src) {
    if (!c || !src) return AS_ERR_ARG;
    c->sp_need_phaseA = true;
    if (which < 0 || which >= AS_ST_COUNT) return fail(c, AS_ERR_ARG, "unknown state buffer %d", which);
    if (which == AS_ST_XSTAR || which == AS_ST_ZSTAR || which == AS_ST_LAMBDA || which == AS_ST_KAPPA ||
        which == AS_ST_LO || which == AS_ST_HI || which == AS_ST_LHAT || which == AS_ST_UHAT ||
        which == AS_ST_SP_SEL)
        return fail(c, AS_ERR_ARG, "state buffer %d is read-only", which);
    if (which == AS_ST_ITER) {
        int v[3];
        CUDA_TRY(c, cudaMemcpy(v, src, sizeof v, cudaMemcpyDefault));
        if (v[0] < 0 || v[1] < 0) return fail(c, AS_ERR_ARG, "negative iteration counter");
        int w[3] = {v[0], v[1], v[2] ? c->opt.sp_init_steps : 0};
        CUDA_TRY(c, cudaMemcpyAsync(c->st.ctr, w, sizeof w, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        c->sp_started = v[2] != 0;
        return recompute_slot_sums(c);
    }
    if (which == AS_ST_SP_STATS) {
        const size_t S = c->net.S, NT = c->net.NT, NH = c->net.NH;
        std::vector<float> h(4 * S * NT), t(S * NH);
        CUDA_TRY(c, cudaMemcpy(h.data(), src, h.size() * 4, cudaMemcpyDefault));
        float* dst3[3] = {c->st.Sb, c->st.G, c->st.C};
        for (int q = 0; q < 3; ++q) {
            for (size_t s = 0; s < S; ++s) std::memcpy(&t[s * NH], &h[(q * S + s) * NT + (NT - NH)], NH * 4);
            CUDA_TRY(c, cudaMemcpyAsync(dst3[q], t.data(), S * NH * 4, cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        }
        CUDA_TRY(c, cudaMemcpyAsync(c->st.P, &h[3 * S * NT], S * NT * 4, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        return AS_OK;
    }
    int par = 0;
    if (which == AS_ST_XSNAP || which == AS_ST_ZSNAP) TRY(snap_parity(c, &par));
    if (which == AS_ST_SP_X || which == AS_ST_SP_Z) TRY(sp_parity(c, &par));
    TRY(copy_pieces(c, nullptr, src, false, composite(c, which, par)));
    if (which == AS_ST_SLOT_BETA || which == AS_ST_XSNAP || which == AS_ST_ZSNAP || which == AS_ST_ALPHA ||
        which == AS_ST_BETA1)
        TRY(recompute_slot_sums(c));
    return AS_OK;
}

#include "cb_host_extra.inc"

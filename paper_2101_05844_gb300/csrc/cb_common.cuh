// Device-side descriptors shared by the kernels and the host API of the convex-barrier library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define CB_MAXL 10
#define CB_MAXCUT 8
#define CB_THREADS 256
#define CB_WARPS (CB_THREADS / 32)

// Kernel ids for per-kernel timing (as_kernel_times).
enum { CB_K_AS_COLA = 0, CB_K_AS_ROWB, CB_K_REDUCE, CB_K_SP_COLA, CB_K_SP_ROWB, CB_K_SP_COLC,
       CB_K_SPI_ROW, CB_K_SPI_COL, CB_K_TC_COL, CB_K_TC_ROW, CB_K_SLOT_SUMS, CB_K_BALL_X0,
       CB_K_BATCH, CB_K_SP_START, CB_K_COUNTER, CB_NPROF };

// One affine layer k (1-based in the paper; stored at index k-1).
struct DLayer {
    int kind;              // 0 linear, 1 conv2d
    int n_in, n_out;
    int ci, hi, wi, co, ho, wo, kh, kw, st, pd;
    const float* W;        // linear [n_out][n_in], conv [co][ci][kh][kw]
    const float* b;        // per output neuron [n_out]
    int in_off, out_off;   // offsets of the input / output neuron layer in [NT] vectors
    int h_in, h_out;       // offsets in [NH] hidden vectors (-1 when not a hidden layer)
    // Active Set walks (hidden-output layers). Tap lists {offset in floats, weight bits} per group,
    // the group's positive weights first: taps [grp[2g], grp[2g+1]) have W > 0 and
    // [grp[2g+1], grp[2g+2]) have W < 0 (zero weights are left out).
    //  row pass: group = output row (linear) or output channel (conv); offsets index the input
    //            records of this layer in positions (zero-padded input plane for conv)
    //  col pass: group = input (linear) or (input channel, stride phase y, stride phase x) (conv);
    //            offsets index the output records in positions (output plane with a zero halo
    //            for conv)
    const int2* rtap;
    const int* rgrp;
    const int2* ctap;
    const int* cgrp;
    int xo, ao;            // offsets (floats) of this layer's input / output records in a subproblem
    int xpos, apos;        // input / output record positions (padded planes for conv)
    int Hp, Wp;            // padded input plane (conv): in + 2 pad
    int Hpo, Wpo, hl, wl;  // output plane with halo (conv): rows hl .. hl + ho - 1 are the outputs
};

#define CB_MAXPH 9   // stride phases of a conv layer in the BF16 form (stride <= 3)

// BF16 form of the Active Set passes, per hidden-output layer: the tensor-core operands
// (channels-last planes, channels padded to a multiple of 8, zero padding and halo) and products.
// Slot 0 carries the unmasked operand (x*, resp. rp), slot 1 + b the operand of active-set slot b.
struct BfLayer {
    int Cip, Cop;             // input / output channels rounded up to 8
    long long PX, PR;         // elements of an input plane [Hp][Wp][Cip], of an output plane [Hpo][Wpo][Cop]
    uint16_t* X;              // [1 + cap][S][2][Hp][Wp][Cip] bf16: x* (slot 0), x* p_b (sign 0) and x* q_b (sign 1)
    uint16_t* R;              // [1 + cap][S][Hpo][Wpo][Cop] bf16: rp (slot 0), bz_b
    float* Drow;              // [(1 + cap) S][co][Ho Wo]: W x* (slot 0) and (W o I_b) x* per output neuron
    int nph;                  // stride phases (stride^2); input j = (c, y, x) is in phase (y + pad) % st, (x + pad) % st
    float* Dcol[CB_MAXPH];    // per phase [(1 + cap) S][2 ci][nY nX]: W+^T and W-^T products per input
    int Y0a[CB_MAXPH], X0a[CB_MAXPH], nY[CB_MAXPH], nX[CB_MAXPH];   // (y + pad) / st spans nY values from Y0a
};

struct DNet {
    int n;                 // affine layers; hidden layers k = 1..n-1
    int S, NT, NH, cap;    // subproblems, all neurons (layers 0..n-1), hidden neurons, max slots
    int RS;                // floats per Active Set record chunk (1 + cap rounded up to 4)
    int XT, AT;            // floats of input / output records per subproblem (all layers)
    DLayer L[CB_MAXL];
    const float* Wout;     // [S][n_{n-1}] property-folded output row
    const float* bout;     // [S]
    const BfLayer* bf;     // [n - 1] device array, BF16 form only (else null)
    int ball;              // 1: the input set is the ellipsoid inscribed in the box (l2 ball for equal
                           // half-widths); 0: the box
};

// Solver schedule constants (float32 copies prepared on the host from the double options).
struct DSched {
    int TM, TA, omega, vpa, maxcut;
    int ntab;              // entries in the per-step tables
    float b1, omb1, b2, omb2, eps;
    float lr_as_end;       // step size after the planned iterations
    float gamma0;
    int sp_init_steps;
    float sp_lr0, sp_lr1;
};

// Device state. Per-subproblem arrays are [S][NT], [S][NH] or [S][cap][NH].
struct DState {
    float *lo, *hi;                  // post-activation bounds, layer 0 = input box
    float *lhat, *uhat;              // pre-activation bounds (hidden)
    float *alpha, *beta0, *beta1;
    float *ma, *va, *m0, *v0, *m1, *v1;
    float *bs, *ms, *vs, *lam, *kap; // slots
    float *arec;                     // [S][AT] output records of each layer, RS floats per position
                                     // stored as RS / 4 planes of float4 over the positions:
                                     // -(alpha - beta1) + sum_b z_b beta_b, then (1 - z_b) beta_b
    float *xin;                      // [S][XT] input records of each layer, one float2 per position:
                                     // {x*, p_b bits | q_b bits << 8}
    float *lz;                       // [S][NH] sum_j W_ij Lcheck_ij (the all-ones mask's lambda)
    float *brad;                     // [S][NH] ellipsoid inputs: |W_i o e|_2 of layer 1's rows
    double *bnrm;                    // [S] ellipsoid inputs: |e o f_0|_2 of the last x_0* evaluation
    float *uz;                       // [S][NH] sum_j W_ij Ucheck_ij (kappa - b of a z = 0 row whose
                                     // inputs are all interior: the mask is then empty but for
                                     // fixed inputs, where Lcheck = Ucheck)
    uint8_t* efix;                   // [S][NT] l == u
    float *xval;                     // x* of the last evaluation [S][NT]
    float *fval;                     // f of the last evaluation [S][NT]
    uint8_t* zcur;                   // z* of the last evaluation [S][NH]
    uint8_t* xsnap[2];               // [S][NT] slot bitsets (double-buffered by addition count)
    uint8_t* zsnap[2];               // [S][NH]
    double* terms;                   // per-neuron bound terms [S][NT]
    double* best;                    // [S]
    const int* caps;                 // [S]
    int* ctr;                        // [0] AS iteration, [1] SP iteration, [2] SP-init step
    const float* lr_tab;             // [ntab] step size per global iteration
    const float* bc1_tab;            // [ntab] 1 / (1 - b1^step), step = index
    const float* bc2_tab;            // [ntab] 1 / (1 - b2^step)
    // Saddle Point
    float* spx[2];                   // [S][NT]
    float* spz[2];                   // [S][NH]
    float *Sb, *G, *C;               // [S][NH]
    float* P;                        // [S][NT], P_k at the inputs of layer k
    float *mua, *mub;                // [S][NH]
    float* xbar;                     // [S][NT]
    uint8_t* zbar;                   // [S][NH]
    float4* spin;                    // [S][XT] Saddle Point input records: two float4 planes per layer
    int* nfree;                      // [S][NH] nonzero weights of each row on free inputs
    uint8_t* sel;                    // [S][NH] selected beta of the conditional gradient (3 = none)
    float *ab, *b0i, *b1i;           // [S][NH] primal-init inner maximisers
    float* arow;                     // [S][NH] ab - b1i (primal-init row values for the col pass)
    int* status;                     // device error word
};

// Iteration schedule of the Big-M / Active Set loop at global iteration it.
struct Step {
    int as_phase;       // 0 Big-M, 1 Active Set
    int t;              // Active Set local iteration (-1 in Big-M)
    int b_new;          // slot added at this iteration (-1: none)
    int nadd_before;    // slots added before this iteration (global, before per-subproblem caps)
    float lr;
};

__host__ __device__ inline int cb_additions_before(int t, const DSched& d) {
    if (t <= 0) return 0;
    int c;
    if (d.omega > 0) {
        int full = t / d.omega, rem = t % d.omega;
        c = full * d.vpa + (rem < d.vpa ? rem : d.vpa);
    } else {
        c = t < d.vpa ? t : d.vpa;
    }
    return c < d.maxcut ? c : d.maxcut;
}

__host__ __device__ inline int cb_slot_at(int t, const DSched& d) {
    int q, r;
    if (d.omega > 0) { q = t / d.omega; r = t % d.omega; }
    else { q = 0; r = t; }
    if (r >= d.vpa) return -1;
    int b = q * d.vpa + r;
    return b < d.maxcut ? b : -1;
}

// Active Set iteration at which slot b is added.
__host__ __device__ inline int cb_slot_added_at(int b, const DSched& d) {
    return d.omega > 0 ? (b / d.vpa) * d.omega + (b % d.vpa) : b;
}

__device__ inline Step cb_step(int it, const DSched& d, const float* lr_tab) {
    Step s;
    s.lr = it < d.ntab ? lr_tab[it] : d.lr_as_end;
    if (it < d.TM) {
        s.as_phase = 0; s.t = -1; s.b_new = -1; s.nadd_before = 0;
    } else {
        s.as_phase = 1; s.t = it - d.TM;
        s.b_new = cb_slot_at(s.t, d);
        s.nadd_before = cb_additions_before(s.t, d);
    }
    return s;
}

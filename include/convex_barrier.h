/*
 * convex_barrier.h - C ABI of the GB300 (sm_103a) library for the sparse dual solvers of
 * De Palma et al., "Scaling the Convex Barrier with Sparse Dual Algorithms" (arXiv 2101.05844).
 *
 * The library bounds min over x_0 in a box of  c_s^T (W_n x_{n-1} + b_n)  for S subproblems at
 * once, through affine layers and ReLUs (problem 1, Sec. 2), using the tighter relaxation of
 * Sec. 2.2 (problem 4). Solvers: Big-M (Alg. 3, App. B), Active Set (Alg. 1, Sec. 4) and Saddle
 * Point (Alg. 2, Sec. 5). All arithmetic runs in CUDA kernels on the current device.
 *
 * Conventions
 *  - Pointers marked "host or device" may point to either; the library copies from them with
 *    unified addressing before the call returns and never keeps them. Outputs marked "host or
 *    device" are written before the call returns (the call synchronises its stream when an output
 *    is in host memory).
 *  - Every function returns an int status (AS_OK = 0). No C++ exception crosses the ABI.
 *    as_last_error() gives a message for the last failure of a context.
 *  - Per-subproblem vectors are row-major [S][n]. "Hidden vectors" concatenate the hidden layers
 *    k = 1..n-1 in order: [S][n_1 + ... + n_{n-1}].
 *  - Calls on one context are ordered on its stream; a context is not thread-safe.
 */
#ifndef CONVEX_BARRIER_H
#define CONVEX_BARRIER_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define AS_OK 0
#define AS_ERR_ARG 1      /* bad argument: null pointer, lo > hi, S < 1, bad option         */
#define AS_ERR_SHAPE 2    /* layer shapes inconsistent                                       */
#define AS_ERR_CUDA 3     /* a CUDA call failed (message in as_last_error)                   */
#define AS_ERR_OOM 4      /* device allocation failed                                        */
#define AS_ERR_NUMERIC 5  /* a bound came out NaN or infinite                                */
#define AS_ERR_TIMEOUT 6  /* a bounded device wait expired (tensor-core kernels only)          */
#define AS_ERR_STATE 7    /* call not valid in the context's current mode                    */
#define AS_ERR_SCRATCH 8  /* the problem does not fit the fixed scratch of as_ibp_noalloc      */

#define AS_LAYER_LINEAR 0
#define AS_LAYER_CONV2D 1

#define AS_MAX_LAYERS 10 /* affine layers, output layer included */
#define AS_MAX_CUTS 8    /* active-set masks per neuron (the paper uses at most 7, Sec. 8.1) */

/* One affine layer x_hat_k = W_k x_{k-1} + b_k (Sec. 2). Hidden layers are followed by a ReLU;
 * the last layer is linear and has no ReLU.
 *  LINEAR: in_c = n_{k-1}, out_c = n_k, other shape fields ignored; W row-major [out_c][in_c].
 *  CONV2D: input [in_c][in_h][in_w], output [out_c][out_h][out_w] (CHW, row-major), square
 *          or rectangular kernel kh x kw, stride, zero padding pad; W [out_c][in_c][kh][kw],
 *          b per output channel. out_h, out_w must equal (in + 2 pad - k) / stride + 1.
 *  W and b: host or device, float32; copied by as_init. */
typedef struct as_layer {
    int kind;
    int in_c, in_h, in_w;
    int out_c, out_h, out_w;
    int kh, kw, stride, pad;
    const float* W;
    const float* b;
} as_layer;

typedef struct as_net {
    int n_layers; /* n >= 2 (at least one hidden layer), <= AS_MAX_LAYERS */
    const as_layer* layers;
} as_net;

/* Solver options; as_default_options() fills the paper's values (Sec. 8.1, App. C). */
typedef struct as_options {
    int bigm_iters;      /* T_M: Big-M iterations before Active Set (its initialisation, App. B) */
    int as_iters;        /* T_A: Active Set iterations (sets the learning-rate schedule)      */
    double bigm_lr0, bigm_lr1; /* Big-M step size, linear from lr0 to lr1 (1e-2 -> 1e-4)       */
    double as_lr0, as_lr1;     /* Active Set step size after reset (1e-3 -> 1e-6)              */
    int omega;           /* iterations between mask additions (450); <= 0: only the first     */
    int vars_per_add;    /* masks per addition, one per iteration (2)                         */
    int max_cuts;        /* masks per neuron, <= AS_MAX_CUTS (7)                              */
    double adam_b1, adam_b2, adam_eps; /* Adam (0.9, 0.999, 1e-8)                             */
    double sp_gamma0;    /* Saddle Point step gamma_t = 1 / (t + sp_gamma0) (10)              */
    double sp_c_alpha, sp_c_beta; /* price caps where the initial duals are zero, eq. (16)   */
    int sp_init_steps;   /* primal initialisation steps, App. C.2 (100)                       */
    double sp_init_lr0, sp_init_lr1; /* its step size, linear (1e-2 -> 1e-5)                  */
    int track_best;      /* 1: evaluate the bound at every iteration and keep the best        */
    int graph_chunk;     /* iterations per captured CUDA graph (0: plain launches)           */
    int profile;         /* 1: time every kernel with CUDA events (disables graphs)           */
    int autotune;        /* 1: as_init times, on this context's net and batch, the float32
                          * passes' team-size targets (threads per layer segment, a few
                          * iterations each; see as_team_targets) or, in the BF16 form, each
                          * tensor-core product's plan (window or gathered operands, N tile
                          * width), and keeps the fastest; 0: defaults                       */
    int precision;       /* products of the Big-M / Active Set passes: 32 (float32, default) or
                          * 16 (the BF16 form: W x* and every masked product (W o I_b) x*, W^T and
                          * every masked W^T product run on the tensor cores with bf16 operands
                          * (W, x*, the dual row sums) and float32 accumulation; duals, Adam and
                          * the mask decisions stay float32; lambda, kappa of every slot are
                          * recomputed in float32 after each addition; as_bound re-evaluates the
                          * bound in float32 with float64 summation). Saddle Point runs in
                          * float32 on any context.                                        */
    int input_l2;        /* 1: the input set of each subproblem is the ellipsoid inscribed in its box,
                          * {sum_j ((x_j - c_j) / e_j)^2 <= 1} with c, e the box's centre and half-widths
                          * (an l2 ball of radius e for equal half-widths; Sec. 2 needs only a closed-form
                          * linear minimisation over the input set): layer 1's interval bounds are its exact
                          * range W c + b -+ |W D|_2 and x_0* = c + e^2 f_0 / |e f_0|_2 (Saddle Point: the
                          * same vertex, and its primal initialisation retracts x_0 radially into the
                          * ellipsoid); the BF16 form takes x_0* into its operand planes. The gradients of
                          * as_bound_backward(_ibp) with respect to x_lo, x_hi treat them as giving c and
                          * e (the value -f_0 c - |e f_0| and layer 1's interval above).
                          * 0 (default): the box itself.                                        */
} as_options;

typedef struct as_ctx as_ctx;

/* Fills *opt with the defaults above. */
void as_default_options(as_options* opt);

/* Creates a context for S subproblems (the initialisation of Alg. 1 and Alg. 3).
 *  x_lo, x_hi: [S][n_0] input boxes, host or device; x_lo <= x_hi elementwise (AS_ERR_ARG).
 *  C:          [S][n_out] property rows, host or device; subproblem s bounds C[s] . x_hat_n.
 *              NULL allowed only when n_out == 1 (then C[s] = 1).
 *  lhat, uhat: hidden vectors of pre-activation bounds (App. E), host or device; both NULL
 *              to compute them on the device by interval propagation (App. E, last paragraph),
 *              accumulated in FP64 and rounded outward to float32.
 *  splits:     hidden vector of int8 ReLU splits (+1 active, -1 inactive, 0 free), or NULL. A
 *              split clamps lhat to 0 (+1) or uhat to 0 (-1) of a neuron whose interval straddles
 *              zero before the next layer is propagated; it is ignored with caller bounds.
 *  caps:       [S] masks per neuron for each subproblem (1..max_cuts), or NULL (= max_cuts).
 *  opt:        NULL for defaults.
 *  stream:     cudaStream_t on which every call of this context is enqueued (NULL = legacy).
 * The context starts with every dual at zero, so its bound is the interval bound (App. B.3). */
int as_init(as_ctx** out, const as_net* net, int S, const float* x_lo, const float* x_hi,
            const float* C, const float* lhat, const float* uhat, const signed char* splits,
            const int* caps, const as_options* opt, void* stream);

/* Restarts a context on a new batch of S subproblems of the same network (branch and bound:
 * new boxes, properties, splits; no reallocation, no synchronisation). Arguments as in as_init,
 * all host or device. Every dual, Adam moment, active-set slot and Saddle Point statistic is
 * zeroed and the iteration counters restart. The box is checked on the device: lo > hi or a
 * non-finite entry is reported by the next as_bound (AS_ERR_ARG). */
int as_reset(as_ctx* ctx, const float* x_lo, const float* x_hi, const float* C, const float* lhat,
             const float* uhat, const signed char* splits, const int* caps);

/* Runs n_iters iterations of Big-M (global iteration < bigm_iters) then Active Set (Alg. 1):
 * closed-form inner minimisation (eqs. 7-8), mask addition by the oracle eq. (3) on the schedule
 * of as_options, supergradient (eq. 9), Adam step and projection. Asynchronous on the stream.
 * AS_ERR_STATE after sp_step has started Saddle Point on this context. */
int as_step(as_ctx* ctx, int n_iters);

/* Runs n_iters Saddle Point iterations (Alg. 2). The first call converts the current duals to
 * sufficient statistics (eq. 10), sets the price caps (eq. 16) and runs the primal
 * initialisation (App. C.2). Asynchronous on the stream. */
int sp_step(as_ctx* ctx, int n_iters);

/* Bound at the current duals (Alg. 1 / Alg. 2 return lines): [S] doubles into out (host or
 * device). precision 32 sums the per-neuron terms in float32, 64 in float64 (the terms
 * themselves are float32 products). best (nullable, host or device): best bound over every
 * evaluated iterate, this one included (needs track_best for the per-iteration part).
 * Returns AS_ERR_NUMERIC if any bound is not finite. */
int as_bound(as_ctx* ctx, int precision, double* out, double* best);

/* Gradient of sum_s grad_bound[s] * bound_s at the current duals and masks, with the
 * intermediate bounds and the signs of W held fixed (envelope theorem; not in the paper).
 * grad_bound: [S] host or device. Outputs are ACCUMULATED (+=) into device buffers:
 *  dW[k], db[k] for k = 0..n-1 (layer k+1, shaped like its W and b; the last layer's gradient
 *  is taken through the property rows C), dlo, dhi: [S][n_0]. Any output pointer may be NULL
 *  (dW and db themselves, or entries of them) to skip it. Active Set mode only. */
int as_bound_backward(as_ctx* ctx, const double* grad_bound, float* const* dW, float* const* db,
                      float* dlo, float* dhi);

/* As as_bound_backward, with the intermediate bounds differentiated too: lhat_k, uhat_k follow W,
 * b and the box through the interval propagation that as_init / as_reset computed them by
 * (App. E), post-activation bounds l_k = max(lhat_k, 0), u_k = max(uhat_k, 0), split clamps held
 * as constants. At fixed duals and masks the bound depends on them through the ends of x_k*'s box,
 * Lcheck / Ucheck of the next layer's masks, and the Big-M rows (d/dlhat = beta_1 (1 - z),
 * d/duhat = -beta_0 z); these adjoints run back through W+ and W- layer by layer (the kink of
 * max(., 0) at 0 takes the zero derivative). Not in the paper. AS_ERR_STATE when the batch's
 * bounds were given by the caller. Allocates 8 bytes per neuron per subproblem for the call. */
int as_bound_backward_ibp(as_ctx* ctx, const double* grad_bound, float* const* dW, float* const* db,
                          float* dlo, float* dhi);

/* Named state buffers, for warm starts and inspection. Sizes in bytes via as_state_size. */
#define AS_ST_ALPHA 0     /* float [S][NH]                                                    */
#define AS_ST_BETA0 1     /* float [S][NH]                                                    */
#define AS_ST_BETA1 2     /* float [S][NH]                                                    */
#define AS_ST_SLOT_BETA 3 /* float [S][max_cuts][NH]: beta_{k,I} of each active-set slot      */
#define AS_ST_XSNAP 4     /* uint8 [S][NT]: bit b = x* at its upper bound when slot b was added
                             (NT = n_0 + NH, neuron layers 0..n-1)                             */
#define AS_ST_ZSNAP 5     /* uint8 [S][NH]: bit b = z* when slot b was added                  */
#define AS_ST_ITER 6      /* int [3]: Active Set iteration, Saddle Point iteration, and 1 when
                             Saddle Point has started (setting 1 skips its initialisation)     */
#define AS_ST_LHAT 7      /* float [S][NH] pre-activation lower bounds                        */
#define AS_ST_UHAT 8      /* float [S][NH] pre-activation upper bounds                        */
#define AS_ST_XSTAR 9     /* float [S][NT] primal minimiser x* of the last evaluation         */
#define AS_ST_ZSTAR 10    /* uint8 [S][NH] z* of the last evaluation                          */
#define AS_ST_LAMBDA 11   /* float [S][max_cuts][NH] sum_j W I Lcheck of each slot            */
#define AS_ST_KAPPA 12    /* float [S][max_cuts][NH] lambda + sum_j W (1-I) Ucheck + b        */
#define AS_ST_ADAM 13     /* float [6][S][NH]: m, v of alpha, beta0, beta1                    */
#define AS_ST_SLOT_ADAM 14 /* float [2][S][max_cuts][NH]: m, v of the slots                   */
#define AS_ST_SP_X 15     /* float [S][NT] Saddle Point primal x (current)                    */
#define AS_ST_SP_Z 16     /* float [S][NH] Saddle Point primal z (current)                    */
#define AS_ST_SP_STATS 17 /* float [4][S][NT]: Sb, G, C (hidden part) and P (P_k indexed by
                             the inputs of layer k), see Sec. 5.1                              */
#define AS_ST_SP_CAPS 18  /* float [2][S][NH]: mu_alpha, mu_beta                              */
#define AS_ST_LO 19       /* float [S][NT] post-activation lower bounds (layer 0: the box)    */
#define AS_ST_HI 20       /* float [S][NT] post-activation upper bounds                       */
#define AS_ST_SP_SEL 21   /* uint8 [S][NH] conditional-gradient choice of the last Saddle Point
                             iteration: 0 beta_0, 1 beta_1, 2 the oracle mask, 3 none (eq. 12) */
#define AS_ST_COUNT 22

int as_state_size(as_ctx* ctx, int which, long long* nbytes);
/* Copies a state buffer out (dst host or device); synchronises when dst is host memory. */
int as_get_state(as_ctx* ctx, int which, void* dst);
/* Replaces a state buffer (src host or device). Setting AS_ST_SLOT_BETA, AS_ST_XSNAP or
 * AS_ST_ZSNAP recomputes lambda and kappa of every filled slot. */
int as_set_state(as_ctx* ctx, int which, const void* src);

/* Number of kernel launches this context has issued (graph nodes counted per replay). */
long long as_launch_count(as_ctx* ctx);

/* Kernel ids for as_kernel_times. */
#define AS_K_AS_COLA 0 /* Active Set col pass: f, x*, z*, bound terms, snapshots      */
#define AS_K_AS_ROWB 1 /* Active Set row pass: products, supergradient, Adam          */
#define AS_K_REDUCE 2  /* bound reduction                                              */
#define AS_K_SP_COLA 3 /* Saddle Point col pass: f, primal conditional gradient        */
#define AS_K_SP_ROWB 4 /* Saddle Point row pass: oracle, dual conditional gradient     */
#define AS_K_SP_COLC 5 /* Saddle Point col pass: masked backward and convex combination,
                          fused with the next iteration's phase A                      */
#define AS_K_SPI_ROW 6 /* Saddle Point primal initialisation, row pass                 */
#define AS_K_SPI_COL 7 /* Saddle Point primal initialisation, col pass                 */
#define AS_K_TC_COL 8  /* BF16 form: tensor-core products of the col pass              */
#define AS_K_TC_ROW 9  /* BF16 form: tensor-core products of the row pass              */
#define AS_K_SLOT_SUMS 10 /* BF16 form: float32 lambda, kappa after an addition        */
#define AS_K_BALL_X0 11   /* ellipsoid input set: x_0*, its bound terms and records       */
#define AS_K_BATCH 12     /* a batch's set-up (as_init, as_reset): box checks, property rows,
                             interval bounds, row constants, fixed inputs                   */
#define AS_K_SP_START 13  /* Saddle Point's start: statistics (eq. 10), caps (eq. 16), records */
#define AS_K_COUNTER 14   /* the one-thread launches that advance the iteration counters  */
#define AS_K_COUNT 15

/* With as_options.profile set: total device time (CUDA events on the context's stream) and
 * launch count of one kernel over the context's life so far. Synchronises the stream. */
int as_kernel_times(as_ctx* ctx, int kernel, double* total_ms, long long* launches);

void as_destroy(as_ctx* ctx);
const char* as_last_error(as_ctx* ctx);

/* Allocation-free interval bounds (no counterpart in the paper; a service of this library).
 *
 * Some callers cannot call cudaMalloc: a verifier embedded in a process whose device memory is
 * entirely reserved by another allocator (a deep-learning framework's caching allocator, or the
 * fixed memory pool of a serving engine), where a direct allocation fails or fragments the pool;
 * and latency-critical callers that cannot afford the implicit device synchronisation of
 * cudaMalloc / cudaFree. as_init cannot serve them, since it allocates its context. This entry
 * point computes the pre-activation bounds that as_init derives by interval propagation, with
 * no allocation: the caller passes every input and output, and the post-activation bounds handed
 * from one layer to the next live in a file-scope device array of AS_NOALLOC_SCRATCH_FLOATS
 * floats (16 MiB) that every GPU which loads the library keeps until the process exits.
 *
 *  net:        as for as_init, except that W and b must be device pointers.
 *  x_lo, x_hi: [S][n_0] input boxes, device memory (lo <= hi is the caller's responsibility).
 *  splits:     hidden vector of int8 ReLU splits as for as_init, device memory, or NULL.
 *  lhat, uhat: outputs, hidden vectors [S][n_1 + ... + n_{n-1}] of float, device memory.
 *  stream:     cudaStream_t the kernels are enqueued on; the call does not synchronise.
 * Every pointer must be memory of the current device (or managed memory).
 * Returns AS_ERR_SCRATCH when 4 x S x (widest hidden layer) exceeds AS_NOALLOC_SCRATCH_FLOATS,
 * AS_ERR_ARG for a null or host pointer or memory of another device, AS_ERR_SHAPE for
 * inconsistent layers. Each call looks up the scratch array's device address on the current
 * device (cudaGetSymbolAddress; a device reset therefore leaves no stale address behind); the
 * first call on a device also loads the library's device code there, so make it before any
 * stream capture. Every call on a device shares the one scratch array (nothing in it needs to
 * start at zero: each call writes every entry it reads), so calls whose kernels overlap on the
 * GPU race; issue them on one stream or otherwise order them. */
#define AS_NOALLOC_SCRATCH_FLOATS (1u << 22)
int as_ibp_noalloc(const as_net* net, int S, const float* x_lo, const float* x_hi,
                   const signed char* splits, float* lhat, float* uhat, void* stream);

/* Intermediate bounds by batched dual solves (App. E): the pre-activation bounds of hidden layer
 * k >= 2 are tightened, layer by layer in order, by the Big-M / Active Set bounds (Alg. 1) of
 * min x_hat_k[i] and of min -x_hat_k[i] over the relaxation of layers 1 .. k-1, with the bounds
 * already tightened for those layers. Each layer's 2 n_k subproblems per box form batches of
 * contexts over the sub-network of layers 1 .. k (a conv layer k enters as its dense operator);
 * the solves run bigm_iters + as_iters iterations of opt (NULL: defaults) and the final iterate's
 * bound is taken. Layer 1 keeps its interval bounds (exact for an affine map of the box); every
 * layer's result is intersected with interval propagation and rounded outward to float32. Splits
 * act through interval propagation (as in as_init), whose clamped intervals contain the tightened
 * ones; every sub-network solve takes the clamped bounds of the layers before it.
 *  net, S, x_lo, x_hi, splits: as for as_init (host or device).
 *  max_batch:  subproblems per context (rounded down to even; 0: 16384), bounding device memory.
 *  lhat, uhat: outputs, hidden vectors [S][n_1 + ... + n_{n-1}] of float, host or device.
 *  stream:     cudaStream_t the work is enqueued on; the call synchronises it.
 * The results feed as_init / as_reset as caller bounds. Returns the first error of the contexts
 * it creates (AS_ERR_ARG, AS_ERR_SHAPE, AS_ERR_OOM, AS_ERR_CUDA, AS_ERR_NUMERIC). */
int as_intermediate_bounds(const as_net* net, int S, const float* x_lo, const float* x_hi,
                           const signed char* splits, const as_options* opt, long long max_batch,
                           float* lhat, float* uhat, void* stream);

/* Branch and bound with stratified bounding (Sec. 6.2) for one property c . f(x) > 0 over one
 * input box (the canonical form: the property holds when the minimum is positive).
 * Domains are (box, ReLU splits); each batch takes the batch / 2 domains with the lowest lower
 * bounds (creation order on ties) and bounds their children together: the split of the ambiguous
 * unsplit neuron with the largest -lhat uhat / (uhat - lhat) into +1 (passing, first) and -1
 * (blocking). A child's lower bound is the larger of its own solve's and its parent's; it is
 * pruned when positive. The network at the input point x_0* of each solve's final iterate gives
 * the upper bound (Sec. 6.2, footnote); the search stops "falsified" at a negative value
 * (confirmed by a float64 forward pass on the host), "verified" when no domain is left, and
 * "unknown" at a limit. Stratification: at the root l_{a_t-a_l} = l_{a_t}(r) - l_{a_l}(r); an
 * exponential moving average i of the parent-to-child increase (children solved by their parent's
 * algorithm; re-solves excluded) gives |s|_l = 2^(-l_{a_l}(p)/i + 1) - 1 and
 * |s|_t = 2^(-(l_{a_l}(p) + l_{a_t-a_l})/i + 1) - 1, and s with its whole subtree moves to a_t when
 * |s|_l / |s|_t > c_{a_t/a_l} (before the first sample: a_l; i <= 0: a_t when l_{a_t-a_l} > 0; a
 * non-positive |s|_t: a_t). Warm start (Sec. 8.2): a child's solve starts from its parent's final
 * alpha, beta_0, beta_1, with zero Adam moments, an empty active set and its algorithm's full
 * schedule. A domain with no ambiguous unsplit neuron left and a non-positive bound (an exact
 * relaxation whose solve has not converged) is solved again from its own duals up to
 * leaf_rebounds times, then set aside (the result is then "unknown" unless falsified).
 * Intermediate bounds of a domain: interval propagation with its split clamps, intersected with
 * the root's as_intermediate_bounds when root_intermediate is set. The input set is the box or,
 * with input_l2 in loose and tight (which must agree: AS_ERR_ARG), its inscribed ellipsoid. */
#define AS_BAB_UNKNOWN 0
#define AS_BAB_VERIFIED 1
#define AS_BAB_FALSIFIED 2
typedef struct as_bab_options {
    as_options loose;        /* a_l: the inexpensive algorithm (default Big-M, 180 iterations: Sec. 8.2) */
    as_options tight;        /* a_t: the tighter one (default: a_l's 180 Big-M iterations, which
                              * initialise Active Set (App. B), then 100 Active Set iterations)     */
    int stratify;            /* 1: switch from a_l to a_t as above; 0: a_t everywhere                */
    double cost_ratio;       /* c_{a_t/a_l}; <= 0: the ratio of the two root solves' measured times   */
    double ema_weight;       /* weight of the newest increase in the moving average (0.3)           */
    int batch;               /* children bounded together, even, >= 2 (Sec. 8.2: 200-300)           */
    long long max_domains;   /* solves after which the search stops "unknown"                       */
    double time_limit;       /* seconds after which it stops "unknown" (<= 0: none)                 */
    int warm_start;          /* 1: children start from their parent's duals                         */
    int leaf_rebounds;       /* re-solves of a domain that cannot be split (8)                      */
    int root_intermediate;   /* 1: tighten the root's intermediate bounds (as_intermediate_bounds)  */
    as_options intermediate; /* the schedule of those solves                                        */
} as_bab_options;

typedef struct as_bab_result {
    int status;              /* AS_BAB_VERIFIED, AS_BAB_FALSIFIED or AS_BAB_UNKNOWN                  */
    double lower;            /* min lower bound over the final frontier (pruned domains when empty)   */
    double upper;            /* least property value found (float64 forward at a solve's x_0*)       */
    long long bounded;       /* solves done (the root counts twice when stratified)                   */
    long long hard_bounded;  /* of which by a_t                                                       */
    long long batches, max_depth, frontier;
    double seconds;          /* wall time of the call                                                 */
    double cost_ratio;       /* the c_{a_t/a_l} in effect                                             */
} as_bab_result;

/* Fills *opt with the defaults above. */
void as_bab_default_options(as_bab_options* opt);

/* Runs the search.
 *  net:        as for as_init (host or device W, b).
 *  x_lo, x_hi: [n_0] the input box, host.
 *  c:          [n_out] the property row, host; NULL when n_out == 1 (c = 1).
 *  res:        host result; x_best: host [n_0] receiving the point of res->upper, or NULL.
 *  stream:     cudaStream_t every solve is enqueued on.
 * Device memory: three contexts of `batch` subproblems (a_l, a_t and a point evaluator) and the
 * alpha, beta_0, beta_1 of every open domain (12 bytes per hidden neuron per domain). Returns
 * AS_OK (the verdict is in res->status) or the first error of a context call. */
int as_bab(const as_net* net, const float* x_lo, const float* x_hi, const float* c, const as_bab_options* opt,
           as_bab_result* res, float* x_best, void* stream);

/* Whole-state export and import (warm starts; as_get_state / as_set_state over every buffer a
 * context needs to go on iterating): the iteration counters, alpha, beta_0, beta_1, the Adam
 * moments, the slots' betas, moments and snapshots (Active Set), or the primal iterate, sufficient
 * statistics and price caps (Saddle Point, once sp_step has started). Host memory of
 * as_export_size bytes; the import checks every buffer's size against the context before it
 * writes any (AS_ERR_SHAPE for another net, batch size or max_cuts, with the context left as it
 * was; AS_ERR_ARG for a blob this function did not write) and expects the batch (boxes,
 * properties, bounds) to be loaded already. The context takes the blob's mode: an Active Set blob
 * puts it in Active Set mode, a Saddle Point blob in Saddle Point mode (its initialisation
 * skipped). Lambda and kappa of the slots are recomputed in float32 from the imported snapshots,
 * so an imported context continues the exporting one's iterations up to that rounding. */
int as_export_size(as_ctx* ctx, long long* nbytes);
int as_export_state(as_ctx* ctx, void* dst);
int as_import_state(as_ctx* ctx, const void* src);

/* The team-size targets of the float32 Active Set passes in effect (threads a layer segment of
 * the row and of the col pass aims for; the lanes per neuron follow from them): the defaults,
 * what as_options.autotune chose, or the values of the environment variables
 * CB_TEAM_TARGET_ROW / CB_TEAM_TARGET_COL, which take precedence and are not tuned. Host
 * pointers; AS_ERR_ARG if any is null. No counterpart in the paper: launch geometry of this
 * implementation. */
int as_team_targets(as_ctx* ctx, long long* row, long long* col);

/* BF16 tensor-core GEMM, D = A . B^T (the building block of the BF16 form of the masked
 * products of Sec. 4.1 / eq. 6 and eq. 9: at Active Set iterates every masked product is a dense
 * product with W+ and W-, and the transposed one with their transposes).
 *  A: [M][K] bf16 (raw 16-bit), row stride lda elements; B: [N][K] bf16, row stride ldb; both
 *     device memory, 16-byte aligned, K, lda and ldb multiples of 8.
 *  D: [M][N] float32 device memory, row stride ldd (>= N); every entry is overwritten.
 *  bn: N tile of a CTA, 32, 64, 128 or 256 (tensor-memory columns it allocates).
 * Products are exact in float32; the sum over K accumulates in float32 in the tensor cores'
 * order. The call synchronises `stream`. Returns AS_ERR_ARG for bad sizes, strides or
 * alignment, AS_ERR_CUDA for a failed launch, AS_ERR_TIMEOUT if a bounded wait of the kernel on
 * its own tensor-core work ran out (D is then unspecified). */
int as_gemm_bf16(const void* A, int lda, const void* B, int ldb, float* D, int ldd, int M, int N, int K, int bn,
                 void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CONVEX_BARRIER_H */

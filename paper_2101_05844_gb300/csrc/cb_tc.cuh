// BF16 tensor-core GEMM on the 5th-generation tensor cores of sm_103a (tcgen05):
//   D[M][N] (float32) = A[M][K] (bf16) . B[N][K]^T (bf16)
// Both operands are K-major (rows of K contiguous elements), as the masked products of the
// Active Set iteration present them: rows of A are (slot, subproblem, position) inputs gathered
// from channels-last planes (an implicit-GEMM convolution, see Gather), rows of B the sign-split
// weights per output channel (row pass) or input channel (col pass).
//
// A CTA of 128 threads owns a 128 x BN tile of D, accumulated in tensor memory (TMEM: lane = row,
// column = output column, float32). K advances in tiles of 64: every thread stages 16-byte pieces
// of the A and B tiles into shared memory with cp.async, in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices; core (r8, k8) at byte ((r8 * 8) + k8) * 128 of the tile, so that
// core matrices adjacent in K are 128 bytes apart and those adjacent in M/N 1024 bytes apart),
// TC_STAGES deep (two: on GB300 more CTAs per SM hid the load latency better than deeper stages,
// measured with four). One thread issues four tcgen05.mma (K = 16 each) per tile and commits them
// to the stage's mbarrier; the stage is refilled once that barrier completes. The epilogue reads the
// accumulator back with tcgen05.ld (each warp its 32 TMEM lanes) and stores it to global memory.
//
// Convolutions whose kernel taps are shifts along one flat grid (stride-1 row passes, every stride
// phase of a col pass) take window operands instead (Window, win_tile): a CTA loads the input
// window of its 128 or 256 rows once, all taps included, and each K step's A descriptor starts at
// the tap's shift inside it, so that an input position is read from memory once per row block
// instead of once per tap; only B streams through the stages.
//
// Every wait is bounded: a stage barrier that does not complete within its limit (stage_limit)
// sets *status and the CTA stops issuing work, then waits for its last commit with the full limit
// (all of its MMAs are then complete), frees its TMEM and returns. Should that drain wait run out as
// well, MMAs may still be writing the CTA's TMEM: the CTA then returns without freeing it (results
// after AS_ERR_TIMEOUT are void either way).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "cb_common.cuh"

namespace cb {
namespace tc {

constexpr int TC_BM = 128, TC_BK = 64, TC_THREADS = 128, TC_STAGES = 2;
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;   // try_wait rounds before a barrier counts as lost
constexpr int TC_ERR_TIMEOUT = 6;             // value written to *status (AS_ERR_TIMEOUT)
constexpr int TC_ZERO_CHUNK = -2147483647 - 1; // K-offset marking a chunk of zeros

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Bounded wait for the completion of phase `parity`: at most `limit` try_wait rounds; false if the
// limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = TC_WAIT_LIMIT) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation of `ncols` columns (a power of two, >= 32) by one whole warp; the address is
// written to shared memory at dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: start address, leading-dimension byte offset (between core
// matrices adjacent in K), stride-dimension byte offset (adjacent in M/N), descriptor version 1,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1u) << 46;
    return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B, float32 D, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive float32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Stage `rows` rows x 64 K of a K-major bf16 matrix (row stride ld elements) into the canonical
// layout at smem byte address dst; rows >= nrows and K >= k_end are zero-filled.
__device__ __forceinline__ void stage_tile(uint32_t dst, const uint16_t* src, int ld, int row0, int nrows, int k0,
                                           int k_end, int rows) {
    for (int c = threadIdx.x; c < rows * 8; c += TC_THREADS) {
        const int r = c >> 3, k8 = c & 7;
        const int gr = row0 + r, gk = k0 + k8 * 8;
        const bool in = gr < nrows && gk < k_end;
        const uint16_t* p = in ? src + (size_t)gr * ld + gk : src;
        cp_async16(dst + static_cast<uint32_t>((((r >> 3) * 8) + k8) * 128 + (r & 7) * 16), p, in ? 16u : 0u);
    }
}

// Rows of the A operand gathered from a bf16 array: row m of A starts at element
//   rowbase(m) = (m / P) * plane + ((m % P) / Wq) * ry + ((m % P) % Wq) * rx + r0
// and its K-chunk c (8 consecutive K elements, 16 bytes) at rowbase(m) + kofs[c] (kofs == null:
// 8 c, a dense row-major matrix; kofs[c] == TC_ZERO_CHUNK: a chunk of zeros; offsets may be
// negative, relative to the row base). With channels-last planes padded to a multiple of 8
// channels this is an implicit-GEMM convolution: (m / P) picks the plane of a (slot, subproblem),
// (m % P) the output position, kofs the kernel tap and the channel octet.
struct Gather {
    const uint16_t* base;
    long long plane;
    int P, Wq;
    int ry, rx, r0;
    const int* kofs;
};

__device__ __forceinline__ long long gather_rowbase(const Gather& g, int m) {
    const int q = m / g.P, p = m - q * g.P;
    const int y = p / g.Wq, x = p - y * g.Wq;
    return (long long)q * g.plane + (long long)y * g.ry + (long long)x * g.rx + g.r0;
}

// Stage 128 rows x 64 K of the gathered A operand (row bases of the tile in rb[]).
__device__ __forceinline__ void stage_gather(uint32_t dst, const Gather& g, const long long* rb, int row0, int nrows,
                                             int k0, int k_end) {
    for (int c = threadIdx.x; c < TC_BM * 8; c += TC_THREADS) {
        const int r = c >> 3, k8 = c & 7;
        const int gk = k0 + k8 * 8;
        int ko = TC_ZERO_CHUNK;
        if (row0 + r < nrows && gk < k_end) ko = g.kofs ? __ldg(g.kofs + (gk >> 3)) : gk;
        const bool in = ko != TC_ZERO_CHUNK;
        const uint16_t* p = in ? g.base + rb[r] + ko : g.base;
        cp_async16(dst + static_cast<uint32_t>((((r >> 3) * 8) + k8) * 128 + (r & 7) * 16), p, in ? 16u : 0u);
    }
}

template <int BN>
constexpr int tc_smem_bytes() {
    return TC_STAGES * (TC_BM * TC_BK * 2 + BN * TC_BK * 2) + 64 + TC_BM * 8;
}

// One CTA's 128 x BN tile (blockIdx.x, blockIdx.y) of D = A . B^T with A [M][K] gathered as
// described by ga, B [N][K] (row stride ldb), D [M][N] (row stride ldd); K and ldb multiples of 8
// (16-byte row pieces).
// D layout: row-major [M][N] (row stride ldd), or with dt_P > 0 plane-transposed: row m = q dt_P + p
// of column n at D[(q N + n) dt_P + p] (for rows (plane, position): the positions of one column
// contiguous, so that lanes holding consecutive rows store consecutive addresses).
template <int BN>
__device__ __forceinline__ void gemm_tile(const Gather& ga, const uint16_t* __restrict__ B, int ldb,
                                          float* __restrict__ D, int ldd, int M, int N, int K, int* status,
                                          int dt_P = 0, uint32_t stage_limit = TC_WAIT_LIMIT) {
    static_assert(BN == 32 || BN == 64 || BN == 128 || BN == 256, "BN");
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int A_BYTES = TC_BM * TC_BK * 2, B_BYTES = BN * TC_BK * 2, STAGE = A_BYTES + B_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TC_STAGES * STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + TC_STAGES);
    long long* rb = reinterpret_cast<long long*>(smem + TC_STAGES * STAGE + 64);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
    if (warp == 0) tmem_alloc(tslot, BN);
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int r = tid; r < TC_BM; r += TC_THREADS) rb[r] = m0 + r < M ? gather_rowbase(ga, m0 + r) : 0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t sbase = smem_u32(smem);
    constexpr uint32_t idesc = idesc_bf16(TC_BM, BN);
    const int KT = (K + TC_BK - 1) / TC_BK;
    bool ok = true;

    // prologue: tiles 0 .. TC_STAGES - 2 in flight (one cp.async group per tile, empty past KT)
#pragma unroll
    for (int p = 0; p < TC_STAGES - 1; ++p) {
        if (p < KT) {
            const uint32_t st = sbase + p * STAGE;
            stage_gather(st, ga, rb, m0, M, p * TC_BK, K);
            stage_tile(st + A_BYTES, B, ldb, n0, N, p * TC_BK, K, BN);
        }
        cp_async_commit();
    }
    int issued = 0;   // commits issued by thread 0 (stage of commit c: c % TC_STAGES)
    for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % TC_STAGES;
        const int kn = kt + TC_STAGES - 1;   // the tile loaded this iteration
        bool w_ok = true;
        // its stage was last read by the MMAs of tile kt - 1
        if (kn < KT && kt >= 1)
            w_ok = mbar_wait(&bars[(kt - 1) % TC_STAGES], ((kt - 1) / TC_STAGES) & 1u, stage_limit);
        if (!__syncthreads_and(w_ok)) {   // the decision is the CTA's, so every thread leaves together
            ok = false;
            break;
        }
        if (kn < KT) {
            const uint32_t st = sbase + (kn % TC_STAGES) * STAGE;
            stage_gather(st, ga, rb, m0, M, kn * TC_BK, K);
            stage_tile(st + A_BYTES, B, ldb, n0, N, kn * TC_BK, K, BN);
        }
        cp_async_commit();
        cp_async_wait<TC_STAGES - 1>();   // tile kt has landed
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a = sbase + s * STAGE, b = a + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk)
                mma_bf16(tmem, smem_desc(a + kk * 256, 128, 1024), smem_desc(b + kk * 256, 128, 1024), idesc,
                         (kt > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&bars[s]);
        }
        ++issued;
    }
    cp_async_wait<0>();
    // every thread waits for the last commit (all MMAs issued before it are then complete)
    bool f_ok = true;
    if (issued > 0) {
        const int last = issued - 1;
        f_ok = mbar_wait(&bars[last % TC_STAGES], (last / TC_STAGES) & 1u);
    }
    const bool drained = __syncthreads_and(f_ok);
    ok = __syncthreads_and(ok && drained);
    if (!ok && tid == 0 && status) atomicExch(status, TC_ERR_TIMEOUT);
    tc_fence_after();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
            if (row < M && dt_P > 1) {   // (one position per plane is the row-major layout)
                const int q = row / dt_P, p = row - q * dt_P;
                float* dr = D + ((size_t)q * N + n0 + c0) * dt_P + p;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (n0 + c0 + j < N) dr[(size_t)j * dt_P] = v[j];
            } else if (row < M) {
                float* dr = D + (size_t)row * ldd + n0 + c0;
                if (n0 + c0 + 16 <= N && (ldd & 3) == 0) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(dr + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (n0 + c0 + j < N) dr[j] = v[j];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && drained) tmem_free(tmem, BN);
}

// A operand of a convolution whose kernel taps are shifts along one flat grid: rows m of A are the
// positions of planes of Pg grid positions laid end to end (plane q = m / Pg), and for tap t row m
// reads source position m + lo + shift[t] (stride 1 over the source grid: a row-pass convolution
// of stride 1 over the zero-padded input plane, or a stride phase of a col-pass transposed
// convolution over the output plane with its zero halo). A source position carries 8-channel
// column blocks (sign, octet): block (g, o) of position p in plane q at element
//   base + q pstride + g sign_off + (p - q Pg) cstride + 8 o,
// zeros outside [0, npos). The K order of B is (tap, block, 8 channels), the blocks padded to an
// even count ncp (zero blocks) so that every K step of 16 lies within one tap. Rows are outputs
// where the grid position (y, x) = ((m % Pg) / Wg, (m % Pg) % Wg) lies in [y0, y0 + ny) x
// [x0, x0 + nx), output index q (ny nx) + (y - y0) nx + (x - x0); the other rows are computed and
// dropped.
constexpr int CB_WIN_TAPS = 16;
struct Window {
    const uint16_t* base;
    long long pstride, sign_off, npos;
    int nsign, noct, ncp, cstride;
    int lo, nw;                     // window start relative to the tile's first row; positions held
    int bwhole;                     // 1: all of B staged at once with the window (one wait), else streamed
    int ntaps;
    int shift[CB_WIN_TAPS];         // per tap, relative to the window start (0 .. nw - rows)
    int Pg, Wg, y0, x0, ny, nx;
};

// Shared memory of a window tile: bst B stages (TC_STAGES, or every K tile of B when it is staged
// whole), the window (ncp blocks of nw positions, 16 bytes each), barriers and the TMEM address.
__host__ __device__ constexpr int win_smem_bytes(int bn, int ncp, int nw, int bst) {
    return bst * bn * TC_BK * 2 + ncp * nw * 16 + 64;
}

// One CTA's MT x 128 rows x BN columns of D = A . B^T with A the window operand w: the CTA loads
// its window once (every tap's rows), then streams B in K tiles of 64 through TC_STAGES stages; the
// MMA of K step c (tap t = c / (ncp / 2), block pair j) takes its A operand at the window position
// shift[t] (+ 128 u for row block u) and blocks 2j, 2j + 1: core matrices adjacent in M 128 bytes
// apart, in K nw * 16 bytes. Accumulators: MT x BN TMEM columns. D plane-transposed over the output
// positions (Pq = ny nx per plane): row m's column n at D[(q N + n) Pq + output index].
template <int BN, int MT>
__device__ __forceinline__ void win_tile(const Window& w, const uint16_t* __restrict__ B, int ldb,
                                         float* __restrict__ D, int M, int N, int K, int* status,
                                         uint32_t stage_limit) {
    static_assert(BN == 16 || BN == 32 || BN == 64 || BN == 128, "BN");
    static_assert(MT == 1 || MT == 2, "MT");
    constexpr int B_BYTES = BN * TC_BK * 2;
    constexpr uint32_t TCOLS = MT * BN < 32 ? 32u : static_cast<uint32_t>(MT * BN);
    extern __shared__ __align__(128) uint8_t smem[];
    const int nw = w.nw, ncp = w.ncp;
    const int KT = (K + TC_BK - 1) / TC_BK, nchunks = K / 16, cpt = ncp / 2;
    const int bst = w.bwhole ? (KT > TC_STAGES ? KT : TC_STAGES) : TC_STAGES;
    uint8_t* winp = smem + bst * B_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(winp + ncp * nw * 16);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + TC_STAGES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * (MT * TC_BM), n0 = blockIdx.y * BN;
    if (warp == 0) tmem_alloc(tslot, TCOLS);
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint32_t sbase = smem_u32(smem), wbase = smem_u32(winp);
    // the window: positions m0 + lo .. m0 + lo + nw - 1, block fastest (a position's blocks are
    // adjacent in global memory). With ncp a power of two a thread keeps one block and walks the
    // positions TC_THREADS / ncp apart, its plane and in-plane position carried along.
    {
        const long long p0 = (long long)m0 + w.lo;
        const int ncols = w.nsign * w.noct;
        const int q0 = p0 >= 0 ? (int)(p0 / w.Pg) : 0;
        if ((ncp & (ncp - 1)) == 0 && ncp <= TC_THREADS) {
            const int lg = __ffs(ncp) - 1, cb = tid & (ncp - 1), dr = TC_THREADS >> lg;
            const int g = cb / w.noct, o = cb - g * w.noct;
            const uint16_t* bsrc = w.base + g * w.sign_off + o * 8;
            int r = tid >> lg, q = q0;
            long long pr = p0 + r - (long long)q0 * w.Pg;
            for (; r < nw; r += dr, pr += dr) {
                while (pr >= w.Pg) {   // a step of dr < Pg positions crosses at most one plane
                    pr -= w.Pg;
                    ++q;
                }
                const long long pos = p0 + r;
                const bool in = cb < ncols && pos >= 0 && pos < w.npos;
                const uint16_t* src = in ? bsrc + (long long)q * w.pstride + pr * w.cstride : w.base;
                cp_async16(wbase + static_cast<uint32_t>((cb * nw + r) * 16), src, in ? 16u : 0u);
            }
        } else {
            for (int i = tid; i < nw * ncp; i += TC_THREADS) {
                const int r = i / ncp, cb = i - r * ncp;
                const long long pos = p0 + r;
                const bool in = cb < ncols && pos >= 0 && pos < w.npos;
                const uint16_t* src = w.base;
                if (in) {
                    int q = q0;
                    long long pr = pos - (long long)q0 * w.Pg;
                    while (pr >= w.Pg) {   // a window spans at most nw / Pg + 1 planes
                        pr -= w.Pg;
                        ++q;
                    }
                    const int g = cb / w.noct, o = cb - g * w.noct;
                    src = w.base + (long long)q * w.pstride + g * w.sign_off + pr * w.cstride + o * 8;
                }
                cp_async16(wbase + static_cast<uint32_t>((cb * nw + r) * 16), src, in ? 16u : 0u);
            }
        }
    }
    if (KT > 0) stage_tile(sbase, B, ldb, n0, N, 0, K, BN);
    if (w.bwhole)
        for (int kt = 1; kt < KT; ++kt) stage_tile(sbase + kt * B_BYTES, B, ldb, n0, N, kt * TC_BK, K, BN);
    cp_async_commit();   // group 0: the window and B tile 0 (all of B when staged whole)
#pragma unroll
    for (int p = 1; p < TC_STAGES - 1; ++p) {
        if (p < KT && !w.bwhole) stage_tile(sbase + p * B_BYTES, B, ldb, n0, N, p * TC_BK, K, BN);
        cp_async_commit();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = idesc_bf16(TC_BM, BN);
    bool ok = true;
    int issued = 0;
    if (w.bwhole && KT > 0) {
        // one wait for the window and B, every MMA, one commit; a wait that runs out (stage_limit)
        // stops the CTA as in the streamed loop, the drain below waiting with the full limit
        cp_async_wait<0>();
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int c = 0; c < nchunks; ++c) {
                const int t = c / cpt, j = c - t * cpt;
                const uint32_t a = wbase + static_cast<uint32_t>((2 * j * nw + w.shift[t]) * 16);
                const uint64_t bd = smem_desc(sbase + (c >> 2) * B_BYTES + (c & 3) * 256, 128, 1024);
#pragma unroll
                for (int u = 0; u < MT; ++u)
                    mma_bf16(tmem + u * BN, smem_desc(a + u * TC_BM * 16, nw * 16, 128), bd, idesc, c > 0 ? 1u : 0u);
            }
            mma_commit(&bars[0]);
        }
        issued = 1;
        ok = __syncthreads_and(mbar_wait(&bars[0], 0u, stage_limit));
    }
    for (int kt = 0; kt < KT && !w.bwhole; ++kt) {
        const int s = kt % TC_STAGES;
        const int kn = kt + TC_STAGES - 1;
        bool w_ok = true;
        if (kn < KT && kt >= 1)
            w_ok = mbar_wait(&bars[(kt - 1) % TC_STAGES], ((kt - 1) / TC_STAGES) & 1u, stage_limit);
        if (!__syncthreads_and(w_ok)) {
            ok = false;
            break;
        }
        if (kn < KT) stage_tile(sbase + (kn % TC_STAGES) * B_BYTES, B, ldb, n0, N, kn * TC_BK, K, BN);
        cp_async_commit();
        cp_async_wait<TC_STAGES - 1>();
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t b = sbase + s * B_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const int c = kt * (TC_BK / 16) + kk;
                if (c < nchunks) {
                    const int t = c / cpt, j = c - t * cpt;
                    const uint32_t a = wbase + static_cast<uint32_t>((2 * j * nw + w.shift[t]) * 16);
                    const uint64_t bd = smem_desc(b + kk * 256, 128, 1024);
#pragma unroll
                    for (int u = 0; u < MT; ++u)
                        mma_bf16(tmem + u * BN, smem_desc(a + u * TC_BM * 16, nw * 16, 128), bd, idesc,
                                 c > 0 ? 1u : 0u);
                }
            }
            mma_commit(&bars[s]);
        }
        ++issued;
    }
    cp_async_wait<0>();
    bool f_ok = true;
    if (issued > 0) {
        const int last = issued - 1;
        f_ok = mbar_wait(&bars[last % TC_STAGES], (last / TC_STAGES) & 1u);
    }
    const bool drained = __syncthreads_and(f_ok);
    ok = __syncthreads_and(ok && drained);
    if (!ok && tid == 0 && status) atomicExch(status, TC_ERR_TIMEOUT);
    tc_fence_after();
    if (ok) {
        const long long Pq = (long long)w.ny * w.nx;
#pragma unroll 1
        for (int u = 0; u < MT; ++u) {
            const int m = m0 + u * TC_BM + warp * 32 + lane;
            long long dofs = -1;
            if (m < M) {
                const int q = m / w.Pg, p = m - q * w.Pg;
                const int y = p / w.Wg - w.y0, x = p % w.Wg - w.x0;
                if (y >= 0 && y < w.ny && x >= 0 && x < w.nx) dofs = (long long)q * N * Pq + (long long)y * w.nx + x;
            }
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + u * BN + c0, v);
                if (dofs >= 0) {
                    float* dr = D + dofs + (long long)(n0 + c0) * Pq;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (n0 + c0 + j < N) dr[(long long)j * Pq] = v[j];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && drained) tmem_free(tmem, TCOLS);
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_bf16(Gather ga, const uint16_t* __restrict__ B, int ldb,
                                                          float* __restrict__ D, int ldd, int M, int N, int K,
                                                          int* status) {
    gemm_tile<BN>(ga, B, ldb, D, ldd, M, N, K, status);
}

// Up to CB_MAXPH GEMMs of one shape class in one launch (blockIdx.z picks one): the stride phases
// of a transposed convolution, or a single row-pass GEMM. The rows in use follow the Active Set
// schedule read from the device iteration counter: (1 + slots) x rows_per_slot, where slots is
// the number of active-set slots the pass consumes (row pass: those added up to and including
// the current iteration; col pass: before it). CTAs past the rows in use return at once.
struct GemmGroup {
    Gather ga[CB_MAXPH];
    Window wa[CB_MAXPH];          // window operands (k_gemm_wgroup_bf16)
    const uint16_t* B[CB_MAXPH];
    float* D[CB_MAXPH];
    int M[CB_MAXPH];              // rows for all 1 + cap slots
    int K[CB_MAXPH];
    int rows_per_slot[CB_MAXPH];
    int ldb[CB_MAXPH];
    int N, ldd;
    int transposed;               // store D plane-transposed with the gather's P (gemm_tile)
    const int* ctr;               // device iteration counter
    DSched sc;
    int row_pass;
    uint32_t stage_limit;         // try_wait rounds of a stage wait (TC_WAIT_LIMIT; smaller only to
                                  // exercise the timeout path)
};

// Rows of GEMM g in use at the current iteration.
__device__ __forceinline__ int group_rows(const GemmGroup& gg, int g) {
    const int it = *gg.ctr;
    int ns = 0;
    if (it >= gg.sc.TM) {
        const int t = it - gg.sc.TM;
        ns = cb_additions_before(t, gg.sc);
        if (gg.row_pass && cb_slot_at(t, gg.sc) >= 0) ++ns;
        ns = ns < gg.sc.maxcut ? ns : gg.sc.maxcut;
    }
    const long long want = (long long)(1 + ns) * gg.rows_per_slot[g];
    return want < gg.M[g] ? (int)want : gg.M[g];
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_group_bf16(GemmGroup gg, int* status) {
    const int g = blockIdx.z;
    const int M = group_rows(gg, g);
    if ((int)blockIdx.x * TC_BM >= M) return;   // the whole CTA leaves together, before any barrier
    gemm_tile<BN>(gg.ga[g], gg.B[g], gg.ldb[g], gg.D[g], gg.ldd, M, gg.N, gg.K[g], status,
                  gg.transposed && gg.ga[g].P > 1 ? gg.ga[g].P : 0, gg.stage_limit);
}

// The group's GEMMs with window operands (win_tile), MT row blocks of 128 per CTA.
template <int BN, int MT>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_wgroup_bf16(GemmGroup gg, int* status) {
    const int g = blockIdx.z;
    const int M = group_rows(gg, g);
    if ((long long)blockIdx.x * (MT * TC_BM) >= M) return;
    win_tile<BN, MT>(gg.wa[g], gg.B[g], gg.ldb[g], gg.D[g], M, gg.N, gg.K[g], status, gg.stage_limit);
}

}  // namespace tc
}  // namespace cb

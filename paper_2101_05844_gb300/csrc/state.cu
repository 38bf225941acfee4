// Whole-state export and import for warm starts, on the library's own state entry points: one
// blob holding every buffer a context needs to continue its iterations exactly (the duals, the
// active set's slots and their snapshots, the Adam moments and the iteration counters; in Saddle
// Point mode its primal iterate, sufficient statistics and price caps instead of the slots).
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/convex_barrier.h"

namespace {

constexpr int32_t kMagic = 0x43425331;   // "CBS1"

// The counter first (the snapshot and primal buffers are double-buffered by its parity); last, a
// buffer whose import rebuilds the derived records: the slots' betas (lambda, kappa of every slot)
// and, in Saddle Point, alpha (the records of alpha and the statistics).
const int kActiveSet[] = {AS_ST_ITER,  AS_ST_ALPHA,    AS_ST_BETA0, AS_ST_BETA1,    AS_ST_ADAM,
                          AS_ST_SLOT_ADAM, AS_ST_XSNAP, AS_ST_ZSNAP, AS_ST_SLOT_BETA};
const int kSaddle[] = {AS_ST_ITER, AS_ST_SP_X, AS_ST_SP_Z, AS_ST_SP_STATS, AS_ST_SP_CAPS, AS_ST_ALPHA};

int mode_of(as_ctx* c, int* sp) {
    int v[3];
    const int r = as_get_state(c, AS_ST_ITER, v);
    if (r == AS_OK) *sp = v[2];
    return r;
}

int layout(as_ctx* c, int sp, std::vector<long long>& sizes) {
    const int* ids = sp ? kSaddle : kActiveSet;
    const int n = sp ? (int)(sizeof kSaddle / sizeof *kSaddle) : (int)(sizeof kActiveSet / sizeof *kActiveSet);
    sizes.assign(n, 0);
    for (int q = 0; q < n; ++q) {
        const int r = as_state_size(c, ids[q], &sizes[q]);
        if (r != AS_OK) return r;
    }
    return AS_OK;
}

}  // namespace

extern "C" int as_export_size(as_ctx* c, long long* nbytes) {
    if (!c || !nbytes) return AS_ERR_ARG;
    int sp = 0, r = mode_of(c, &sp);
    std::vector<long long> sizes;
    if (r == AS_OK) r = layout(c, sp, sizes);
    if (r != AS_OK) return r;
    long long t = 2 * sizeof(int32_t);
    for (long long b : sizes) t += sizeof(long long) + b;
    *nbytes = t;
    return AS_OK;
}

extern "C" int as_export_state(as_ctx* c, void* dst) {
    if (!c || !dst) return AS_ERR_ARG;
    int sp = 0, r = mode_of(c, &sp);
    std::vector<long long> sizes;
    if (r == AS_OK) r = layout(c, sp, sizes);
    if (r != AS_OK) return r;
    const int* ids = sp ? kSaddle : kActiveSet;
    std::vector<unsigned char> tmp;
    unsigned char* p = static_cast<unsigned char*>(dst);
    const int32_t head[2] = {kMagic, sp};
    std::memcpy(p, head, sizeof head);
    p += sizeof head;
    for (size_t q = 0; q < sizes.size(); ++q) {
        std::memcpy(p, &sizes[q], sizeof(long long));
        p += sizeof(long long);
        tmp.resize(sizes[q]);
        if ((r = as_get_state(c, ids[q], tmp.data())) != AS_OK) return r;
        std::memcpy(p, tmp.data(), sizes[q]);
        p += sizes[q];
    }
    return AS_OK;
}

extern "C" int as_import_state(as_ctx* c, const void* src) {
    if (!c || !src) return AS_ERR_ARG;
    const unsigned char* p = static_cast<const unsigned char*>(src);
    int32_t head[2];
    std::memcpy(head, p, sizeof head);
    p += sizeof head;
    if (head[0] != kMagic || (head[1] != 0 && head[1] != 1)) return AS_ERR_ARG;
    const int sp = head[1];
    std::vector<long long> sizes;
    int r = layout(c, sp, sizes);
    if (r != AS_OK) return r;
    // every section's size first, so that a blob of another net, batch size or max_cuts leaves the
    // context untouched
    const unsigned char* q = p;
    for (size_t k = 0; k < sizes.size(); ++k) {
        long long b = 0;
        std::memcpy(&b, q, sizeof b);
        if (b != sizes[k]) return AS_ERR_SHAPE;
        q += sizeof b + b;
    }
    const int* ids = sp ? kSaddle : kActiveSet;
    for (size_t k = 0; k < sizes.size(); ++k) {
        p += sizeof(long long);
        if ((r = as_set_state(c, ids[k], p)) != AS_OK) return r;
        p += sizes[k];
    }
    return AS_OK;
}

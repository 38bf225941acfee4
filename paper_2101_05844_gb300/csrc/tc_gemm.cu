// C ABI of the BF16 tensor-core GEMM (cb_tc.cuh): the building block of the BF16 form of the
// masked products. Exposed so that its numerics are checked on their own.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/convex_barrier.h"
#include "cb_tc.cuh"

using namespace cb::tc;

namespace {
__device__ int g_tc_status;

template <int BN>
cudaError_t launch(const uint16_t* A, int lda, const uint16_t* B, int ldb, float* D, int ldd, int M, int N, int K,
                   int* status, cudaStream_t s) {
    const int smem = tc_smem_bytes<BN>();
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((M + TC_BM - 1) / TC_BM, (N + BN - 1) / BN);
    Gather ga{A, (long long)lda, 1, 1, 0, 0, 0, nullptr};   // dense: row m at m * lda
    k_gemm_bf16<BN><<<grid, TC_THREADS, smem, s>>>(ga, B, ldb, D, ldd, M, N, K, status);
    return cudaGetLastError();
}
}  // namespace

extern "C" int as_gemm_bf16(const void* A, int lda, const void* B, int ldb, float* D, int ldd, int M, int N, int K,
                            int bn, void* stream) {
    if (!A || !B || !D || M < 1 || N < 1 || K < 1) return AS_ERR_ARG;
    if (K % 8 || lda % 8 || ldb % 8 || lda < K || ldb < K || ldd < N) return AS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) return AS_ERR_ARG;
    if (bn != 32 && bn != 64 && bn != 128 && bn != 256) return AS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* status = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&status), g_tc_status) != cudaSuccess) return AS_ERR_CUDA;
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return AS_ERR_CUDA;
    const uint16_t* a = static_cast<const uint16_t*>(A);
    const uint16_t* b = static_cast<const uint16_t*>(B);
    cudaError_t e;
    switch (bn) {
        case 32: e = launch<32>(a, lda, b, ldb, D, ldd, M, N, K, status, s); break;
        case 64: e = launch<64>(a, lda, b, ldb, D, ldd, M, N, K, status, s); break;
        case 128: e = launch<128>(a, lda, b, ldb, D, ldd, M, N, K, status, s); break;
        default: e = launch<256>(a, lda, b, ldb, D, ldd, M, N, K, status, s); break;
    }
    if (e != cudaSuccess) return AS_ERR_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return AS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return AS_ERR_CUDA;
    return h ? AS_ERR_TIMEOUT : AS_OK;
}

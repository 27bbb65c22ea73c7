// qmcrt_mlp.cu -- launchers of the tensor-core GEMM (qmcrt_gemm.cuh) used by the
// learned proposal.
#include "qmcrt.h"
#include "qmcrt_gemm.cuh"
#include "qmcrt_internal.h"

namespace qmcrt {

template <int N>
static cudaError_t launch_n(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int K, int k_per, dim3 grid,
                            const GemmEpi &ep, cudaStream_t s)
{
    constexpr int smem = gemm_smem_bytes<N>();
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_gemm_bf16<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    k_gemm_bf16<N><<<grid, GEMM_THREADS, smem, s>>>(A, B, M, K, k_per, ep);
    return cudaGetLastError();
}

cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int splits,
                             const GemmEpi &ep, cudaStream_t s)
{
    const int k_per = ((K + splits - 1) / splits + GEMM_BK - 1) / GEMM_BK * GEMM_BK;
    const dim3 grid((M + GEMM_BM - 1) / GEMM_BM, (K + k_per - 1) / k_per);
    switch (N) {
    case 32: return launch_n<32>(A, B, M, K, k_per, grid, ep, s);
    case 64: return launch_n<64>(A, B, M, K, k_per, grid, ep, s);
    case 128: return launch_n<128>(A, B, M, K, k_per, grid, ep, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qmcrt

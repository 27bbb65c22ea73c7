// qmcrt_mlp.cu -- launchers of the tensor-core GEMM (qmcrt_gemm.cuh) used by the
// learned proposal.
#include "qmcrt.h"
#include "qmcrt_gemm.cuh"
#include "qmcrt_internal.h"

namespace qmcrt {

cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int splits,
                             const GemmEpi &ep, cudaStream_t s)
{
    const int k_per = ((K + splits - 1) / splits + GEMM_BK - 1) / GEMM_BK * GEMM_BK;
    const dim3 grid((M + GEMM_BM - 1) / GEMM_BM, (K + k_per - 1) / k_per);
    switch (N) {
    case 32: k_gemm_bf16<32><<<grid, GEMM_THREADS, 0, s>>>(A, B, M, K, k_per, ep); break;
    case 64: k_gemm_bf16<64><<<grid, GEMM_THREADS, 0, s>>>(A, B, M, K, k_per, ep); break;
    case 128: k_gemm_bf16<128><<<grid, GEMM_THREADS, 0, s>>>(A, B, M, K, k_per, ep); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace qmcrt

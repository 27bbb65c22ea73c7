// qmcrt_mlp.cu -- launchers of the tensor-core GEMM (qmcrt_gemm.cuh) used by the
// learned proposal: the persistent warp-specialised tensor-copy form for K <= 128 without
// a K split, the tensor-copy split-K form for the weight gradients (one 128-row tile,
// FP32 vector reductions), the streaming form otherwise (and wherever a tensor map cannot
// be made).
#include <cudaTypedefs.h>

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

// Tensor map of a K-contiguous bf16 matrix [rows][K]: boxes of 8 elements x box_rows.
static bool make_tmap(CUtensorMap *m, const void *ptr, int K, int rows, int box_rows)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// false: the persistent form does not apply (the caller streams instead).
template <int N>
static bool launch_tma(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int K, const GemmEpi &ep,
                       cudaStream_t s, cudaError_t &err)
{
    constexpr int smem = gemm_ws_smem_bytes<N>();
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_gemm_bf16_ws<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return false;
    CUtensorMap ma, mb;
    if (!make_tmap(&ma, A, K, M, GEMM_BM) || !make_tmap(&mb, B, K, N, N)) return false;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return false;
    const int ntiles = (M + GEMM_BM - 1) / GEMM_BM;
    k_gemm_bf16_ws<N><<<ntiles < sms ? ntiles : sms, GEMM_WS_THREADS, smem, s>>>(ma, mb, M, K, ep);
    err = cudaGetLastError();
    return true;
}

// false: the tensor-copy split-K form does not apply.
template <int N>
static bool launch_splitk(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int K, int k_per, dim3 grid,
                          const GemmEpi &ep, cudaStream_t s, cudaError_t &err)
{
    constexpr int smem = gemm_sk_smem_bytes<N>();
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_gemm_bf16_splitk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return false;
    CUtensorMap ma, mb;
    if (!make_tmap(&ma, A, K, M, GEMM_BM) || !make_tmap(&mb, B, K, N, N)) return false;
    k_gemm_bf16_splitk<N><<<grid, GEMM_THREADS, smem, s>>>(ma, mb, M, K, k_per, ep);
    err = cudaGetLastError();
    return true;
}

cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int splits,
                             const GemmEpi &ep, cudaStream_t s)
{
    if (splits <= 1 && !ep.atomic_f32 && K <= GEMM_T_KMAX && K % 16 == 0) {
        cudaError_t err = cudaSuccess;
        bool done = false;
        switch (N) {
        case 32: done = launch_tma<32>(A, B, M, K, ep, s, err); break;
        case 64: done = launch_tma<64>(A, B, M, K, ep, s, err); break;
        case 128: done = launch_tma<128>(A, B, M, K, ep, s, err); break;
        default: return cudaErrorInvalidValue;
        }
        if (done) return err;
    }
    const int k_per = ((K + splits - 1) / splits + GEMM_BK - 1) / GEMM_BK * GEMM_BK;
    const dim3 grid((M + GEMM_BM - 1) / GEMM_BM, (K + k_per - 1) / k_per);
    if (ep.atomic_f32 && ep.out_f32 && !ep.bias && !ep.mask && !ep.out_bf16 && !ep.out_bf16_t && M <= GEMM_BM) {
        cudaError_t err = cudaSuccess;
        bool done = false;
        switch (N) {
        case 32: done = launch_splitk<32>(A, B, M, K, k_per, grid, ep, s, err); break;
        case 64: done = launch_splitk<64>(A, B, M, K, k_per, grid, ep, s, err); break;
        case 128: done = launch_splitk<128>(A, B, M, K, k_per, grid, ep, s, err); break;
        default: return cudaErrorInvalidValue;
        }
        if (done) return err;
    }
    switch (N) {
    case 32: return launch_n<32>(A, B, M, K, k_per, grid, ep, s);
    case 64: return launch_n<64>(A, B, M, K, k_per, grid, ep, s);
    case 128: return launch_n<128>(A, B, M, K, k_per, grid, ep, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qmcrt

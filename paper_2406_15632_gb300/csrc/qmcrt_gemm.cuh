// qmcrt_gemm.cuh -- BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05)
// with fused epilogues: the building block of the learned proposal's MLP (inference
// and training).
//
//   D[M x N] = A[M x K] . B[N x K]^T  (+ bias, ReLU, ReLU-mask, ...)
//
// A and B are BF16, row-major with K contiguous, in global memory.  One CTA of 128
// threads computes one 128-row tile of D (N = 32, 64 or 128 columns); a split of the K
// range over gridDim.y adds partial tiles atomically.  Per 32-wide K chunk the CTA
// copies the A and B chunks into shared memory in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices, contiguous; adjacent core matrices along K
// 128 bytes apart, along M/N 512 bytes apart), one thread issues two
// tcgen05.mma.cta_group::1.kind::f16 (K = 16 each) into an FP32 accumulator in tensor
// memory, and commits them to an mbarrier that all threads wait on (bounded: a wait
// that runs out sets an error word and the kernel skips to the end, freeing its tensor
// memory).  The epilogue reads the accumulator with tcgen05.ld (each warp its 32
// lanes = rows).
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace qmcrt {

// Epilogue of one GEMM launch.  Output pointers that are null are skipped.
struct GemmEpi {
    const float *bias;          // [N] added to every row
    int relu;                   // max(0, .) after the bias
    const __nv_bfloat16 *mask;  // [M][N]: zero the entry where mask <= 0 (ReLU backward)
    float *out_f32;             // [M][N] (overwritten, or added atomically when split over K)
    __nv_bfloat16 *out_bf16;    // [M][N]
    __nv_bfloat16 *out_bf16_t;  // [N][ldt]: transposed copy, row n holds column n of D
    int ldt;                    // leading dimension of out_bf16_t (>= M)
    int atomic_f32;             // add into out_f32 with atomics (K split over gridDim.y)
    int *error;                 // set to 1 if a tensor-core wait gives up
};

constexpr int GEMM_BM = 128;     // rows per CTA (one TMEM lane per row)
constexpr int GEMM_BK = 32;      // K per shared-memory chunk (two MMAs of K = 16)
constexpr int GEMM_THREADS = 128;
constexpr long long GEMM_WAIT_LIMIT = 1ll << 24;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major, no swizzle: start address, leading byte
// offset (between core matrices adjacent along K), stride byte offset (between 8-row
// groups), descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // version
    return d;                // base offset 0, relative LBO, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, dense.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int N>
struct GemmSmem {
    alignas(128) uint8_t a[GEMM_BM * GEMM_BK * 2];  // 8 KB
    alignas(128) uint8_t b[N * GEMM_BK * 2];
    alignas(8) unsigned long long mbar;
    uint32_t tmem;
    int fail;
};

// Copy a [rows x 32] BF16 chunk (row stride ld elements) into the canonical layout:
// row r, element c -> ((r / 8) * 4 + c / 8) * 128 + (r % 8) * 16 + (c % 8) * 2 bytes.
template <int ROWS>
__device__ __forceinline__ void stage_chunk(uint8_t *dst, const __nv_bfloat16 *src, int row0, int nrows, long long ld,
                                            int k0, int K)
{
    constexpr int VEC = ROWS * GEMM_BK / 8;  // 16-byte vectors
    for (int v = threadIdx.x; v < VEC; v += GEMM_THREADS) {
        const int r = v >> 2, kb = v & 3;
        uint4 val = make_uint4(0, 0, 0, 0);
        const int gr = row0 + r, gk = k0 + kb * 8;
        if (gr < nrows && gk < K) val = *reinterpret_cast<const uint4 *>(src + (long long)gr * ld + gk);
        *reinterpret_cast<uint4 *>(dst + ((r >> 3) * 4 + kb) * 128 + (r & 7) * 16) = val;
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase)
{
    for (long long it = 0; it < GEMM_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int N>
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm_bf16(const __nv_bfloat16 *__restrict__ A,
                                                           const __nv_bfloat16 *__restrict__ B, int M, int K,
                                                           int k_per_split, GemmEpi ep)
{
    static_assert(N == 32 || N == 64 || N == 128, "N tile");
    constexpr int TMEM_COLS = N < 32 ? 32 : N;
    __shared__ GemmSmem<N> sm;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * GEMM_BM;
    const int kbeg = blockIdx.y * k_per_split, kend = min(K, kbeg + k_per_split);
    if (tid == 0) {
        sm.fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm.tmem;
    const uint32_t idesc = umma_idesc_bf16(GEMM_BM, N);
    uint32_t phase = 0;
    bool any = false;
    for (int k0 = kbeg; k0 < kend; k0 += GEMM_BK) {
        stage_chunk<GEMM_BM>(sm.a, A, row0, M, K, k0, kend);
        stage_chunk<N>(sm.b, B, 0, N, K, k0, kend);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < GEMM_BK / 16; ++s) {
                const uint64_t ad = umma_desc(smem_u32(sm.a) + s * 256, 128, 512);
                const uint64_t bd = umma_desc(smem_u32(sm.b) + s * 256, 128, 512);
                const uint32_t acc = (any || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&sm.mbar))
                         : "memory");
        }
        any = true;
        if (!mbar_wait(smem_u32(&sm.mbar), phase)) sm.fail = 1;
        phase ^= 1u;
        __syncthreads();
        if (sm.fail) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!sm.fail && any) {
        // epilogue: this thread owns row (32 * warp + lane) of the tile
        const int row = row0 + warp * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 32) {
            uint32_t r[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = c0 + j;
                    float v = __uint_as_float(r[j]);
                    if (ep.bias) v += ep.bias[col];
                    if (ep.relu) v = fmaxf(v, 0.0f);
                    if (ep.mask && !(__bfloat162float(ep.mask[(long long)row * N + col]) > 0.0f)) v = 0.0f;
                    if (ep.out_f32) {
                        if (ep.atomic_f32) atomicAdd(ep.out_f32 + (long long)row * N + col, v);
                        else ep.out_f32[(long long)row * N + col] = v;
                    }
                    if (ep.out_bf16) ep.out_bf16[(long long)row * N + col] = __float2bfloat16_rn(v);
                    if (ep.out_bf16_t) ep.out_bf16_t[(long long)col * ep.ldt + row] = __float2bfloat16_rn(v);
                }
            }
        }
    }
    if (sm.fail && tid == 0 && ep.error) atomicExch(ep.error, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace qmcrt

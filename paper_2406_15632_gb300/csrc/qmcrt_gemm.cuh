// qmcrt_gemm.cuh -- BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05)
// with fused epilogues: the building block of the learned proposal's MLP (inference
// and training).
//
//   D[M x N] = A[M x K] . B[N x K]^T  (+ bias, ReLU, ReLU-mask, ...)
//
// A and B are BF16, row-major with K contiguous, in global memory.  One CTA of 128
// threads computes one 128-row tile of D (N = 32, 64 or 128 columns); a split of the K
// range over gridDim.y adds partial tiles atomically.  K is taken in 64-wide chunks
// through two shared-memory stages: asynchronous 16-byte copies (cp.async) write the A
// and B chunks in the canonical K-major layout without swizzle (8-row x 16-byte core
// matrices; adjacent core matrices along K 128 bytes apart, along M/N 1024 bytes
// apart); one thread issues four tcgen05.mma.cta_group::1.kind::f16 (K = 16 each) into
// an FP32 accumulator in tensor memory and commits them to the stage's mbarrier; the
// stage is refilled once that barrier completes, while the other stage's copies are in
// flight.  Every wait is bounded: one that runs out sets an error word and the kernel
// skips to the end, freeing its tensor memory.  The epilogue reads the accumulator with
// tcgen05.ld (each warp its 32 lanes = rows).
//
// For K <= 128 without a K split (every GEMM of the training step over the rows) a
// persistent warp-specialised form runs instead, one CTA of 320 threads per SM: B stays in
// shared memory, A is fetched a 128-row tile at a time by 2-D tensor copies
// (cp.async.bulk.tensor, boxes of 8 K-elements x 128 rows, no swizzle, rows beyond M read
// as zeros) three tiles ahead, two TMEM accumulators alternate, and the epilogue warps
// store through a shared-memory staging tile with coalesced 16-byte stores.  The weight
// gradients (one 128-row tile, K split over CTAs) take a tensor-copy split-K form.
#pragma once

#include <cstdint>

#include <cuda.h>
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
constexpr int GEMM_BK = 64;      // K per shared-memory stage (four MMAs of K = 16)
constexpr int GEMM_STAGES = 2;   // stages in flight: the next chunk loads while the MMAs run
constexpr int GEMM_THREADS = 128;
constexpr long long GEMM_WAIT_LIMIT = 1ll << 24;  // mbarrier polls before giving up

template <int N>
constexpr int gemm_smem_bytes()
{
    return GEMM_STAGES * (GEMM_BM + N) * GEMM_BK * 2 + 64 + 128;  // stages, barriers, alignment slack
}

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

// Start copying a [ROWS x GEMM_BK] BF16 chunk (row stride ld) into the canonical layout
// with asynchronous 16-byte copies: row r, element c -> ((r / 8) * 8 + c / 8) * 128 +
// (r % 8) * 16 + (c % 8) * 2 bytes.  Rows >= nrows and columns >= kend are zero-filled
// (a copy of 0 source bytes).
template <int ROWS>
__device__ __forceinline__ void stage_async(uint8_t *dst, const __nv_bfloat16 *src, int row0, int nrows, long long ld,
                                            int k0, int kend)
{
    constexpr int KV = GEMM_BK / 8;  // 16-byte vectors per row
    constexpr int VEC = ROWS * KV;
    for (int v = threadIdx.x; v < VEC; v += GEMM_THREADS) {
        const int r = v / KV, kb = v % KV;
        const int gr = row0 + r, gk = k0 + kb * 8;
        const bool in = gr < nrows && gk < kend;
        const __nv_bfloat16 *g = in ? src + (long long)gr * ld + gk : src;
        const uint32_t d = smem_u32(dst + ((r >> 3) * KV + kb) * 128 + (r & 7) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g), "r"(in ? 16 : 0) : "memory");
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

// D[M x N] = A[M x K] . B[N x K]^T for the 128-row tile blockIdx.x and the K range
// blockIdx.y, two shared-memory stages deep: while the tensor core works on chunk c,
// the asynchronous copies of chunk c + 1 are already in flight.
template <int N>
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm_bf16(const __nv_bfloat16 *__restrict__ A,
                                                           const __nv_bfloat16 *__restrict__ B, int M, int K,
                                                           int k_per_split, GemmEpi ep)
{
    static_assert(N == 32 || N == 64 || N == 128, "N tile");
    constexpr int TMEM_COLS = N < 32 ? 32 : N;
    constexpr int A_STAGE = GEMM_BM * GEMM_BK * 2, B_STAGE = N * GEMM_BK * 2;
    constexpr int SBO = (GEMM_BK / 8) * 128;  // 8-row group stride
    extern __shared__ uint8_t gemm_smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gemm_smem_raw) + 127) & ~uintptr_t(127));
    uint8_t *sa = sm, *sb = sm + GEMM_STAGES * A_STAGE;
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(sb + GEMM_STAGES * B_STAGE);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(mbar + GEMM_STAGES);
    int *s_fail = reinterpret_cast<int *>(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * GEMM_BM;
    const int kbeg = blockIdx.y * k_per_split, kend = min(K, kbeg + k_per_split);
    const int nchunks = kend > kbeg ? (kend - kbeg + GEMM_BK - 1) / GEMM_BK : 0;
    if (tid == 0) {
        *s_fail = 0;
        for (int st = 0; st < GEMM_STAGES; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[st])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // prologue: the first stages' copies
    for (int c = 0; c < GEMM_STAGES && c < nchunks; ++c) {
        const int k0 = kbeg + c * GEMM_BK;
        stage_async<GEMM_BM>(sa + c * A_STAGE, A, row0, M, K, k0, kend);
        stage_async<N>(sb + c * B_STAGE, B, 0, N, K, k0, kend);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    const uint32_t idesc = umma_idesc_bf16(GEMM_BM, N);
    uint32_t phase[GEMM_STAGES] = {0u, 0u};
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int st = c % GEMM_STAGES;
        // this thread's copies of chunk c have landed (the newer group may still fly)
        if (c + 1 < nchunks) asm volatile("cp.async.wait_group 1;" ::: "memory");
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int k16 = 0; k16 < GEMM_BK / 16; ++k16) {
                const uint64_t ad = umma_desc(smem_u32(sa + st * A_STAGE) + k16 * 256, 128, SBO);
                const uint64_t bd = umma_desc(smem_u32(sb + st * B_STAGE) + k16 * 256, 128, SBO);
                const uint32_t acc = (c > 0 || k16 > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[st]))
                         : "memory");
        }
        const int next = c + GEMM_STAGES;
        if (next < nchunks || c == nchunks - 1) {
            // the MMAs reading stage st must finish before it is refilled (or, for the
            // last chunk, before the accumulator is read)
            if (!mbar_wait(smem_u32(&mbar[st]), phase[st])) atomicExch(s_fail, 1);
            phase[st] ^= 1u;
            __syncthreads();
            if (*reinterpret_cast<volatile int *>(s_fail)) {
                ok = false;
                break;
            }
            if (next < nchunks) {
                const int k0 = kbeg + next * GEMM_BK;
                stage_async<GEMM_BM>(sa + st * A_STAGE, A, row0, M, K, k0, kend);
                stage_async<N>(sb + st * B_STAGE, B, 0, N, K, k0, kend);
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && nchunks > 0) {
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
                // a thread owns 32 consecutive values of its row: row-major reads and
                // writes go as 16-byte vectors; the transposed copy is coalesced across
                // the warp (its 32 rows are adjacent)
                const long long rbase = (long long)row * N + c0;
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    v[j] = __uint_as_float(r[j]);
                    if (ep.bias) v[j] += ep.bias[c0 + j];
                    if (ep.relu) v[j] = fmaxf(v[j], 0.0f);
                }
                if (ep.mask) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 mv = reinterpret_cast<const uint4 *>(ep.mask + rbase)[q];
                        const __nv_bfloat162 *mh = reinterpret_cast<const __nv_bfloat162 *>(&mv);
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const float2 m2 = __bfloat1622float2(mh[h]);
                            if (!(m2.x > 0.0f)) v[q * 8 + 2 * h] = 0.0f;
                            if (!(m2.y > 0.0f)) v[q * 8 + 2 * h + 1] = 0.0f;
                        }
                    }
                }
                if (ep.out_f32) {
                    if (ep.atomic_f32) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) atomicAdd(ep.out_f32 + rbase + j, v[j]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            reinterpret_cast<float4 *>(ep.out_f32 + rbase)[q] =
                                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                }
                if (ep.out_bf16) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t w[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            __nv_bfloat162 p2 = __floats2bfloat162_rn(v[q * 8 + 2 * h], v[q * 8 + 2 * h + 1]);
                            w[h] = *reinterpret_cast<uint32_t *>(&p2);
                        }
                        reinterpret_cast<uint4 *>(ep.out_bf16 + rbase)[q] = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
                if (ep.out_bf16_t) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        ep.out_bf16_t[(long long)(c0 + j) * ep.ldt + row] = __float2bfloat16_rn(v[j]);
                }
            }
        }
    }
    if (tid == 0 && *s_fail && ep.error) atomicExch(ep.error, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

constexpr int GEMM_T_KMAX = 128;   // K of the persistent form (B and the A tiles fit in shared memory)
constexpr int GEMM_T_ABUF = 3;     // A tiles in flight

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_expect_only(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Load rows [row0, row0 + ROWS) x K of a K-contiguous matrix as KP / 8 boxes of
// 8 elements x ROWS rows; box j lands at dst + j * ROWS * 16.  ARRIVE: this thread's
// arrival on the barrier comes with the expected bytes (else they are only added).
template <int ROWS, bool ARRIVE>
__device__ __forceinline__ void tma_tile(uint32_t dst, const CUtensorMap *map, int row0, int KP, uint32_t mbar)
{
    if (ARRIVE) mbar_expect(mbar, (uint32_t)(KP / 8) * ROWS * 16);
    else mbar_expect_only(mbar, (uint32_t)(KP / 8) * ROWS * 16);
    for (int j = 0; j < KP / 8; ++j) tma_load_2d(dst + j * ROWS * 16, map, 8 * j, row0, mbar);
}

// The persistent form (K <= GEMM_T_KMAX, no K split): every training GEMM over the
// rows.  Warp 0 (one lane) issues the tensor copies of B once and of the A tiles
// GEMM_T_ABUF deep; warp 1 (one lane) issues each tile's MMAs into one of two TMEM
// accumulators; warps 2..9 drain an accumulator (each its 32 TMEM lanes and half the
// columns), release it to the MMA warp and stage the bf16 results in shared memory
// (row-major with the 16-byte chunks of a row XOR-permuted, and transposed), from where
// both outputs leave as coalesced 16-byte stores.  So the MMAs of tile i + 1 and the
// copies of the tiles after it run while tile i is stored.  mbarriers: full/empty per A
// buffer (copy -> MMA -> copy), tfull/tempty per accumulator (MMA -> epilogue -> MMA);
// every wait is bounded, and the epilogue warps decide together (after a named barrier)
// whether to stop.
constexpr int GEMM_WS_EPI_WARPS = 8;
constexpr int GEMM_WS_THREADS = 64 + 32 * GEMM_WS_EPI_WARPS;

template <int N>
constexpr int gemm_ws_smem_bytes()
{
    return N * GEMM_T_KMAX * 2 + GEMM_T_ABUF * GEMM_BM * GEMM_T_KMAX * 2 + GEMM_BM * N * 2 * 2 + 256 + 1024;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void epi_bar()
{
    asm volatile("bar.sync 1, %0;" ::"r"(32 * GEMM_WS_EPI_WARPS) : "memory");
}

template <int N>
__global__ void __launch_bounds__(GEMM_WS_THREADS, 1) k_gemm_bf16_ws(const __grid_constant__ CUtensorMap tmA,
                                                                   const __grid_constant__ CUtensorMap tmB, int M,
                                                                   int K, GemmEpi ep)
{
    constexpr int ACC = N < 32 ? 32 : N;  // TMEM columns of one accumulator
    constexpr int TMEM_COLS = 2 * ACC;
    constexpr int A_BUF = GEMM_BM * GEMM_T_KMAX * 2;
    constexpr int NB = GEMM_T_ABUF;
    extern __shared__ uint8_t gemm_smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gemm_smem_raw) + 1023) & ~uintptr_t(1023));
    const int KP = (K + 15) / 16 * 16;
    uint8_t *sb = sm;
    uint8_t *sa = sb + N * GEMM_T_KMAX * 2;
    uint8_t *ss = sa + NB * A_BUF;
    uint8_t *st = ss + GEMM_BM * N * 2;
    unsigned long long *full = reinterpret_cast<unsigned long long *>(st + GEMM_BM * N * 2);
    unsigned long long *empty = full + NB, *tfull = empty + NB, *tempty = tfull + 2, *bfull = tempty + 2;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bfull + 1);
    int *s_fail = reinterpret_cast<int *>(s_tmem + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (M + GEMM_BM - 1) / GEMM_BM;
    if (tid == 0) {
        *s_fail = 0;
        for (int q = 0; q < NB; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[q])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[q])) : "memory");
        }
        for (int q = 0; q < 2; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull[q])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tempty[q])),
                         "r"(GEMM_WS_EPI_WARPS)
                         : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bfull)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    volatile int *vfail = s_fail;

    if (warp == 0) {
        if (lane == 0 && (int)blockIdx.x < ntiles) {
            tma_tile<N, true>(smem_u32(sb), &tmB, 0, KP, smem_u32(bfull));
            int issued = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++issued) {
                const int b = issued % NB;
                if (issued >= NB && !mbar_wait(smem_u32(&empty[b]), (uint32_t)((issued / NB - 1) & 1))) {
                    *vfail = 1;
                    break;
                }
                if (*vfail) break;
                tma_tile<GEMM_BM, true>(smem_u32(sa + b * A_BUF), &tmA, t * GEMM_BM, KP, smem_u32(&full[b]));
            }
            // copies still in flight must land before the shared memory is released (only
            // after a failure can one be unconsumed)
            mbar_wait(smem_u32(bfull), 0u);
            for (int q = issued - NB < 0 ? 0 : issued - NB; q < issued; ++q)
                mbar_wait(smem_u32(&full[q % NB]), (uint32_t)((q / NB) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0 && (int)blockIdx.x < ntiles) {
            const uint32_t idesc = umma_idesc_bf16(GEMM_BM, N);
            bool ok = mbar_wait(smem_u32(bfull), 0u);
            int i = 0;
            for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++i) {
                const int b = i % NB, acc = i & 1;
                ok = mbar_wait(smem_u32(&full[b]), (uint32_t)((i / NB) & 1));
                if (ok && i >= 2) ok = mbar_wait(smem_u32(&tempty[acc]), (uint32_t)((i / 2 - 1) & 1));
                if (!ok || *vfail) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(sa + b * A_BUF), b0 = smem_u32(sb);
                const uint32_t d = tmem + (uint32_t)(acc * ACC);
                for (int k16 = 0; k16 < KP / 16; ++k16) {
                    const uint64_t ad = umma_desc(a0 + k16 * 2 * GEMM_BM * 16, GEMM_BM * 16, 128);
                    const uint64_t bd = umma_desc(b0 + k16 * 2 * N * 16, N * 16, 128);
                    const uint32_t accum = k16 > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                        : "memory");
                }
                // both barriers track these MMAs: the A buffer and the accumulator
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty[b]))
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&tfull[acc]))
                             : "memory");
            }
            if (!ok) *vfail = 1;
        }
    } else {
        const int e = tid - 64;  // epilogue thread 0 .. 255
        const int lg = warp & 3, half = (warp - 2) >> 2;
        const int rl = lg * 32 + lane;  // row within the tile
        constexpr int CH = N >= 64 ? N / 2 : N;  // columns per warp
        const bool active = N >= 64 || half == 0;
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int acc = i & 1;
            if (lane == 0 && !mbar_wait(smem_u32(&tfull[acc]), (uint32_t)((i / 2) & 1))) *vfail = 1;
            epi_bar();
            if (*vfail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = t * GEMM_BM + rl;
            const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(acc * ACC);
            if (active) {
#pragma unroll
                for (int cc = 0; cc < CH; cc += 32) {
                    const int c0 = half * CH + cc;
                    uint32_t r[32];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                        : "r"(taddr + (uint32_t)c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    float v[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        v[j] = __uint_as_float(r[j]);
                        if (ep.bias) v[j] += __ldg(ep.bias + c0 + j);
                        if (ep.relu) v[j] = fmaxf(v[j], 0.0f);
                    }
                    const long long rbase = (long long)row * N + c0;
                    if (ep.mask && row < M) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint4 mv = reinterpret_cast<const uint4 *>(ep.mask + rbase)[q];
                            const __nv_bfloat162 *mh = reinterpret_cast<const __nv_bfloat162 *>(&mv);
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const float2 m2 = __bfloat1622float2(mh[h]);
                                if (!(m2.x > 0.0f)) v[q * 8 + 2 * h] = 0.0f;
                                if (!(m2.y > 0.0f)) v[q * 8 + 2 * h + 1] = 0.0f;
                            }
                        }
                    }
                    if (ep.out_f32 && row < M) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            reinterpret_cast<float4 *>(ep.out_f32 + rbase)[q] =
                                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                    if (ep.out_bf16) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            uint32_t w[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                __nv_bfloat162 p2 = __floats2bfloat162_rn(v[q * 8 + 2 * h], v[q * 8 + 2 * h + 1]);
                                w[h] = *reinterpret_cast<uint32_t *>(&p2);
                            }
                            const int chunk = (c0 / 8 + q) ^ (rl & (N * 2 / 16 - 1));
                            *reinterpret_cast<uint4 *>(ss + rl * (N * 2) + chunk * 16) =
                                make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
                    if (ep.out_bf16_t) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            *reinterpret_cast<__nv_bfloat16 *>(st + (c0 + j) * (GEMM_BM * 2) + rl * 2) =
                                __float2bfloat16_rn(v[j]);
                    }
                }
            }
            // the accumulator is in registers and shared memory: hand it back to the MMA warp
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
            epi_bar();
            const int row0 = t * GEMM_BM;
            if (ep.out_bf16) {
                constexpr int CPR = N * 2 / 16;  // 16-byte chunks per row
                for (int id = e; id < GEMM_BM * CPR; id += 32 * GEMM_WS_EPI_WARPS) {
                    const int rr = id / CPR, q = id % CPR;
                    if (row0 + rr < M) {
                        const uint4 val = *reinterpret_cast<const uint4 *>(ss + rr * (N * 2) + (q ^ (rr & (CPR - 1))) * 16);
                        *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(ep.out_bf16) + ((long long)(row0 + rr) * N) * 2 +
                                                   q * 16) = val;
                    }
                }
            }
            if (ep.out_bf16_t) {
                const bool whole = row0 + GEMM_BM <= M && (ep.ldt % 8) == 0;
                for (int id = e; id < N * (GEMM_BM / 8); id += 32 * GEMM_WS_EPI_WARPS) {
                    const int c = id / (GEMM_BM / 8), q = id % (GEMM_BM / 8);
                    const uint8_t *srcp = st + c * (GEMM_BM * 2) + q * 16;
                    __nv_bfloat16 *dst = ep.out_bf16_t + (long long)c * ep.ldt + row0 + q * 8;
                    if (whole) {
                        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(srcp);
                    } else {
                        for (int x = 0; x < 8; ++x)
                            if (row0 + q * 8 + x < M) dst[x] = reinterpret_cast<const __nv_bfloat16 *>(srcp)[x];
                    }
                }
            }
            epi_bar();  // the staging tiles are free for the next tile
        }
    }
    __syncthreads();
    if (tid == 0 && *vfail && ep.error) atomicExch(ep.error, 1);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Split-K form for the weight gradients (M <= 128 rows, K = the training rows split in
// k_per_split slices over blockIdx.y): 64-wide K chunks of A (128 x 64) and B (N x 64)
// arrive by tensor copies in GEMM_SK_STAGES stages; thread 0 issues copies and MMAs, and
// refills a stage once its MMAs have completed, so GEMM_SK_STAGES - 1 chunks are always in
// flight.  The epilogue adds the FP32 partial tile into out_f32 with vector reductions.
constexpr int GEMM_SK_STAGES = 4;

template <int N>
constexpr int gemm_sk_smem_bytes()
{
    return GEMM_SK_STAGES * (GEMM_BM + N) * GEMM_BK * 2 + 128 + 1024;
}

template <int N>
__global__ void __launch_bounds__(GEMM_THREADS, 1) k_gemm_bf16_splitk(const __grid_constant__ CUtensorMap tmA,
                                                                     const __grid_constant__ CUtensorMap tmB, int M,
                                                                     int K, int k_per_split, GemmEpi ep)
{
    constexpr int TMEM_COLS = N < 32 ? 32 : N;
    constexpr int A_ST = GEMM_BM * GEMM_BK * 2, B_ST = N * GEMM_BK * 2;
    extern __shared__ uint8_t gemm_smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gemm_smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sa = sm, *sb = sm + GEMM_SK_STAGES * A_ST;
    unsigned long long *full = reinterpret_cast<unsigned long long *>(sb + GEMM_SK_STAGES * B_ST);
    unsigned long long *done = full + GEMM_SK_STAGES;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(done + GEMM_SK_STAGES);
    int *s_fail = reinterpret_cast<int *>(s_tmem + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kbeg = blockIdx.y * k_per_split, kend = min(K, kbeg + k_per_split);
    const int nchunks = kend > kbeg ? (kend - kbeg + GEMM_BK - 1) / GEMM_BK : 0;
    if (tid == 0) {
        *s_fail = 0;
        for (int q = 0; q < 2 * GEMM_SK_STAGES; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[q])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    if (tid == 0) {
        const uint32_t idesc = umma_idesc_bf16(GEMM_BM, N);
        constexpr uint32_t BYTES = (uint32_t)(A_ST + B_ST);
        int issued = 0;
        auto issue = [&](int c) {
            const int st = c % GEMM_SK_STAGES, k0 = kbeg + c * GEMM_BK;
            const uint32_t mb = smem_u32(&full[st]);
            mbar_expect(mb, BYTES);
            for (int j = 0; j < GEMM_BK / 8; ++j) {
                tma_load_2d(smem_u32(sa + st * A_ST) + j * GEMM_BM * 16, &tmA, k0 + 8 * j, 0, mb);
                tma_load_2d(smem_u32(sb + st * B_ST) + j * N * 16, &tmB, k0 + 8 * j, 0, mb);
            }
            ++issued;
        };
        for (int c = 0; c < GEMM_SK_STAGES && c < nchunks; ++c) issue(c);
        bool ok = true;
        int c = 0;
        for (; c < nchunks && ok; ++c) {
            const int st = c % GEMM_SK_STAGES;
            const uint32_t par = (uint32_t)((c / GEMM_SK_STAGES) & 1);
            ok = mbar_wait(smem_u32(&full[st]), par);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int k16 = 0; k16 < GEMM_BK / 16; ++k16) {
                const uint64_t ad = umma_desc(smem_u32(sa + st * A_ST) + k16 * 2 * GEMM_BM * 16, GEMM_BM * 16, 128);
                const uint64_t bd = umma_desc(smem_u32(sb + st * B_ST) + k16 * 2 * N * 16, N * 16, 128);
                const uint32_t acc = (c > 0 || k16 > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&done[st]))
                         : "memory");
            if (c + GEMM_SK_STAGES < nchunks || c == nchunks - 1) {
                // the stage's MMAs must finish before it is refilled (or, after the last
                // chunk, before the accumulator is read)
                ok = mbar_wait(smem_u32(&done[st]), par);
                if (ok && c + GEMM_SK_STAGES < nchunks) issue(c + GEMM_SK_STAGES);
            }
        }
        if (!ok) {
            *s_fail = 1;
            // loads issued but not consumed must land before the shared memory is released
            for (int q = c; q < issued; ++q)
                mbar_wait(smem_u32(&full[q % GEMM_SK_STAGES]), (uint32_t)((q / GEMM_SK_STAGES) & 1));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!*reinterpret_cast<volatile int *>(s_fail) && nchunks > 0) {
        const int row = warp * 32 + lane;
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
                // 16-byte vector reductions (out_f32 is 16-byte aligned, N a multiple of 32)
                float *dst = ep.out_f32 + (long long)row * N + c0;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4 * q),
                                 "f"(__uint_as_float(r[4 * q])), "f"(__uint_as_float(r[4 * q + 1])),
                                 "f"(__uint_as_float(r[4 * q + 2])), "f"(__uint_as_float(r[4 * q + 3]))
                                 : "memory");
            }
        }
    }
    if (tid == 0 && *s_fail && ep.error) atomicExch(ep.error, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace qmcrt

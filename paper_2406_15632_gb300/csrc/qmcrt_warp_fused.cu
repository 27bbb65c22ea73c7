// qmcrt_warp_fused.cu -- forward pass of the learned warp, one fused tensor-core
// kernel per conditional.
//
// A CTA keeps the four weight matrices of one MLP resident in shared memory (104 KB,
// canonical K-major layout without swizzle) and runs three row groups of 128 threads
// (4 warps each) that take 128-row tiles in turn.  Per tile a group writes the one-blob
// features of its rows straight into its shared-memory activation tile, then for each
// layer one elected thread issues the tcgen05.mma chain (M = 128, N = 128 or 32, K in
// steps of 16) into the group's 128 TMEM columns and commits it to the group's
// mbarrier; every thread reads its own row of the accumulator back with tcgen05.ld,
// adds the bias, applies the ReLU and writes the bf16 row into the activation tile for
// the next layer.  After the last layer each thread turns its 32 logits into the
// conditional (softmax, uniform mixture) and samples its coordinate.  Only u, x and
// log |dx/du| touch global memory.  The groups interleave: their epilogues run while
// the tensor core works on another group's layer (three groups, 200 KB of shared memory
// and 384 of the 512 TMEM columns: 1.29x the throughput of two).
//
// The arithmetic is the layer-by-layer path's (same bf16 roundings, same FP32 bias and
// ReLU, same sampling functions); the feature columns that are identically zero are
// skipped in the first layer, which adds nothing to the accumulators.
#include <algorithm>

#include "qmcrt.h"
#include "qmcrt_flow.cuh"
#include "qmcrt_gemm.cuh"
#include "qmcrt_internal.h"

namespace qmcrt {
namespace {

using namespace flow;

constexpr int FG = 3;                                 // row groups per CTA
constexpr int FT = 128 * FG;                          // threads per CTA
constexpr int TMEM_ALLOC = FG * 128 <= 256 ? 256 : 512;  // a power of two >= the groups' columns
constexpr int W_LAYER = WD * WD * 2;                  // bytes of a 128 x 128 bf16 layer
constexpr int W_BYTES = 3 * W_LAYER + KB * WD * 2;    // the four layers of one MLP
constexpr int A_BYTES = 128 * WD * 2;                 // one activation tile
constexpr int SBO = (WD / 8) * 128;                   // 8-row group stride (K = 128)
constexpr int N_BIAS = 3 * WD + KB;
constexpr int SMEM_BYTES = W_BYTES + FG * A_BYTES + N_BIAS * 4 + KB * 4 + FG * 8 + 4 + FG * 4 + 1024;

// Byte offset of element (r, k) of a [rows x 128] bf16 tile in the canonical K-major
// layout: 8 x 16-byte core matrices, K-adjacent ones 128 bytes apart, 8-row groups
// SBO bytes apart.
__device__ __forceinline__ uint32_t canon(int r, int k)
{
    return (uint32_t)((((r >> 3) * (WD / 8) + (k >> 3)) * 128) + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void group_bar(int id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(128) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);  // a in the low half (lower address)
    return *reinterpret_cast<uint32_t *>(&p);
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Conditional MI (0: x1 from MLP0(one-blob x0), sampling x0 first; 1: x2 from
// MLP1(one-blob x0, one-blob x1)) for rows [0, n).
template <int MI>
__global__ void __launch_bounds__(FT, 1) k_warp_fused(const float *__restrict__ params,
                                                     const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ u,
                                                     float *__restrict__ x, float *__restrict__ logj, int n, float mix,
                                                     int *__restrict__ error)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sW = sm;
    uint8_t *sA0 = sm + W_BYTES;
    float *sBias = reinterpret_cast<float *>(sA0 + FG * A_BYTES);
    float *sQ0 = sBias + N_BIAS;  // the x0 bin masses (MI 0), the same for every row
    unsigned long long *sBar = reinterpret_cast<unsigned long long *>(sQ0 + KB);
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(sBar + FG);
    int *sFail = reinterpret_cast<int *>(sTmem + 1);  // one flag per group, written by that group only

    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid >> 7, t = tid & 127;
    constexpr int K_IN = MI == 0 ? BLOB : 2 * BLOB;  // nonzero feature columns

    // weights of MLP MI: bf16 [out][in] row-major -> canonical K-major
    for (int l = 0; l < 4; ++l) {
        const __nv_bfloat16 *src = wb + bf_w(MI, l);
        uint8_t *dst = sW + l * W_LAYER;
        for (int v = tid; v < out_dim(l) * (WD / 8); v += FT) {
            const int r = v / (WD / 8), kb = v % (WD / 8);
            *reinterpret_cast<uint4 *>(dst + canon(r, kb * 8)) =
                *reinterpret_cast<const uint4 *>(src + (long long)r * WD + kb * 8);
        }
    }
    for (int i = tid; i < N_BIAS; i += FT) {
        const int l = i < 3 * WD ? i / WD : 3, o = i < 3 * WD ? i % WD : i - 3 * WD;
        sBias[i] = params[param_b(MI, l) + o];
    }
    if (MI == 0 && tid == 0) {
        float z[KB], q[KB];
        for (int k = 0; k < KB; ++k) z[k] = params[k];
        softmax32(z, q);
        if (mix != 0.0f)
            for (int k = 0; k < KB; ++k) q[k] = mixed(q[k], mix);
        for (int k = 0; k < KB; ++k) sQ0[k] = q[k];
    }
    if (tid == 0) {
        for (int k = 0; k < FG; ++k) sFail[k] = 0;
        for (int k = 0; k < FG; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sBar[k])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                     "r"(TMEM_ALLOC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const uint32_t tmem = *sTmem + (uint32_t)(g * 128);                  // this group's columns
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's 32 lanes
    uint8_t *sA = sA0 + g * A_BYTES;
    const uint32_t bar = smem_u32(&sBar[g]);
    uint32_t phase = 0;
    const int tiles = (n + 127) / 128;
    bool ok = true;

    for (int tile = blockIdx.x * FG + g; ok && tile < tiles; tile += gridDim.x * FG) {
        const long long j = (long long)tile * 128 + t;
        const bool live = j < n;
        float x0, x1 = 0.5f, lj;
        if (MI == 0) {
            float q[KB], lq;
#pragma unroll
            for (int k = 0; k < KB; ++k) q[k] = sQ0[k];
            sample_bin(q, live ? u[3 * j] : 0.5f, x0, lq);
            lj = -lq;
        } else {
            x0 = live ? x[3 * j] : 0.5f;
            x1 = live ? x[3 * j + 1] : 0.5f;
            lj = live ? logj[j] : 0.0f;
        }
        // one-blob features of this row (columns >= K_IN are never read)
#pragma unroll
        for (int kb = 0; kb < K_IN / 8; ++kb) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int f = kb * 8 + 2 * h;
                const float v0 = f < BLOB ? blob(x0, f) : blob(x1, f - BLOB);
                const float v1 = f + 1 < BLOB ? blob(x0, f + 1) : blob(x1, f + 1 - BLOB);
                w[h] = pack_bf16(v0, v1);
            }
            *reinterpret_cast<uint4 *>(sA + canon(t, kb * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
        }

        for (int l = 0; l < 4; ++l) {
            const int N = out_dim(l);
            const int KS = (l == 0 ? K_IN : WD) / 16;
            // the activation tile written by every thread is visible to the tensor core,
            // and the previous layer's accumulator reads are complete
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            group_bar(1 + g);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (t == 0) {
                const uint32_t idesc = umma_idesc_bf16(128, N);
                const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sW + l * W_LAYER);
                for (int s = 0; s < KS; ++s) {
                    const uint64_t ad = umma_desc(a0 + s * 256, 128, SBO);
                    const uint64_t bd = umma_desc(b0 + s * 256, 128, SBO);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(s > 0 ? 1u : 0u)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                             : "memory");
            }
            const bool got = mbar_wait(bar, phase);
            phase ^= 1u;
            if (!got) atomicExch(&sFail[g], 1);
            group_bar(1 + g);
            if (*reinterpret_cast<volatile int *>(&sFail[g])) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (l < 3) {
                const float *bias = sBias + l * WD;
#pragma unroll 1
                for (int c0 = 0; c0 < WD; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(lane_addr + (uint32_t)c0, r);
#pragma unroll
                    for (int q8 = 0; q8 < 4; ++q8) {
                        uint32_t w[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int c = q8 * 8 + 2 * h;
                            const float v0 = fmaxf(__uint_as_float(r[c]) + bias[c0 + c], 0.0f);
                            const float v1 = fmaxf(__uint_as_float(r[c + 1]) + bias[c0 + c + 1], 0.0f);
                            w[h] = pack_bf16(v0, v1);
                        }
                        *reinterpret_cast<uint4 *>(sA + canon(t, c0 + q8 * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
            } else {
                uint32_t r[32];
                tmem_ld32(lane_addr, r);
                float z[KB], q[KB], xv, lq;
#pragma unroll
                for (int k = 0; k < KB; ++k) z[k] = __uint_as_float(r[k]) + sBias[3 * WD + k];
                softmax32(z, q);
                if (mix != 0.0f) {
#pragma unroll
                    for (int k = 0; k < KB; ++k) q[k] = mixed(q[k], mix);
                }
                sample_bin(q, live ? u[3 * j + 1 + MI] : 0.5f, xv, lq);
                if (live) {
                    if (MI == 0) x[3 * j] = x0;
                    x[3 * j + 1 + MI] = xv;
                    logj[j] = lj - lq;
                }
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && error) {
        int f = 0;
        for (int k = 0; k < FG; ++k) f |= sFail[k];
        if (f) atomicExch(error, 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*sTmem), "r"(TMEM_ALLOC)
                     : "memory");
    }
}

template <int MI>
cudaError_t launch_one(const float *params, const __nv_bfloat16 *wb, const float *u, float *x, float *logj, int n,
                       float mix, int *error, int ctas, cudaStream_t s)
{
    static cudaError_t attr = cudaFuncSetAttribute(k_warp_fused<MI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   SMEM_BYTES);
    if (attr != cudaSuccess) return attr;
    k_warp_fused<MI><<<ctas, FT, SMEM_BYTES, s>>>(params, wb, u, x, logj, n, mix, error);
    return cudaGetLastError();
}

}  // namespace

// x[n][3], logj[n] = T(u), log |dx/du| with both conditionals fused on the tensor cores.
cudaError_t launch_warp_forward_fused(const float *params, const __nv_bfloat16 *wb, const float *u, float *x,
                                      float *logj, long long n, float mix, int *error, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // rows beyond 2^31 - 128 go in further launches
    for (long long base = 0; base < n; base += (1ll << 30)) {
        const int cnt = (int)std::min<long long>(n - base, 1ll << 30);
        const long long tiles = (cnt + 127) / 128;
        const int ctas = (int)std::max(1ll, std::min<long long>((tiles + FG - 1) / FG, sms));
        if ((e = launch_one<0>(params, wb, u + 3 * base, x + 3 * base, logj + base, cnt, mix, error, ctas, s)))
            return e;
        if ((e = launch_one<1>(params, wb, u + 3 * base, x + 3 * base, logj + base, cnt, mix, error, ctas, s)))
            return e;
    }
    return cudaSuccess;
}

}  // namespace qmcrt

// qmcrt_flow.cuh -- pieces of the learned warp shared by the layer-by-layer kernels
// (training) and the fused forward kernel: parameter layout, one-blob features,
// softmax with the uniform mixture, and the piecewise-linear inverse CDF.  Both paths
// call these same functions, so they sample identically.
#pragma once

#include <cuda_bf16.h>

#include "qmcrt.h"

namespace qmcrt {
namespace flow {

constexpr int KB = QMCRT_WARP_BINS;
constexpr int WD = QMCRT_WARP_WIDTH;
constexpr int BLOB = 32;

__host__ __device__ constexpr int out_dim(int l) { return l == 3 ? KB : WD; }
__host__ __device__ constexpr int mlp_params() { return 3 * (WD * WD + WD) + (KB * WD + KB); }
__host__ __device__ inline int param_w(int m, int l)
{
    int o = KB + m * mlp_params();
    for (int j = 0; j < l; ++j) o += out_dim(j) * WD + out_dim(j);
    return o;
}
__host__ __device__ inline int param_b(int m, int l) { return param_w(m, l) + out_dim(l) * WD; }
__host__ __device__ inline int bf_w(int m, int l)
{
    int o = m * (3 * WD * WD + KB * WD);
    for (int j = 0; j < l; ++j) o += out_dim(j) * WD;
    return o;
}
static_assert(KB + 2 * mlp_params() == QMCRT_WARP_PARAMS, "parameter count");
static_assert(2 * (3 * WD * WD + KB * WD) == QMCRT_WARP_BF16_WEIGHTS, "weight count");

// One-blob feature k of v: a Gaussian bump (sigma = one bin) at the centre of bin k.
__device__ __forceinline__ float blob(float v, int k)
{
    const float d = (v - (k + 0.5f) / BLOB) * BLOB;
    return __expf(-0.5f * d * d);
}

__device__ __forceinline__ void softmax32(const float *z, float *q)
{
    float mx = z[0];
#pragma unroll
    for (int k = 1; k < KB; ++k) mx = fmaxf(mx, z[k]);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        q[k] = expf(z[k] - mx);
        s += q[k];
    }
    const float inv = 1.0f / s;
#pragma unroll
    for (int k = 0; k < KB; ++k) q[k] *= inv;
}

// Defensive mixture with the uniform density: Q = (1 - mix) softmax + mix / 32, so
// 32 Q >= mix and |dx/du| = 1 / q(x) <= mix^-3.
__device__ __forceinline__ float mixed(float s, float mix) { return (1.0f - mix) * s + mix * (1.0f / KB); }

// x = F^-1(uu) for the piecewise-constant pdf 32 q[b] on 32 equal bins, and
// lq = log(32 q[b]) of the bin it falls in (log |dx/du| = -lq).  The bin search is
// unrolled with selects so that q stays in registers.
__device__ __forceinline__ void sample_bin(const float *q, float uu, float &xv, float &lq)
{
    float c = 0.0f, cb = 0.0f, qb = q[KB - 1];
    int b = KB - 1;
    bool found = false;
#pragma unroll
    for (int k = 0; k < KB - 1; ++k) {
        const bool hit = !found && uu < c + q[k];
        b = hit ? k : b;
        qb = hit ? q[k] : qb;
        cb = hit ? c : cb;
        found = found || hit;
        c += q[k];
    }
    if (!found) cb = c;
    xv = fminf(fmaxf((b + (uu - cb) / qb) / KB, 0.0f), 1.0f);
    lq = logf(KB * qb);
}

}  // namespace flow
}  // namespace qmcrt

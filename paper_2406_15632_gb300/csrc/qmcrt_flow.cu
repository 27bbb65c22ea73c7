// qmcrt_flow.cu -- the learned proposal: a piecewise-linear autoregressive warp of the
// first-scattering coordinates with two 4-layer MLP conditionals, its cross-entropy
// gradient and Adam.  Dense layers run on the tensor cores (qmcrt_gemm.cuh); the
// kernels here are the element-wise parts.  Every GEMM operand is produced by the
// previous step already in the K-major form the tensor cores read (activations and
// backward signals are written both as is and transposed), so no transposed
// descriptor is needed:
//   forward   H[l+1] = relu(H[l] . W[l]^T + b[l])         A = H[l],     B = W[l]
//   backward  dH[l]  = (dP[l] . W[l]) * (H[l] > 0)        A = dP[l],    B = W[l]^T
//             dW[l]  = dP[l]^T . H[l]                      A = dP[l]^T, B = H[l]^T (K = rows)
#include <cmath>
#include <cstring>

#include "qmcrt.h"
#include "qmcrt_flow.cuh"
#include "qmcrt_gemm.cuh"
#include "qmcrt_internal.h"

namespace qmcrt {
namespace {

using namespace flow;
constexpr int ROW_BYTES = 3328;  // workspace bytes per row (see carve)


struct Work {
    __nv_bfloat16 *F, *Ft, *H[3], *Ht[3], *dL, *dLt, *dP[2], *dPt[2];
    float *L;
    double *wsum;
    int rows;
};

uint64_t round128(uint64_t r) { return (r + 127) & ~127ull; }

Work carve(void *ws, int rows)
{
    Work w;
    char *p = (char *)ws;
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 255) & ~(size_t)255;
        return q;
    };
    w.rows = rows;
    w.wsum = (double *)take(256);
    w.F = (__nv_bfloat16 *)take((size_t)rows * WD * 2);
    w.Ft = (__nv_bfloat16 *)take((size_t)rows * WD * 2);
    for (int i = 0; i < 3; ++i) {
        w.H[i] = (__nv_bfloat16 *)take((size_t)rows * WD * 2);
        w.Ht[i] = (__nv_bfloat16 *)take((size_t)rows * WD * 2);
    }
    w.L = (float *)take((size_t)rows * KB * 4);
    w.dL = (__nv_bfloat16 *)take((size_t)rows * KB * 2);
    w.dLt = (__nv_bfloat16 *)take((size_t)rows * KB * 2);
    for (int i = 0; i < 2; ++i) {
        w.dP[i] = (__nv_bfloat16 *)take((size_t)rows * WD * 2);
        w.dPt[i] = (__nv_bfloat16 *)take((size_t)rows * WD * 2);
    }
    return w;
}

uint64_t bytes_for(uint64_t rows) { return (uint64_t)ROW_BYTES * rows + 8192; }

int rows_for(uint64_t ws_bytes)
{
    if (ws_bytes < bytes_for(128)) return 0;
    uint64_t r = (ws_bytes - 8192) / ROW_BYTES;
    r &= ~127ull;
    return (int)std::min<uint64_t>(r, 1u << 22);
}


// Input features of MLP m for rows [0, rows): one-blob(x0) [, one-blob(x1)], zero padded;
// rows >= n use x = 0.5 (their loss weight is zero).  One block per 32 rows: each thread
// writes 16 features of one row as two 16-byte vectors, and the transposed copy leaves
// through a shared-memory tile, 16 rows of one feature per thread.
constexpr int FEAT_ROWS = 32;
__global__ void __launch_bounds__(256) k_features(const float *__restrict__ x, int n, int rows, int m,
                                                 __nv_bfloat16 *__restrict__ F, __nv_bfloat16 *__restrict__ Ft)
{
    __shared__ __nv_bfloat16 tile[WD][FEAT_ROWS + 8];
    const int t = threadIdx.x;
    const int r = t >> 3, c = t & 7;  // row in the tile, 16-feature chunk
    const int j = blockIdx.x * FEAT_ROWS + r;
    const float x0 = j < n ? x[3ll * j] : 0.5f, x1 = j < n ? x[3ll * j + 1] : 0.5f;
    uint32_t w[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        float v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int f = c * 16 + 2 * h + e;
            v[e] = 0.0f;
            if (f < BLOB) v[e] = blob(x0, f);
            else if (m == 1 && f < 2 * BLOB) v[e] = blob(x1, f - BLOB);
        }
        __nv_bfloat162 p2 = __floats2bfloat162_rn(v[0], v[1]);
        w[h] = *reinterpret_cast<uint32_t *>(&p2);
        tile[c * 16 + 2 * h][r] = p2.x;
        tile[c * 16 + 2 * h + 1][r] = p2.y;
    }
    uint4 *dst = reinterpret_cast<uint4 *>(F + (long long)j * WD + c * 16);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    if (!Ft) return;
    __syncthreads();
    const int f = t >> 1, half = t & 1;  // feature, which 16 rows of the tile
    const uint4 *srcv = reinterpret_cast<const uint4 *>(&tile[f][half * 16]);
    uint4 *dt = reinterpret_cast<uint4 *>(Ft + (long long)f * rows + blockIdx.x * FEAT_ROWS + half * 16);
    dt[0] = srcv[0];
    dt[1] = srcv[1];
}

// Sampling step of coordinate `layer`: x_l = F^-1(u_l) for the pdf 32 Q[b] on bin b;
// log |dx/du| accumulates -log(32 Q[b]).
__global__ void k_sample(int layer, const float *__restrict__ theta0, const float *__restrict__ L,
                         const float *__restrict__ u, float *__restrict__ x, float *__restrict__ logj, int n,
                         float mix)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float z[KB], q[KB];
    const float *src = layer == 0 ? theta0 : L + (long long)j * KB;
    for (int k = 0; k < KB; ++k) z[k] = src[k];
    softmax32(z, q);
    if (mix != 0.0f)
        for (int k = 0; k < KB; ++k) q[k] = mixed(q[k], mix);
    float xv, lq;
    sample_bin(q, u[3ll * j + layer], xv, lq);
    x[3ll * j + layer] = xv;
    logj[j] = layer == 0 ? -lq : logj[j] - lq;
}

__global__ void k_wsum(const float *__restrict__ w, int n, double *out)
{
    double s = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) s += w[j];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Loss and d loss / d logits of coordinate `layer` (0: theta0; 1, 2: MLP0, MLP1 logits
// in L) for rows [0, rows); rows >= n have weight zero.
__global__ void k_loss_grad(int layer, const float *__restrict__ theta0, const float *__restrict__ L,
                            const float *__restrict__ x, const float *__restrict__ w, int n, int rows,
                            const double *__restrict__ wsum, float *__restrict__ loss, float *__restrict__ dtheta,
                            __nv_bfloat16 *__restrict__ dL, __nv_bfloat16 *__restrict__ dLt, float mix)
{
    __shared__ float s_dt[KB];
    __shared__ float s_loss;
    if (threadIdx.x < KB) s_dt[threadIdx.x] = 0.0f;
    if (threadIdx.x == 0) s_loss = 0.0f;
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < rows) {
        const float ww = j < n ? (float)(w[j] / *wsum) : 0.0f;
        float z[KB], q[KB];
        if (layer == 0) {
            for (int k = 0; k < KB; ++k) z[k] = theta0[k];
        } else {
            const float4 *src = reinterpret_cast<const float4 *>(L + (long long)j * KB);
#pragma unroll
            for (int v = 0; v < KB / 4; ++v) {
                const float4 f4 = src[v];
                z[4 * v] = f4.x;
                z[4 * v + 1] = f4.y;
                z[4 * v + 2] = f4.z;
                z[4 * v + 3] = f4.w;
            }
        }
        softmax32(z, q);
        const float xv = j < n ? x[3ll * j + layer] : 0.5f;
        const int b = min((int)(xv * KB), KB - 1);
        // d log Q_b / d z_k = r (delta_bk - s_k), r = (1 - mix) s_b / Q_b (1 without mixing)
        float Qb = q[0], qb = q[0];
#pragma unroll
        for (int k = 1; k < KB; ++k)
            if (k == b) qb = q[k];
        Qb = mixed(qb, mix);
        const float r = mix != 0.0f ? (1.0f - mix) * qb / Qb : 1.0f;
        if (ww != 0.0f) atomicAdd(&s_loss, -ww * logf(KB * Qb));
        float g[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) g[k] = -ww * r * ((k == b ? 1.0f : 0.0f) - q[k]);
        if (layer != 0) {
            uint32_t pk[KB / 2];
#pragma unroll
            for (int k = 0; k < KB; k += 2) {
                __nv_bfloat162 p2 = __floats2bfloat162_rn(g[k], g[k + 1]);
                pk[k / 2] = *reinterpret_cast<uint32_t *>(&p2);
                dLt[(long long)k * rows + j] = p2.x;
                dLt[(long long)(k + 1) * rows + j] = p2.y;
            }
            uint4 *dst = reinterpret_cast<uint4 *>(dL + (long long)j * KB);
#pragma unroll
            for (int v = 0; v < KB / 8; ++v)
                dst[v] = make_uint4(pk[4 * v], pk[4 * v + 1], pk[4 * v + 2], pk[4 * v + 3]);
        } else {
            // theta0's gradient: warp sums, then one shared atomic per warp and bin
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                float sk = g[k];
                for (int o = 16; o; o >>= 1) sk += __shfl_xor_sync(__activemask(), sk, o);
                if ((threadIdx.x & 31) == 0) atomicAdd(&s_dt[k], sk);
            }
        }
    }
    __syncthreads();
    if (layer == 0 && threadIdx.x < KB) atomicAdd(dtheta + threadIdx.x, s_dt[threadIdx.x]);
    if (threadIdx.x == 0) atomicAdd(loss, s_loss);
}

// out[r] += sum_j At[r][j] (bias gradient from a transposed backward signal): one warp
// per (row, 2048-column slice), 16-byte vector loads, one atomic per warp.
constexpr int ROWSUM_SLICE = 2048;
__global__ void k_rowsum(const __nv_bfloat16 *__restrict__ At, int nrows, int rows, float *__restrict__ out)
{
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (r >= nrows) return;
    const int lane = threadIdx.x & 31;
    const int j0 = blockIdx.y * ROWSUM_SLICE, j1 = min(rows, j0 + ROWSUM_SLICE);
    const __nv_bfloat16 *row = At + (long long)r * rows;
    float s = 0.0f;
    for (int j = j0 + lane * 8; j < j1; j += 32 * 8) {  // rows is a multiple of 128: whole vectors
        const uint4 v = *reinterpret_cast<const uint4 *>(row + j);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(h[q]);
            s += f.x + f.y;
        }
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicAdd(out + r, s);
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

__global__ void k_sync(const float *__restrict__ p, __nv_bfloat16 *__restrict__ wb, __nv_bfloat16 *__restrict__ wt)
{
    const int total = QMCRT_WARP_BF16_WEIGHTS;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int m = e / (3 * WD * WD + KB * WD), r = e % (3 * WD * WD + KB * WD), l = 0;
        while (r >= out_dim(l) * WD) {
            r -= out_dim(l) * WD;
            ++l;
        }
        const int o = r / WD, i = r % WD;
        const __nv_bfloat16 b = __float2bfloat16_rn(p[param_w(m, l) + r]);
        wb[e] = b;
        wt[bf_w(m, l) + i * out_dim(l) + o] = b;
    }
}

unsigned blocks(long long n, int t = 256)
{
    long long b = (n + t - 1) / t;
    return (unsigned)std::max(1ll, std::min(b, 152ll * 32));
}

int gemm(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int splits, GemmEpi ep, cudaStream_t s)
{
    cudaError_t e = launch_gemm_bf16(A, B, M, N, K, splits, ep, s);
    return e == cudaSuccess ? QMCRT_OK : set_error(QMCRT_ERR_CUDA, "flow gemm: %s", cudaGetErrorString(e));
}

GemmEpi epi(int *err)
{
    GemmEpi e;
    memset(&e, 0, sizeof e);
    e.error = err;
    return e;
}

// Forward of MLP m on the features in W.F; keeps activations (and their transposes when
// `keep_t`), logits in W.L.
int mlp_forward(const qmcrt_warp *wp, const Work &W, int m, bool keep_t, cudaStream_t s)
{
    const auto *wb = (const __nv_bfloat16 *)wp->d_weights;
    const __nv_bfloat16 *in = W.F;
    for (int l = 0; l < 3; ++l) {
        GemmEpi e = epi(wp->d_error);
        e.bias = wp->d_params + param_b(m, l);
        e.relu = 1;
        e.out_bf16 = W.H[l];
        if (keep_t) {
            e.out_bf16_t = W.Ht[l];
            e.ldt = W.rows;
        }
        int rc = gemm(in, wb + bf_w(m, l), W.rows, WD, WD, 1, e, s);
        if (rc) return rc;
        in = W.H[l];
    }
    GemmEpi e = epi(wp->d_error);
    e.bias = wp->d_params + param_b(m, 3);
    e.out_f32 = W.L;
    return gemm(in, wb + bf_w(m, 3), W.rows, KB, WD, 1, e, s);
}

int check_warp(const qmcrt_warp *w)
{
    if (!w || w->struct_size != sizeof(qmcrt_warp)) return set_error(QMCRT_ERR_INVALID_ARG, "warp descriptor");
    if (!w->d_params || !w->d_weights || !w->d_weights_t) return set_error(QMCRT_ERR_INVALID_ARG, "NULL warp buffers");
    if (((uintptr_t)w->d_weights | (uintptr_t)w->d_weights_t) & 15)
        return set_error(QMCRT_ERR_INVALID_ARG, "warp weights must be 16-byte aligned");
    if (!(w->uniform_mix >= 0.0f && w->uniform_mix < 1.0f))
        return set_error(QMCRT_ERR_INVALID_ARG, "uniform_mix must lie in [0, 1)");
    return QMCRT_OK;
}

int launch_status(const char *what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QMCRT_OK : set_error(QMCRT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace
}  // namespace qmcrt

using namespace qmcrt;

extern "C" {

uint64_t qmcrt_warp_workspace_bytes(uint64_t rows) { return bytes_for(round128(rows ? rows : 1)); }

int qmcrt_warp_sync(const qmcrt_warp *warp, void *stream)
{
    int rc = check_warp(warp);
    if (rc) return rc;
    k_sync<<<blocks(QMCRT_WARP_BF16_WEIGHTS), 256, 0, (cudaStream_t)stream>>>(
        warp->d_params, (__nv_bfloat16 *)warp->d_weights, (__nv_bfloat16 *)warp->d_weights_t);
    return launch_status("warp sync");
}

int qmcrt_warp_forward(const qmcrt_warp *warp, const float *d_u, float *d_x, float *d_logj, uint64_t n,
                       void *d_workspace, uint64_t workspace_bytes, void *stream)
{
    (void)d_workspace;
    (void)workspace_bytes;
    int rc = check_warp(warp);
    if (rc) return rc;
    if (!d_u || !d_x || !d_logj) return set_error(QMCRT_ERR_INVALID_ARG, "NULL buffer");
    cudaError_t e = launch_warp_forward_fused(warp->d_params, (const __nv_bfloat16 *)warp->d_weights, d_u, d_x,
                                              d_logj, (long long)n, warp->uniform_mix, warp->d_error,
                                              (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(QMCRT_ERR_CUDA, "warp forward: %s", cudaGetErrorString(e));
    return QMCRT_OK;
}

int qmcrt_warp_grad(const qmcrt_warp *warp, const float *d_x, const float *d_w, uint64_t n, float *d_grad,
                    float *d_loss, void *d_workspace, uint64_t workspace_bytes, void *stream)
{
    int rc = check_warp(warp);
    if (rc) return rc;
    if (!d_x || !d_w || !d_grad || !d_loss || !d_workspace) return set_error(QMCRT_ERR_INVALID_ARG, "NULL buffer");
    const int R = rows_for(workspace_bytes);
    if (R < 128) return set_error(QMCRT_ERR_INVALID_ARG, "workspace below one pass of 128 rows");
    cudaStream_t s = (cudaStream_t)stream;
    const Work W0 = carve(d_workspace, R);
    const auto *wt = (const __nv_bfloat16 *)warp->d_weights_t;
    cudaError_t e = cudaMemsetAsync(W0.wsum, 0, sizeof(double), s);
    if (e != cudaSuccess) return set_error(QMCRT_ERR_CUDA, "warp grad: %s", cudaGetErrorString(e));
    if (n) k_wsum<<<blocks((long long)n), 256, 0, s>>>(d_w, (int)n, W0.wsum);
    for (uint64_t base = 0; base < n; base += (uint64_t)R) {
        const int cnt = (int)std::min<uint64_t>((uint64_t)R, n - base);
        Work W = W0;
        W.rows = (int)round128(cnt);
        const float *x = d_x + 3 * base, *w = d_w + base;
        k_loss_grad<<<(W.rows + 255) / 256, 256, 0, s>>>(0, warp->d_params, nullptr, x, w, cnt, W.rows, W.wsum, d_loss,
                                                          d_grad, nullptr, nullptr, warp->uniform_mix);
        for (int m = 0; m < 2; ++m) {
            k_features<<<W.rows / FEAT_ROWS, 256, 0, s>>>(x, cnt, W.rows, m, W.F, W.Ft);
            if ((rc = mlp_forward(warp, W, m, true, s))) return rc;
            k_loss_grad<<<(W.rows + 255) / 256, 256, 0, s>>>(m + 1, warp->d_params, W.L, x, w, cnt, W.rows, W.wsum,
                                                              d_loss, d_grad, W.dL, W.dLt, warp->uniform_mix);
            if ((rc = launch_status("warp loss"))) return rc;
            const int splits = std::max(1, W.rows / 512);  // weight gradients: K = rows split over CTAs
            // layer 3: signal dL [rows x 32]
            const __nv_bfloat16 *dP = W.dL, *dPt = W.dLt;
            for (int l = 3; l >= 0; --l) {
                const int N_out = out_dim(l);
                const __nv_bfloat16 *Xt = l == 0 ? W.Ft : W.Ht[l - 1];
                GemmEpi gw = epi(warp->d_error);  // dW[l] = dP^T . X  (M = out, N = in, K = rows)
                gw.out_f32 = d_grad + param_w(m, l);
                gw.atomic_f32 = splits > 1;
                if (gw.atomic_f32 == 0) gw.atomic_f32 = 1;  // accumulate into the caller's gradient
                if ((rc = gemm(dPt, Xt, N_out, WD, W.rows, splits, gw, s))) return rc;
                k_rowsum<<<dim3((N_out + 7) / 8, (W.rows + ROWSUM_SLICE - 1) / ROWSUM_SLICE), 256, 0, s>>>(
                    dPt, N_out, W.rows, d_grad + param_b(m, l));
                if ((rc = launch_status("warp bias grad"))) return rc;
                if (l == 0) break;
                GemmEpi gx = epi(warp->d_error);  // dH[l-1] = (dP . W[l]) * (H[l-1] > 0)
                gx.mask = W.H[l - 1];
                gx.out_bf16 = W.dP[l & 1];
                gx.out_bf16_t = W.dPt[l & 1];
                gx.ldt = W.rows;
                if ((rc = gemm(dP, wt + bf_w(m, l), W.rows, WD, N_out, 1, gx, s))) return rc;
                dP = W.dP[l & 1];
                dPt = W.dPt[l & 1];
            }
        }
    }
    return launch_status("warp grad");
}

int qmcrt_warp_adam(const qmcrt_warp *warp, const float *d_grad, float *d_m, float *d_v, const qmcrt_adam *opt,
                    void *stream)
{
    int rc = check_warp(warp);
    if (rc) return rc;
    if (!d_grad || !d_m || !d_v || !opt || opt->struct_size != sizeof(qmcrt_adam) || opt->step < 1)
        return set_error(QMCRT_ERR_INVALID_ARG, "adam arguments");
    const float bc1 = (float)(1.0 - std::pow(opt->beta1, opt->step));
    const float bc2 = (float)(1.0 - std::pow(opt->beta2, opt->step));
    k_adam<<<blocks(QMCRT_WARP_PARAMS), 256, 0, (cudaStream_t)stream>>>(
        warp->d_params, d_grad, d_m, d_v, QMCRT_WARP_PARAMS, (float)opt->lr, (float)opt->beta1, (float)opt->beta2,
        (float)opt->eps, bc1, bc2);
    if ((rc = launch_status("warp adam"))) return rc;
    return qmcrt_warp_sync(warp, stream);
}

}  // extern "C"

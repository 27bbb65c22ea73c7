// qmcrt_trace_single.cu -- single-scattering tracer kernel (Sec. 3.2-3.6).
//
// Packet mapping: warp task w (0 <= w < stride = ceil(count/32)) traces the packets
// j = lane * stride + w.  The 32 packets of a warp differ only in the high bits of
// their index, so for Sobol points (whose leading bits in every coordinate depend
// only on the low bits of the index) they start in nearly the same direction, march
// through the same cells and usually land in the same pixel: the warp stays coherent
// and its deposits collapse to one atomic.
#include "qmcrt_device.cuh"

namespace qmcrt {

template <class T>
__global__ void __launch_bounds__(256) k_trace_single(const __grid_constant__ TraceP<T> P)
{
    const int lane = threadIdx.x & 31;
    const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= P.stride) return;  // uniform per warp
    const uint64_t j = (uint64_t)lane * P.stride + w;
    const bool live = j < P.count;
    T S[3] = {T(0), T(0), T(0)};
    T x = T(0), y = T(0);
    int status = 1;
    T pos[3] = {T(0), T(0), T(0)};
    if (live) {
        const uint64_t i = P.first + j;
        T d[3], a[3], wgt, W1;
        const T wd = emit(P, i, pos, d, a, wgt);
        if (forced_step(P, pos, d, wd, W1)) {
            const T W0 = wgt * W1 * P.dust.albedo;
            status = peel_unpolarized(P, pos, d, W0, S, x, y) ? 0 : 2;
        }
        if (P.log) {
            double *r = P.log + j * 9;
            r[0] = pos[0];
            r[1] = pos[1];
            r[2] = pos[2];
            r[3] = status == 0 ? (double)S[0] : 0.0;
            r[4] = status == 0 ? (double)S[1] : 0.0;
            r[5] = status == 0 ? (double)S[2] : 0.0;
            r[6] = x;
            r[7] = y;
            r[8] = status;
        }
    }
    splat(P, status == 0, 0, x, y, S);
}

template <class T>
static cudaError_t launch(const TraceP<T> &p, int block, cudaStream_t s)
{
    if (p.count == 0) return cudaSuccess;
    const uint64_t threads = p.stride * 32;
    const uint64_t grid = (threads + block - 1) / block;
    k_trace_single<T><<<(unsigned)grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_trace_single_f32(const TraceP<float> &p, int block, cudaStream_t s) { return launch(p, block, s); }
cudaError_t launch_trace_single_f64(const TraceP<double> &p, int block, cudaStream_t s) { return launch(p, block, s); }

}  // namespace qmcrt

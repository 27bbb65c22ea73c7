// qmcrt_trace_single.cu -- single-scattering tracer kernel (Sec. 3.2-3.6).
//
// Packet mapping (OrderP): for Sobol point sets a warp receives 32 points from
// adjacent elementary boxes of the first three coordinates, so its packets start in
// nearly the same direction, scatter at nearly the same depth, walk the same cells
// and usually land in the same pixel: the warp stays coherent and its deposits
// collapse to one atomic per Stokes component.
#include "qmcrt_device.cuh"

namespace qmcrt {

template <class T>
__global__ void __launch_bounds__(256) k_trace_single(const __grid_constant__ TraceP<T> P)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((tid & ~31ull) >= P.ord.threads) return;  // uniform per warp
    uint64_t i;
    const bool live_index = packet_index(P.ord, P.first, P.count, tid, i);
    if (!__any_sync(FULL_MASK, live_index)) return;
    const uint64_t j = i - P.first;
    const bool live = live_index;
    T S[3] = {T(0), T(0), T(0)};
    T x = T(0), y = T(0);
    int status = 1;
    T pos[3] = {T(0), T(0), T(0)};
    if (live) {
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
    const uint64_t threads = (p.ord.threads + 31) & ~31ull;
    const uint64_t grid = (threads + block - 1) / block;
    k_trace_single<T><<<(unsigned)grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_trace_single_f32(const TraceP<float> &p, int block, cudaStream_t s) { return launch(p, block, s); }
cudaError_t launch_trace_single_f64(const TraceP<double> &p, int block, cudaStream_t s) { return launch(p, block, s); }

}  // namespace qmcrt

// qmcrt_trace_multiple.cu -- multiple-scattering tracer kernel (Sec. 3.5, 3.7).
//
// One thread per packet, the same warp-coherent packet mapping as the single-
// scattering kernel; the orders are in qmcrt_orders.cuh.  With a learned warp the
// first-order coordinates come from a buffer (x = T(u) and log |dx/du| per packet);
// the optional training log records, per packet, the coordinates used and two norms
// of the intensities its peel-offs put into the image (their sum, and the square root
// of their sum of squares).
#include "qmcrt_orders.cuh"

namespace qmcrt {

template <class T>
struct OneObserver {
    const TraceP<T> &P;
    T total, total2;  // in-image Stokes I of this packet's peel-offs: sum, sum of squares
    __device__ __forceinline__ void operator()(int k, bool alive, const T pos[3], const T n[3], const T a[3],
                                               const T S[3])
    {
        T out[3] = {T(0), T(0), T(0)};
        T x = T(0), y = T(0);
        const bool contrib = alive && peel_polarized(P, pos, n, a, S, out, x, y);
        if (contrib && x >= -P.obs.hw && x < P.obs.hw && y >= -P.obs.hw && y < P.obs.hw) {
            total += out[0];
            total2 += out[0] * out[0];
        }
        splat(P, contrib, P.per_order ? k - 1 : 0, x, y, out);
    }
};

// FP32: at most 64 registers, 4 blocks (32 warps) per SM: the walks are latency-bound
// and the extra warps pay for a few spilled registers (9 % faster than 80 registers).
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_trace_multiple(const __grid_constant__ TraceP<T> P)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((tid & ~31ull) >= P.ord.threads) return;  // uniform per warp
    uint64_t i = P.first;
    const bool live_index = packet_index(P.ord, P.first, P.count, tid, i);
    if (!__any_sync(FULL_MASK, live_index)) return;
    const uint64_t j = i - P.first;
    OneObserver<T> peel{P, T(0), T(0)};
    trace_orders(P, i, j, live_index, peel);
    if (P.train_log && live_index) {
        float *r = P.train_log + 5 * j;
        if (P.warp_x) {
            r[0] = P.warp_x[3 * j];
            r[1] = P.warp_x[3 * j + 1];
            r[2] = P.warp_x[3 * j + 2];
        } else {
            r[0] = (float)point<T>(P.pts, i, 0);
            r[1] = (float)point<T>(P.pts, i, 1);
            r[2] = (float)point<T>(P.pts, i, 2);
        }
        r[3] = (float)peel.total;
        r[4] = (float)Mth<T>::sqrt_(peel.total2);
    }
}

template <class T>
static cudaError_t launch(const TraceP<T> &p, int block, cudaStream_t s)
{
    if (p.count == 0) return cudaSuccess;
    const uint64_t threads = (p.ord.threads + 31) & ~31ull;
    const uint64_t grid = (threads + block - 1) / block;
    k_trace_multiple<T><<<(unsigned)grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_trace_multiple_f32(const TraceP<float> &p, int block, cudaStream_t s) { return launch(p, block, s); }
cudaError_t launch_trace_multiple_f64(const TraceP<double> &p, int block, cudaStream_t s) { return launch(p, block, s); }

}  // namespace qmcrt

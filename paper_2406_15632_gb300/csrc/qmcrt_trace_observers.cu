// qmcrt_trace_observers.cu -- one trace feeding up to QMCRT_MAX_OBSERVERS observers.
//
// A packet's emission, forced depths and scatterings are computed once; at each
// scattering the peel-off (optical depth toward the observer, phase function, Stokes
// rotation into the observer's sky frame) and the binning are repeated per observer
// into that observer's image stack.  The per-observer arithmetic is the one-observer
// kernels' (same functions), so stack o equals the single-observer result bit for bit
// in fixed point.  The observer loop is uniform across the warp, so deposits stay
// warp-aggregated.
#include "qmcrt_orders.cuh"

namespace qmcrt {

template <class T>
struct ObserverSet {
    const TraceP<T> &P;
    const ObsSet<T> &S;
    __device__ __forceinline__ void operator()(int k, bool alive, const T pos[3], const T n[3], const T a[3],
                                               const T Sv[3])
    {
        for (int o = 0; o < S.n; ++o) {
            T out[3] = {T(0), T(0), T(0)};
            T x = T(0), y = T(0);
            const bool c = alive && peel_polarized(P, S.o[o], pos, n, a, Sv, out, x, y);
            splat(S.o[o], P.acc, (size_t)o * S.stack, c, P.per_order ? k - 1 : 0, x, y, out);
        }
    }
};

template <class T>
__global__ void __launch_bounds__(256) k_trace_observers_single(const __grid_constant__ TraceP<T> P,
                                                               const __grid_constant__ ObsSet<T> S)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((tid & ~31ull) >= P.ord.threads) return;  // uniform per warp
    uint64_t i = P.first;
    const bool live = packet_index(P.ord, P.first, P.count, tid, i);
    if (!__any_sync(FULL_MASK, live)) return;
    T pos[3] = {T(0), T(0), T(0)}, d[3] = {T(0), T(0), T(1)};
    T W0 = T(0);
    bool scattered = false;
    if (live) {
        T a[3], wgt, W1;
        const T wd = emit(P, i, pos, d, a, wgt);
        if (forced_step(P, pos, d, wd, W1)) {
            W0 = wgt * W1 * P.dust.albedo;
            scattered = true;
        }
    }
    for (int o = 0; o < S.n; ++o) {
        T Sv[3] = {T(0), T(0), T(0)};
        T x = T(0), y = T(0);
        const bool c = scattered && peel_unpolarized(P, S.o[o], pos, d, W0, Sv, x, y);
        splat(S.o[o], P.acc, (size_t)o * S.stack, c, 0, x, y, Sv);
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_trace_observers_multiple(const __grid_constant__ TraceP<T> P,
                                                                 const __grid_constant__ ObsSet<T> S)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((tid & ~31ull) >= P.ord.threads) return;  // uniform per warp
    uint64_t i = P.first;
    const bool live = packet_index(P.ord, P.first, P.count, tid, i);
    if (!__any_sync(FULL_MASK, live)) return;
    ObserverSet<T> peel{P, S};
    trace_orders(P, i, i - P.first, live, peel);
}

template <class T>
static cudaError_t launch(const TraceP<T> &p, const ObsSet<T> &obs, int block, cudaStream_t s)
{
    if (p.count == 0) return cudaSuccess;
    const uint64_t threads = (p.ord.threads + 31) & ~31ull;
    const uint64_t grid = (threads + block - 1) / block;
    if (p.max_orders > 1)
        k_trace_observers_multiple<T><<<(unsigned)grid, block, 0, s>>>(p, obs);
    else
        k_trace_observers_single<T><<<(unsigned)grid, block, 0, s>>>(p, obs);
    return cudaGetLastError();
}

cudaError_t launch_trace_observers_f32(const TraceP<float> &p, const ObsSet<float> &obs, int block, cudaStream_t s)
{
    return launch(p, obs, block, s);
}

cudaError_t launch_trace_observers_f64(const TraceP<double> &p, const ObsSet<double> &obs, int block, cudaStream_t s)
{
    return launch(p, obs, block, s);
}

}  // namespace qmcrt

// qmcrt_wavefront.cu -- multiple scattering as a wavefront of orders (Sec. 3.5, 3.7).
//
// The one-kernel tracer keeps a packet on one thread for all its orders.  Its first
// order is coherent (net-ordered warps start 32 packets in nearly the same direction),
// but from the second order on each lane scatters into its own direction and the warp
// waits for its longest walk.  Here every order is a launch over the packets still
// alive, and between orders the live packets are regrouped by a key built from their
// position (3 bits per axis) and their new direction (8 bins in cos theta x 16 in phi),
// so a warp again traces 32 similar rays:
//
//   order 1:   emission, forced step, peel-off, roulette, scattering for order 2 -> queue
//   order k:   key + histogram -> bucket offsets (one block) -> scatter into buckets ->
//              forced step (or march), peel-off, roulette, scattering for k+1 -> queue
//
// Per packet the arithmetic is the one-kernel tracer's, step for step (the scattering
// that opens order k runs at the end of order k-1), so fixed-point images are identical.
// Launch sizes do not depend on the live counts, which stay on the device: the order
// kernels are persistent and read their count when they start.
#include <algorithm>

#include "qmcrt_device.cuh"

namespace qmcrt {

namespace {

constexpr int WV_FIELDS = 14;  // pos[3], n[3], a[3], S[3], in-image I sum, sum of squares
constexpr int WV_KEY_BITS = 16;
constexpr int WV_BUCKETS = 1 << WV_KEY_BITS;

template <class T>
struct WaveQueue {
    T *v[WV_FIELDS];
    uint32_t *idx;  // point index - first
};

template <class T>
struct WaveWork {
    WaveQueue<T> q[2];
    uint32_t *count;  // [2] live packets in q[0], q[1]
    uint32_t *keys;   // [cap]
    uint32_t *hist;   // [WV_BUCKETS] histogram, then bucket cursors
};

template <class T>
struct Packet {
    T pos[3], n[3], a[3], S[3], tot, tot2;
};

template <class T>
__device__ __forceinline__ void load(const WaveQueue<T> &Q, uint32_t q, Packet<T> &p)
{
    for (int c = 0; c < 3; ++c) {
        p.pos[c] = Q.v[c][q];
        p.n[c] = Q.v[3 + c][q];
        p.a[c] = Q.v[6 + c][q];
        p.S[c] = Q.v[9 + c][q];
    }
    p.tot = Q.v[12][q];
    p.tot2 = Q.v[13][q];
}

template <class T>
__device__ __forceinline__ void store(const WaveQueue<T> &Q, uint32_t q, const Packet<T> &p, uint32_t j)
{
    for (int c = 0; c < 3; ++c) {
        Q.v[c][q] = p.pos[c];
        Q.v[3 + c][q] = p.n[c];
        Q.v[6 + c][q] = p.a[c];
        Q.v[9 + c][q] = p.S[c];
    }
    Q.v[12][q] = p.tot;
    Q.v[13][q] = p.tot2;
    Q.idx[q] = j;
}

// Append the lanes with `keep` to queue Q (one atomic per warp).  All 32 lanes call.
template <class T>
__device__ __forceinline__ void append(const WaveQueue<T> &Q, uint32_t *count, bool keep, const Packet<T> &p,
                                       uint32_t j)
{
    const unsigned m = __ballot_sync(FULL_MASK, keep);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int first = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == first) base = atomicAdd(count, (uint32_t)__popc(m));
    base = __shfl_sync(FULL_MASK, base, first);
    if (keep) store(Q, base + __popc(m & ((1u << lane) - 1u)), p, j);
}

template <class T>
__device__ __forceinline__ void write_log(const TraceP<T> &P, uint64_t i, uint64_t j, const Packet<T> &p)
{
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
    r[3] = (float)p.tot;
    r[4] = (float)Mth<T>::sqrt_(p.tot2);
}

// Order k of a packet that is alive at its start (scattered already if k > 1), with
// depth coordinate wd; then roulette and the scattering that opens order k + 1.  All 32
// lanes call (the peel-off bins into the image).  Returns whether it lives on.
template <class T>
__device__ __forceinline__ bool run_order(const TraceP<T> &P, int k, uint64_t i, bool alive, T wd, Packet<T> &p)
{
    const int base = 4 * (k - 1);
    if (alive) {
        if (k == 1 || P.force_all) {
            T W1;
            if (forced_step(P, p.pos, p.n, wd, W1)) {
                p.S[0] *= W1;
                p.S[1] *= W1;
                p.S[2] *= W1;
            } else {
                alive = false;
            }
        } else if (!march(P.med, p.pos, p.n, -Mth<T>::log_(wd))) {
            alive = false;
        }
        if (alive) {
            p.S[0] *= P.dust.albedo;
            p.S[1] *= P.dust.albedo;
            p.S[2] *= P.dust.albedo;
        }
    }
    T out[3] = {T(0), T(0), T(0)};
    T x = T(0), y = T(0);
    const bool contrib = alive && peel_polarized(P, p.pos, p.n, p.a, p.S, out, x, y);
    if (contrib && x >= -P.obs.hw && x < P.obs.hw && y >= -P.obs.hw && y < P.obs.hw) {
        p.tot += out[0];
        p.tot2 += out[0] * out[0];
    }
    splat(P, contrib, P.per_order ? k - 1 : 0, x, y, out);
    if (alive) {
        if (k == P.max_orders) {
            alive = false;
        } else if (p.S[0] < P.rr_threshold) {
            if (point<T>(P.pts, i, base + 3) < P.rr_survival) {
                p.S[0] /= P.rr_survival;
                p.S[1] /= P.rr_survival;
                p.S[2] /= P.rr_survival;
            } else {
                alive = false;
            }
        }
    }
    if (alive) scatter(P.dust, point<T>(P.pts, i, base + 4), point<T>(P.pts, i, base + 5), p.n, p.a, p.S);
    return alive;
}

template <class T>
__global__ void __launch_bounds__(256) k_wave_first(const __grid_constant__ TraceP<T> P, WaveQueue<T> out,
                                                   uint32_t *count)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((tid & ~31ull) >= P.ord.threads) return;  // uniform per warp
    uint64_t i = P.first;
    const bool live = packet_index(P.ord, P.first, P.count, tid, i);
    if (!__any_sync(FULL_MASK, live)) return;
    const uint64_t j = i - P.first;
    Packet<T> p;
    for (int c = 0; c < 3; ++c) p.pos[c] = p.a[c] = p.S[c] = T(0);
    p.n[0] = p.n[1] = T(0);
    p.n[2] = T(1);
    p.a[0] = T(1);
    p.tot = p.tot2 = T(0);
    T wd = T(0);
    if (live) {
        T wgt;
        if (P.warp_x) {  // learned proposal: first-order coordinates and their Jacobian
            T sp, cp;
            direction_from((T)P.warp_x[3 * j], (T)P.warp_x[3 * j + 1], p.n, p.a, sp, cp);
            wd = (T)P.warp_x[3 * j + 2];
            wgt = Mth<T>::exp_((T)P.warp_logj[j]);
        } else {
            const int e = 4 * P.max_orders;  // a finite star's two extra emission coordinates
            wd = emit(P, i, p.pos, p.n, p.a, wgt, e, e + 1, 2);
        }
        p.S[0] = wgt;
    }
    const bool on = run_order(P, 1, i, live, wd, p);
    append(out, count, on, p, (uint32_t)j);
    if (live && !on && P.train_log) write_log(P, i, j, p);
}

template <class T>
__device__ __forceinline__ uint32_t wave_key(const MediumP<T> &G, const T pos[3], const T n[3])
{
    uint32_t key = 0;
    for (int c = 0; c < 3; ++c) {
        const T f = (pos[c] - G.lo[c]) / (G.hi[c] - G.lo[c]) * T(8);
        key = (key << 3) | (uint32_t)min(7, max(0, (int)f));
    }
    const int ct = min(7, max(0, (int)((n[2] + T(1)) * T(4))));
    const float ph = atan2f((float)n[1], (float)n[0]);  // the key only orders packets
    const int pb = min(15, max(0, (int)((ph + 3.14159265f) * 2.54647909f)));  // 16 / (2 pi)
    return (key << 7) | (uint32_t)(ct << 4) | (uint32_t)pb;
}

template <class T>
__global__ void __launch_bounds__(256) k_wave_key(const __grid_constant__ TraceP<T> P, WaveQueue<T> in,
                                                 const uint32_t *count, uint32_t *keys, uint32_t *hist)
{
    const uint32_t n = *count;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const T pos[3] = {in.v[0][q], in.v[1][q], in.v[2][q]};
        const T d[3] = {in.v[3][q], in.v[4][q], in.v[5][q]};
        const uint32_t key = wave_key(P.med, pos, d);
        keys[q] = key;
        atomicAdd(hist + key, 1u);
    }
}

// Exclusive scan of the bucket histogram into cursors (one block of 1024 threads).
__global__ void __launch_bounds__(1024) k_wave_scan(uint32_t *hist)
{
    __shared__ uint32_t part[1024];
    constexpr int PER = WV_BUCKETS / 1024;
    const int t = threadIdx.x;
    uint32_t s = 0;
    for (int b = 0; b < PER; ++b) s += hist[t * PER + b];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = t ? part[t - 1] : 0u;
    for (int b = 0; b < PER; ++b) {
        const uint32_t h = hist[t * PER + b];
        hist[t * PER + b] = run;
        run += h;
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_wave_scatter(WaveQueue<T> in, const uint32_t *count, const uint32_t *keys,
                                                     uint32_t *cursor, WaveQueue<T> out)
{
    const uint32_t n = *count;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const uint32_t dst = atomicAdd(cursor + keys[q], 1u);
        for (int f = 0; f < WV_FIELDS; ++f) out.v[f][dst] = in.v[f][q];
        out.idx[dst] = in.idx[q];
    }
}

// Order k >= 2 over the sorted queue `in`; survivors go to `out`.
template <class T>
__global__ void __launch_bounds__(256) k_wave_order(const __grid_constant__ TraceP<T> P, int k, WaveQueue<T> in,
                                                   const uint32_t *in_count, WaveQueue<T> out, uint32_t *out_count)
{
    const uint32_t n = *in_count;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); q0 < n; q0 += stride) {  // uniform per warp
        const uint32_t q = q0 + (threadIdx.x & 31u);
        const bool live = q < n;
        Packet<T> p;
        uint32_t j = 0;
        if (live) {
            load(in, q, p);
            j = in.idx[q];
        } else {
            for (int c = 0; c < 3; ++c) p.pos[c] = p.n[c] = p.a[c] = p.S[c] = T(0);
            p.tot = p.tot2 = T(0);
        }
        const uint64_t i = P.first + j;
        const T wd = live ? point<T>(P.pts, i, 4 * (k - 1) + 2) : T(0);
        const bool on = run_order(P, k, i, live, wd, p);
        append(out, out_count, on, p, j);
        if (live && !on && P.train_log) write_log(P, i, j, p);
    }
}

template <class T>
WaveWork<T> carve(void *ws, uint64_t cap)
{
    WaveWork<T> W;
    char *c = (char *)ws;
    auto take = [&](size_t bytes) {
        char *r = c;
        c += (bytes + 255) & ~(size_t)255;
        return r;
    };
    for (int b = 0; b < 2; ++b) {
        for (int f = 0; f < WV_FIELDS; ++f) W.q[b].v[f] = (T *)take(cap * sizeof(T));
        W.q[b].idx = (uint32_t *)take(cap * 4);
    }
    W.count = (uint32_t *)take(2 * 4);
    W.keys = (uint32_t *)take(cap * 4);
    W.hist = (uint32_t *)take(WV_BUCKETS * 4);
    return W;
}

template <class T>
cudaError_t launch_wave(const TraceP<T> &P, void *ws, uint64_t cap, int sms, cudaStream_t s)
{
    if (P.count == 0) return cudaSuccess;
    WaveWork<T> W = carve<T>(ws, cap);
    cudaError_t e = cudaMemsetAsync(W.count, 0, 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const uint64_t threads = (P.ord.threads + 31) & ~31ull;
    k_wave_first<T><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(P, W.q[1], W.count + 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::max(1, sms * 8);
    for (int k = 2; k <= P.max_orders; ++k) {
        // the queue of order k is q[1] (count[1]); sort it into q[0], trace into q[1]
        if ((e = cudaMemsetAsync(W.hist, 0, WV_BUCKETS * sizeof(uint32_t), s)) != cudaSuccess) return e;
        k_wave_key<T><<<grid, 256, 0, s>>>(P, W.q[1], W.count + 1, W.keys, W.hist);
        k_wave_scan<<<1, 1024, 0, s>>>(W.hist);
        k_wave_scatter<T><<<grid, 256, 0, s>>>(W.q[1], W.count + 1, W.keys, W.hist, W.q[0]);
        if ((e = cudaMemcpyAsync(W.count, W.count + 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(W.count + 1, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
        k_wave_order<T><<<grid, 256, 0, s>>>(P, k, W.q[0], W.count, W.q[1], W.count + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

uint64_t wavefront_workspace_bytes(uint64_t cap, int precision)
{
    const uint64_t t = precision == QMCRT_PREC_F64 ? 8 : 4;
    auto pad = [](uint64_t b) { return (b + 255) & ~255ull; };
    return 2 * (WV_FIELDS * pad(cap * t) + pad(cap * 4)) + pad(8) + pad(cap * 4) + pad(WV_BUCKETS * 4);
}

cudaError_t launch_trace_wavefront_f32(const TraceP<float> &p, void *ws, uint64_t cap, int sms, cudaStream_t s)
{
    return launch_wave(p, ws, cap, sms, s);
}

cudaError_t launch_trace_wavefront_f64(const TraceP<double> &p, void *ws, uint64_t cap, int sms, cudaStream_t s)
{
    return launch_wave(p, ws, cap, sms, s);
}

}  // namespace qmcrt

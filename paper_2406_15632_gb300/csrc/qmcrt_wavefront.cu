// qmcrt_wavefront.cu -- multiple scattering as a wavefront of orders (Sec. 3.5, 3.7).
//
// The one-kernel tracer keeps a packet on one thread for all its orders.  Its first
// order is coherent (net-ordered warps start 32 packets in nearly the same direction),
// but from the second order on each lane scatters into its own direction and the warp
// waits for its longest walk.  Here every order is a launch over the packets still
// alive, and between orders the live packets are regrouped by a key built from their
// position (one of 16^3 cells of the box) and their new direction (32 bins in cos theta
// x 64 in phi), so a warp again traces 32 similar rays:
//
//   order 1:   emission, forced step, peel-off, roulette, scattering for order 2 ->
//              queue (with each packet's key, counted in the bucket histogram)
//   order k:   bucket offsets (a tiled scan) -> record indices into
//              buckets -> forced step (or march), peel-off, roulette, scattering for
//              k+1 -> the other queue
//
// A queued packet is one 64-byte record (128 in FP64) that stays where it was appended:
// the sort moves 4-byte indices, and order k gathers its records through them (two
// whole sectors per record), appending the survivors to the other queue.
//
// Per packet the arithmetic is the one-kernel tracer's, step for step (the scattering
// that opens order k runs at the end of order k-1), so fixed-point images are identical.
// Launch sizes do not depend on the live counts, which stay on the device: the order
// kernels are persistent and read their count when they start.
#include <algorithm>

#include "qmcrt_device.cuh"

namespace qmcrt {

namespace {

// Key split measured on the clumpy envelope (2^24 packets, 20 orders): 16^3 position
// cells with 32 x 64 direction bins (2^23 buckets, position-major) take 77 ms, against
// 89 ms for the octant with the same direction bins (2^14 buckets) and 80 ms for 8^3
// cells; finer direction bins or position cells gain nothing more (77-79 ms), 2^25 buckets
// lose it again to the histogram's clearing and scan (83 ms).  Packets that start close
// together in nearly one direction cross nearly the same cells, so a warp's loads share
// cache lines.
constexpr int WV_POS_BITS = 4;  // per axis: 16 position cells
constexpr int WV_COS_BITS = 5;  // direction bins: 32 in cos theta
constexpr int WV_PHI_BITS = 6;  //                 x 64 in phi
constexpr int WV_KEY_BITS = 3 * WV_POS_BITS + WV_COS_BITS + WV_PHI_BITS;
constexpr int WV_BUCKETS = 1 << WV_KEY_BITS;
static_assert(WV_KEY_BITS >= 20 && WV_KEY_BITS <= 30, "the scan takes 1024-bucket tiles, their totals in one block");

template <class T>
struct Packet {
    T pos[3], n[3], a[3], S[3], tot, tot2;
};

// One queued packet: its state and its index, one contiguous record (64 bytes in FP32,
// 128 in FP64) moved with 16-byte vector accesses.
template <class T>
struct alignas(16) Rec {
    Packet<T> p;
    uint32_t j;  // point index - first
    uint32_t pad[sizeof(T) == 4 ? 1 : 3];
};
static_assert(sizeof(Rec<float>) == 64 && sizeof(Rec<double>) == 128, "record size");

template <class T>
struct WaveWork {
    Rec<T> *q[2];       // [cap] each: order k reads q[(k + 1) & 1] and appends to q[k & 1]
    uint32_t *count;    // [3] packets of this order, packets appended for the next, chunk counter
    uint32_t *keys;     // [cap] bucket of each appended record
    uint32_t *perm;     // [cap] record indices of the queue being read, in bucket order
    uint32_t *hist;     // [WV_BUCKETS] histogram of the appended records, then bucket cursors
};

template <class T>
__device__ __forceinline__ void copy_rec(Rec<T> *dst, const Rec<T> *src)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int v = 0; v < (int)(sizeof(Rec<T>) / 16); ++v) d[v] = s[v];
}

template <class T>
__device__ __forceinline__ uint32_t wave_key(const MediumP<T> &G, const T pos[3], const T n[3])
{
    constexpr int NP = 1 << WV_POS_BITS, NC = 1 << WV_COS_BITS, NF = 1 << WV_PHI_BITS;
    uint32_t key = 0;
    for (int c = 0; c < 3; ++c) {
        const T f = (pos[c] - G.lo[c]) / (G.hi[c] - G.lo[c]) * T(NP);
        key = (key << WV_POS_BITS) | (uint32_t)min(NP - 1, max(0, (int)f));
    }
    const int ct = min(NC - 1, max(0, (int)((n[2] + T(1)) * T(NC / 2.0))));
    const float ph = atan2f((float)n[1], (float)n[0]);  // the key only orders packets
    const int pb = min(NF - 1, max(0, (int)((ph + 3.14159265f) * (float)(NF / 6.283185307179586))));
    return (key << (WV_COS_BITS + WV_PHI_BITS)) | (uint32_t)(ct << WV_PHI_BITS) | (uint32_t)pb;
}

// Append the lanes with `keep` to queue dst with their bucket keys and count them in
// the histogram of the next sort (one queue atomic per warp).  All 32 lanes call.
template <class T>
__device__ __forceinline__ void append(const TraceP<T> &P, const WaveWork<T> &W, Rec<T> *dst, bool keep,
                                       const Packet<T> &p, uint32_t j)
{
    const unsigned m = __ballot_sync(FULL_MASK, keep);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int first = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == first) base = atomicAdd(W.count + 1, (uint32_t)__popc(m));
    base = __shfl_sync(FULL_MASK, base, first);
    const uint32_t key = keep ? wave_key(P.med, p.pos, p.n) : 0xffffffffu;
    // lanes with equal keys count into the histogram with one atomic (a warp's
    // packets come from one bucket of the last sort and mostly share their key)
    const unsigned peers = __match_any_sync(FULL_MASK, key);
    if (keep) {
        const uint32_t q = base + __popc(m & ((1u << lane) - 1u));
        Rec<T> r;
        r.p = p;
        r.j = j;
        for (int k = 0; k < (int)(sizeof(r.pad) / 4); ++k) r.pad[k] = 0u;
        copy_rec(dst + q, &r);
        W.keys[q] = key;
        if (lane == __ffs(peers) - 1) atomicAdd(W.hist + key, (uint32_t)__popc(peers));
    }
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
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_wave_first(const __grid_constant__ TraceP<T> P, WaveWork<T> W)
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
    append(P, W, W.q[1], on, p, (uint32_t)j);
    if (live && !on && P.train_log) write_log(P, i, j, p);
}

// Exclusive scan of the bucket histogram into cursors, in three launches: each block scans
// a tile of 1024 buckets in shared memory and records the tile's total; one block scans
// the totals; every bucket then adds its tile's offset.
__global__ void __launch_bounds__(1024) k_wave_scan_tiles(uint32_t *hist, uint32_t *tile_sum)
{
    __shared__ uint32_t s[1024];
    const int t = threadIdx.x;
    const size_t b = (size_t)blockIdx.x * 1024 + t;
    const uint32_t x = hist[b];
    s[t] = x;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = t >= off ? s[t - off] : 0u;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    hist[b] = s[t] - x;
    if (t == 1023) tile_sum[blockIdx.x] = s[1023];
}

// exclusive scan of the n tile totals (n a multiple of 1024), one block
__global__ void __launch_bounds__(1024) k_wave_scan_sums(uint32_t *tile_sum, int n)
{
    __shared__ uint32_t s[1024];
    const int t = threadIdx.x, per = n / 1024;
    uint32_t tot = 0;
    for (int q = 0; q < per; ++q) tot += tile_sum[t * per + q];
    s[t] = tot;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = t >= off ? s[t - off] : 0u;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    uint32_t run = s[t] - tot;
    for (int q = 0; q < per; ++q) {
        const uint32_t x = tile_sum[t * per + q];
        tile_sum[t * per + q] = run;
        run += x;
    }
}

__global__ void __launch_bounds__(1024) k_wave_scan_add(uint32_t *hist, const uint32_t *tile_sum)
{
    hist[(size_t)blockIdx.x * 1024 + threadIdx.x] += tile_sum[blockIdx.x];
}

// Bucket order of the appended records: perm[cursor of its key] = record index, one
// cursor atomic per run of equal keys in a warp.
template <class T>
__global__ void __launch_bounds__(256) k_wave_scatter(WaveWork<T> W)
{
    const uint32_t n = W.count[1];
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); q0 < n; q0 += stride) {  // uniform per warp
        const uint32_t q = q0 + lane;
        const bool v = q < n;
        const uint32_t key = v ? W.keys[q] : 0xffffffffu;
        const unsigned peers = __match_any_sync(FULL_MASK, key);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (v && lane == leader) base = atomicAdd(W.hist + key, (uint32_t)__popc(peers));
        base = __shfl_sync(FULL_MASK, base, leader);
        if (v) W.perm[base + __popc(peers & ((1u << lane) - 1u))] = q;
    }
}

// Order k >= 2 over queue q[(k + 1) & 1] in bucket order; survivors are appended to
// q[k & 1].  FP32 is held to 64 registers (4 blocks, 32 warps per SM; 7 % faster than
// at 80 registers).
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_wave_order(const __grid_constant__ TraceP<T> P, int k, WaveWork<T> W)
{
    const uint32_t n = W.count[0];
    const int lane = threadIdx.x & 31;
    Rec<T> *const src = (k & 1) ? W.q[0] : W.q[1];  // selects, not an indexed parameter array
    Rec<T> *const dst = (k & 1) ? W.q[1] : W.q[0];
    // warps claim 32-packet chunks from a counter, one chunk ahead: walk lengths differ
    // from chunk to chunk, and a warp that finishes early takes the next one (n <= 2^31,
    // so the counter, which passes n by at most two chunks per warp, cannot wrap)
    auto claim = [&]() {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(W.count + 2, 32u);
        return __shfl_sync(FULL_MASK, c, 0);
    };
    uint32_t q0 = claim();
    while (q0 < n) {  // uniform per warp
        const uint32_t q1 = claim();
        const uint32_t q = q0 + lane;
        const bool live = q < n;
        Rec<T> r;
        if (live) {
            const uint32_t qn = q1 + lane;
            const uint32_t pn = qn < n ? W.perm[qn] : 0u;
            copy_rec(&r, src + W.perm[q]);
            // the record this lane gathers next: into L2 while this one is traced
            if (qn < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(src + pn));
        } else {
            for (int c = 0; c < 3; ++c) r.p.pos[c] = r.p.n[c] = r.p.a[c] = r.p.S[c] = T(0);
            r.p.tot = r.p.tot2 = T(0);
            r.j = 0;
        }
        const uint64_t i = P.first + r.j;
        const T wd = live ? point<T>(P.pts, i, 4 * (k - 1) + 2) : T(0);
        const bool on = run_order(P, k, i, live, wd, r.p);
        append(P, W, dst, on, r.p, r.j);
        if (live && !on && P.train_log) write_log(P, i, r.j, r.p);
        q0 = q1;
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
    W.q[0] = (Rec<T> *)take(cap * sizeof(Rec<T>));
    W.q[1] = (Rec<T> *)take(cap * sizeof(Rec<T>));
    W.count = (uint32_t *)take(3 * 4);
    W.keys = (uint32_t *)take(cap * 4);
    W.perm = (uint32_t *)take(cap * 4);
    W.hist = (uint32_t *)take(WV_BUCKETS * 4 + WV_BUCKETS / 256);
    return W;
}

template <class T>
cudaError_t launch_wave(const TraceP<T> &P, void *ws, uint64_t cap, int sms, cudaStream_t s)
{
    if (P.count == 0) return cudaSuccess;
    WaveWork<T> W = carve<T>(ws, cap);
    cudaError_t e = cudaMemsetAsync(W.count, 0, 3 * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(W.hist, 0, WV_BUCKETS * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const uint64_t threads = (P.ord.threads + 31) & ~31ull;
    k_wave_first<T><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(P, W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::max(1, sms * 8);
    for (int k = 2; k <= P.max_orders; ++k) {
        // the queue appended by order k - 1 holds order k's packets with their keys and
        // histogram: their indices in bucket order into perm
        k_wave_scan_tiles<<<WV_BUCKETS / 1024, 1024, 0, s>>>(W.hist, W.hist + WV_BUCKETS);
        k_wave_scan_sums<<<1, 1024, 0, s>>>(W.hist + WV_BUCKETS, WV_BUCKETS / 1024);
        k_wave_scan_add<<<WV_BUCKETS / 1024, 1024, 0, s>>>(W.hist, W.hist + WV_BUCKETS);
        k_wave_scatter<T><<<grid, 256, 0, s>>>(W);
        if ((e = cudaMemcpyAsync(W.count, W.count + 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(W.count + 1, 0, 2 * sizeof(uint32_t), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(W.hist, 0, WV_BUCKETS * sizeof(uint32_t), s)) != cudaSuccess) return e;
        k_wave_order<T><<<grid, 256, 0, s>>>(P, k, W);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

uint64_t wavefront_workspace_bytes(uint64_t cap, int precision)
{
    const uint64_t rec = precision == QMCRT_PREC_F64 ? sizeof(Rec<double>) : sizeof(Rec<float>);
    auto pad = [](uint64_t b) { return (b + 255) & ~255ull; };
    return 2 * pad(cap * rec) + pad(12) + 2 * pad(cap * 4) + pad(WV_BUCKETS * 4 + WV_BUCKETS / 256);
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

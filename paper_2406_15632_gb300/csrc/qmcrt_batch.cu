// qmcrt_batch.cu -- many tracing problems in one persistent launch.
//
// An instance is one observer direction, one wavelength (albedo, g, p_l, opacity
// multiplier) and one packet budget over the same medium and source.  Work is cut into
// aligned chunks of 2^m point indices per instance (m = log2 of the budget, capped,
// so every chunk is as coherent as a launch of that instance alone) and each chunk
// into tiles of blockDim x packets_per_thread packets.  A fixed grid of CTAs (a few per SM) pulls
// tiles from one atomic counter, so instances with very different budgets keep every
// SM busy until the whole batch is done.  Per tile the CTA holds the instance's
// parameter block in shared memory; the packet code is the single-scattering code.
#include "qmcrt_device.cuh"

namespace qmcrt {

// Chunk size of an instance: the largest aligned block its budget fills, capped.
__device__ __forceinline__ int instance_m(const qmcrt_instance &I, int m_cap)
{
    const int lg = I.count ? 63 - __clzll((long long)I.count) : 0;
    return max(NET_MIN_M, min(lg, m_cap));
}

// Work tiles of instance i: (aligned 2^m blocks that meet [first, first + count)) x
// (tiles per block).
__device__ __forceinline__ uint64_t instance_tiles(const qmcrt_instance &I, int m_cap, uint64_t tile_packets)
{
    if (I.count == 0) return 0;
    const int m = instance_m(I, m_cap);
    const uint64_t chunks = ((I.first_index + I.count - 1) >> m) - (I.first_index >> m) + 1;
    return chunks * (((1ull << m) + tile_packets - 1) / tile_packets);
}

// Workspace: [0] tile counter, [1 .. n] tile prefix sums (prefix[i] = tiles of the
// instances before i, prefix[n] = all tiles).  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_batch_plan(const qmcrt_instance *__restrict__ inst, int n, int m_cap,
                                                    uint64_t tile_packets, unsigned long long *__restrict__ ws)
{
    __shared__ unsigned long long part[1024];
    const int t = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int a = min(n, t * per), b = min(n, a + per);
    unsigned long long s = 0;
    for (int i = a; i < b; ++i) s += instance_tiles(inst[i], m_cap, tile_packets);
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan (Hillis-Steele)
        const unsigned long long v = t >= off ? part[t - off] : 0ull;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned long long run = t ? part[t - 1] : 0ull;
    for (int i = a; i < b; ++i) {
        ws[1 + i] = run;
        run += instance_tiles(inst[i], m_cap, tile_packets);
    }
    if (t == 1023) ws[1 + n] = part[1023];
    if (t == 0) ws[0] = 0ull;
}

template <class T>
__device__ __forceinline__ void set_instance(TraceP<T> &P, const TraceP<T> &base, const qmcrt_instance &I, int index)
{
    // observer
    double st, ct, sp, cp;
    sincos(I.theta, &st, &ct);
    sincos(I.phi, &sp, &cp);
    P.obs.k[0] = (T)(st * cp);
    P.obs.k[1] = (T)(st * sp);
    P.obs.k[2] = (T)ct;
    P.obs.ex[0] = (T)(-sp);
    P.obs.ex[1] = (T)cp;
    P.obs.ex[2] = T(0);
    P.obs.ey[0] = (T)(-ct * cp);
    P.obs.ey[1] = (T)(-ct * sp);
    P.obs.ey[2] = (T)st;
    for (int a = 0; a < 3; ++a) P.obs.inv_k[a] = T(1) / P.obs.k[a];
    // a tail map holds for one direction: the instance's own, if it has one
    P.obs.tail = base.med.pad ? I.d_tail : nullptr;
    P.obs.tail_thr = tail_threshold(base.tail_eps, (double)base.med.kscale * I.kscale);
    // dust
    P.dust.albedo = (T)I.albedo;
    P.dust.g = (T)I.g;
    P.dust.p_l = (T)I.p_l;
    P.dust.one_m_g2 = (T)(1.0 - I.g * I.g);
    P.dust.one_p_g2 = (T)(1.0 + I.g * I.g);
    P.dust.two_g = (T)(2.0 * I.g);
    P.dust.isotropic = fabs(I.g) < 1e-6;
    // opacity
    P.med.kscale = (T)(base.med.kscale * I.kscale);
    P.med.inv_kscale = (T)(1.0 / ((double)base.med.kscale * I.kscale));
    P.med.sph_k = (T)((double)base.med.sph_k * I.kscale);
    // points and image (a Hammersley instance is the set of N = its last index)
    P.first = I.first_index;
    P.count = I.count;
    P.pts.total_n = I.first_index + I.count - 1;
    P.acc.ptr = (char *)base.acc.ptr + (size_t)index * 3 * base.acc.plane * sizeof(long long);
}

template <class T>
__global__ void __launch_bounds__(256) k_trace_batch(const __grid_constant__ TraceP<T> base,
                                                    const __grid_constant__ NetTables tab,
                                                    const qmcrt_instance *__restrict__ inst, int n_inst,
                                                    unsigned long long *__restrict__ ws, int per_thread)
{
    __shared__ TraceP<T> sP;
    __shared__ unsigned long long s_tile;
    __shared__ int s_inst;
    const unsigned long long tile_packets = (unsigned long long)blockDim.x * per_thread;
    const unsigned long long total_tiles = ws[1 + n_inst];
    if (threadIdx.x == 0) {
        sP = base;
        s_inst = -1;
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(ws, 1ull);
        __syncthreads();
        const unsigned long long w = s_tile;
        if (w >= total_tiles) break;
        if (threadIdx.x == 0) {
            int lo = 0, hi = n_inst - 1;  // last instance whose prefix <= w
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ws[1 + mid] <= w) lo = mid;
                else hi = mid - 1;
            }
            const qmcrt_instance I = inst[lo];
            const int m = instance_m(I, tab.m_cap);
            if (lo != s_inst) {
                set_instance(sP, base, I, lo);
                sP.ord = tab.ord[m - NET_MIN_M];
                sP.ord.m = m;
                s_inst = lo;
            }
            const unsigned long long tpc = ((1ull << m) + tile_packets - 1) / tile_packets;
            const unsigned long long local = w - ws[1 + lo];
            sP.ord.block0 = (I.first_index >> m) + local / tpc;
            if (sP.ord.net && sP.ord.g0_block != sP.ord.block0) {  // the block's term, once per tile
                sP.ord.g0 = block_columns(sP.ord, sP.ord.block0 << m);
                sP.ord.g0_block = sP.ord.block0;
            }
            sP.ord.threads = (local % tpc) * tile_packets;  // first position of this tile
        }
        __syncthreads();
        const TraceP<T> &P = sP;
        const int m = P.ord.m;
        for (int j = 0; j < per_thread; ++j) {
            const unsigned long long pos = P.ord.threads + (unsigned long long)j * blockDim.x + threadIdx.x;
            uint64_t i = 0;
            bool live = false;
            if (pos < (1ull << m)) {
                if (P.ord.net) {
                    live = packet_index(P.ord, P.first, P.count, pos, i);
                } else {
                    i = (P.ord.block0 << m) + pos;
                    live = i >= P.first && i < P.first + P.count;
                }
            }
            if (!__any_sync(FULL_MASK, live)) continue;  // uniform per warp
            T S[3] = {T(0), T(0), T(0)};
            T x = T(0), y = T(0);
            int status = 1;
            if (live) {
                T pos3[3], d[3], a[3], wgt, W1;
                const T wd = emit(P, i, pos3, d, a, wgt);
                if (forced_step(P, pos3, d, wd, W1)) {
                    const T W0 = wgt * W1 * P.dust.albedo;
                    status = peel_unpolarized(P, pos3, d, W0, S, x, y) ? 0 : 2;
                }
            }
            splat(P, status == 0, 0, x, y, S);
        }
    }
}

// out[i][s][p] = raw[i][s][p] * 2^-frac_bits / count_i  (units of the source luminosity).
__global__ void __launch_bounds__(256) k_batch_reduce(const long long *__restrict__ acc,
                                                     const qmcrt_instance *__restrict__ inst, size_t per_inst,
                                                     size_t total, double frac_scale, double *__restrict__ out)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const uint64_t c = inst[e / per_inst].count;
        out[e] = c ? (double)acc[e] * frac_scale / (double)c : 0.0;
    }
}

template <class T>
static cudaError_t launch_batch(const TraceP<T> &p, const NetTables &tab, const qmcrt_instance *inst, int n_inst,
                                unsigned long long *ws, int block, int ctas, int per_thread, cudaStream_t s)
{
    k_batch_plan<<<1, 1024, 0, s>>>(inst, n_inst, tab.m_cap, (uint64_t)block * per_thread, ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_trace_batch<T><<<ctas, block, 0, s>>>(p, tab, inst, n_inst, ws, per_thread);
    return cudaGetLastError();
}

cudaError_t launch_trace_batch_f32(const TraceP<float> &p, const NetTables &tab, const qmcrt_instance *inst,
                                   int n_inst, unsigned long long *ws, int block, int ctas, int per_thread,
                                   cudaStream_t s)
{
    return launch_batch(p, tab, inst, n_inst, ws, block, ctas, per_thread, s);
}

cudaError_t launch_trace_batch_f64(const TraceP<double> &p, const NetTables &tab, const qmcrt_instance *inst,
                                   int n_inst, unsigned long long *ws, int block, int ctas, int per_thread,
                                   cudaStream_t s)
{
    return launch_batch(p, tab, inst, n_inst, ws, block, ctas, per_thread, s);
}

cudaError_t launch_batch_reduce(const long long *acc, const qmcrt_instance *inst, int n_inst, size_t per_inst,
                                double frac_scale, double *out, cudaStream_t s)
{
    const size_t total = per_inst * (size_t)n_inst;
    if (total == 0) return cudaSuccess;
    size_t g = (total + 255) / 256;
    if (g > 152 * 64) g = 152 * 64;
    k_batch_reduce<<<(unsigned)g, 256, 0, s>>>(acc, inst, per_inst, total, frac_scale, out);
    return cudaGetLastError();
}

int batch_occupancy(int block, int precision)
{
    int n = 0;
    if (precision == QMCRT_PREC_F64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_batch<double>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_batch<float>, block, 0);
    return n;
}

}  // namespace qmcrt

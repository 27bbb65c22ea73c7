// qmcrt_trace_multiple.cu -- multiple-scattering tracer kernel (Sec. 3.5, 3.7).
//
// One thread per packet, the same warp-coherent packet mapping as the single-
// scattering kernel.  With a learned warp the first-order coordinates come from a
// buffer (x = T(u) and log |dx/du| per packet); the optional training log records,
// per packet, the coordinates used and two norms of the intensities its peel-offs put
// into the image (their sum, and the square root of their sum of squares).
// Order k reads coordinates 4(k-1) + {0 azimuth, 1 cos Theta, 2 depth, 3 roulette};
// the order loop is uniform across the warp so deposits stay
// convergent, and the warp leaves the loop once all its packets are done.
#include "qmcrt_device.cuh"

namespace qmcrt {

template <class T>
__global__ void __launch_bounds__(256) k_trace_multiple(const __grid_constant__ TraceP<T> P)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((tid & ~31ull) >= P.ord.threads) return;  // uniform per warp
    uint64_t i = P.first;
    const bool live_index = packet_index(P.ord, P.first, P.count, tid, i);
    if (!__any_sync(FULL_MASK, live_index)) return;
    bool alive = live_index;
    T pos[3] = {T(0), T(0), T(0)}, n[3] = {T(0), T(0), T(1)}, a[3] = {T(1), T(0), T(0)};
    T S[3] = {T(0), T(0), T(0)};
    T wd = T(0), total = T(0), total2 = T(0);
    const uint64_t j = i - P.first;
    if (alive) {
        T wgt;
        if (P.warp_x) {  // learned proposal: first-order coordinates and their Jacobian
            T sp, cp;
            direction_from((T)P.warp_x[3 * j], (T)P.warp_x[3 * j + 1], n, a, sp, cp);
            pos[0] = pos[1] = pos[2] = T(0);
            wd = (T)P.warp_x[3 * j + 2];
            wgt = Mth<T>::exp_((T)P.warp_logj[j]);
        } else {
            wd = emit(P, i, pos, n, a, wgt);
        }
        S[0] = wgt;
    }
    for (int k = 1; k <= P.max_orders; ++k) {
        if (!__any_sync(FULL_MASK, alive)) break;
        const int base = 4 * (k - 1);
        T out[3] = {T(0), T(0), T(0)};
        T x = T(0), y = T(0);
        bool contrib = false;
        if (alive) {
            if (k > 1) {
                scatter(P.dust, point<T>(P.pts, i, base), point<T>(P.pts, i, base + 1), n, a, S);
                wd = point<T>(P.pts, i, base + 2);
            }
            if (k == 1 || P.force_all) {
                T W1;
                if (forced_step(P, pos, n, wd, W1)) {
                    S[0] *= W1;
                    S[1] *= W1;
                    S[2] *= W1;
                } else {
                    alive = false;
                }
            } else if (!march(P.med, pos, n, -Mth<T>::log_(wd))) {
                alive = false;
            }
            if (alive) {
                S[0] *= P.dust.albedo;
                S[1] *= P.dust.albedo;
                S[2] *= P.dust.albedo;
                contrib = peel_polarized(P, pos, n, a, S, out, x, y);
                if (contrib && x >= -P.obs.hw && x < P.obs.hw && y >= -P.obs.hw && y < P.obs.hw) {
                    total += out[0];
                    total2 += out[0] * out[0];
                }
            }
        }
        splat(P, contrib, P.per_order ? k - 1 : 0, x, y, out);
        if (alive) {
            if (k == P.max_orders) {
                alive = false;
            } else if (S[0] < P.rr_threshold) {
                if (point<T>(P.pts, i, base + 3) < P.rr_survival) {
                    S[0] /= P.rr_survival;
                    S[1] /= P.rr_survival;
                    S[2] /= P.rr_survival;
                } else {
                    alive = false;
                }
            }
        }
    }
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
        r[3] = (float)total;
        r[4] = (float)Mth<T>::sqrt_(total2);
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

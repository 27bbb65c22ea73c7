// qmcrt_internal.h -- kernel parameter blocks and launcher declarations shared by the
// host-side ABI (qmcrt_api.cu) and the kernel translation units.  Every block is
// passed to its kernel by value (one constant-bank parameter, no device allocation).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "qmcrt.h"

namespace qmcrt {

// Point set of Sec. 3.1.  Indices are global point indices (>= 1).
struct PointsP {
    int kind;          // QMCRT_SOBOL .. QMCRT_FAURE
    int dims;
    uint32_t faure_b;  // Faure base: the smallest prime >= dims
    uint64_t seed;
    uint64_t total_n;  // Hammersley N
    double inv_total_n;
};

// Medium of Sec. 3.4.  Grid cells hold kappa*rho; walks compare sums of cell values
// (without kscale) against optical depths divided by kscale, which saves a multiply
// per cell step.
template <class T>
struct MediumP {
    const float *k;
    int kind;          // QMCRT_MEDIUM_GRID / QMCRT_MEDIUM_SPHERE
    int n[3];
    int pad;           // sentinel layers around the grid (0: plain grid, walked with cell counters)
    int stride[3];     // linear index step of one cell along x, y, z (of the padded array if pad > 0)
    T lo[3], hi[3], h[3];
    T inv_h[3];        // 1 / h: the first estimate of a start cell
    T kscale, inv_kscale;
    T sph_r, sph_k;    // analytic sphere: radius, kscale * extinction
    const double *sky; // optional bound map (qmcrt_sky_bound), sky_m texels per edge, for rays that start
    int sky_m;         // within sky_r2 = R^2 of the origin
    T sky_r2;
};

template <class T>
struct SourceP {
    int kind;          // QMCRT_SOURCE_*
    int order;         // QMCRT_ORDER_*
    T R;
    T limb_u, limb_norm;  // weight (1 - u + u mu) * limb_norm, limb_norm = 1 / (1 - u/3)
};

template <class T>
struct DustP {
    T albedo, g, p_l;
    T one_m_g2, one_p_g2, two_g;  // 1 - g^2, 1 + g^2, 2 g
    int isotropic;                // |g| < 1e-6: cos Theta = 2 v - 1
};

template <class T>
struct ObsP {
    T k[3], ex[3], ey[3];  // direction toward the observer and sky axes
    T inv_k[3];            // 1 / k (the peel-off walk's face distances), rounded as the device rounds T(1) / k
    T hw;                  // half width of the image
    T pix_x, pix_y;        // pixels per unit sky length: n / (2 hw)
    int nx, ny, splat;
    const uint8_t *tail;   // optional qmcrt_tail_map codes for k on the padded grid (NULL: walk to the edge)
    int tail_thr;          // a peel-off walk stops after a batch whose first cell's code is <= this
};

struct AccumP {
    void *ptr;         // [n_images][3][ny][nx] int64 or double
    int mode;          // QMCRT_ACCUM_*
    int n_images;
    double scale;      // 2^frac_bits (I64)
    size_t plane;      // nx * ny
};

// Packet order.  Linear: thread t traces point first + t.  Net order (Sobol kinds):
// the index range is covered by aligned blocks of 2^m indices, and inside a block
// thread t traces the point whose leading (a, b, c) bits of coordinates (0, 1, 2)
// form the t-th elementary box in Morton order (2^tt points per box, tt = the
// t-value of the chosen split).  With y(i) the vector of those leading bits and g the
// Gray code of the index inside the block, y(i) = y(block start) ^ L g over GF(2);
// the host inverts L: g = R (y ^ y(block start)) ^ K e, e selecting within the box.
// Consecutive threads, hence a warp, receive points from adjacent boxes: packets that
// start in nearly the same direction and scatter at nearly the same depth.
constexpr int NET_MAX_M = 28;

constexpr int NET_MAX_TT = 6;  // points per elementary box up to 2^6

struct OrderP {
    int net;            // 0 linear, 1 net order of Sobol (Gray code), 2 of Niederreiter (natural order)
    int m, bits, tt;    // block 2^m, bits = m - tt Morton bits, tt kernel bits
    int nb[5];          // leading bits taken from coordinates 0, 1, 2, xdim[0], xdim[1]
    int xdim[2];        // the two further coordinates ordered (a finite star's emission point)
    uint64_t block0;    // first block index
    uint64_t threads;   // threads to launch (count when linear)
    uint32_t rm[NET_MAX_M];  // R column for Morton bit j of the thread's box index
    uint32_t ry[NET_MAX_M];  // R column for bit j of y
    uint32_t k[NET_MAX_TT];  // kernel basis of L
    uint64_t g0_block;       // a block whose y part is precomputed (the launch's first)
    uint32_t g0;             // XOR of ry over the bits of that block's y
};

// Net-order tables for every block size a batch may use (m = NET_MIN_M .. NET_MAX_M).
constexpr int NET_MIN_M = 7;
struct NetTables {
    OrderP ord[NET_MAX_M - NET_MIN_M + 1];
    int m_cap;           // largest chunk a batch uses: instance i takes min(floor(log2 count_i), m_cap)
};

template <class T>
struct TraceP {
    OrderP ord;
    MediumP<T> med;
    SourceP<T> src;
    DustP<T> dust;
    ObsP<T> obs;
    PointsP pts;
    AccumP acc;
    T tau_min;
    uint64_t first;    // first point index
    uint64_t count;    // packets
    double *log;       // optional [count][9]
    const float *warp_x;     // optional [count][3]: first-order coordinates (learned warp)
    const float *warp_logj;  // [count] log |dx/du| of warp_x (multiplies the packet weight)
    float *train_log;        // optional [count][4]: coordinates used, total peel-off intensity
    int max_orders, force_all, per_order;
    T rr_threshold, rr_survival, inv_rr_survival;
    double tail_eps;         // peel-off depth a tail map lets a walk leave out (with kscale)
};

// Observers fed by one trace (qmcrt_trace_observers); image o is the stack that
// starts o * stack values into the accumulator.
template <class T>
struct ObsSet {
    int n;
    size_t stack;  // values per observer: n_images * 3 * nx * ny
    ObsP<T> o[QMCRT_MAX_OBSERVERS];
};

cudaError_t launch_trace_observers_f32(const TraceP<float> &p, const ObsSet<float> &obs, int block, cudaStream_t s);
cudaError_t launch_trace_observers_f64(const TraceP<double> &p, const ObsSet<double> &obs, int block, cudaStream_t s);

cudaError_t launch_direct_light_f32(const TraceP<float> &p, int subsamples, double weight, cudaStream_t s);
cudaError_t launch_direct_light_f64(const TraceP<double> &p, int subsamples, double weight, cudaStream_t s);

uint64_t wavefront_workspace_bytes(uint64_t cap, int precision);
cudaError_t launch_trace_wavefront_f32(const TraceP<float> &p, void *ws, uint64_t cap, int sms, cudaStream_t s);
cudaError_t launch_trace_wavefront_f64(const TraceP<double> &p, void *ws, uint64_t cap, int sms, cudaStream_t s);

struct GemmEpi;
cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int splits,
                             const GemmEpi &ep, cudaStream_t s);

// Records a message for qmcrt_last_error() on the calling thread; returns code.
int set_error(int code, const char *fmt, ...);

// The status qmcrt_trace_single would return for these arguments, from its host-side
// checks alone (nothing is enqueued).
int check_trace_single(const qmcrt_medium *md, const qmcrt_source *src, const qmcrt_dust *du,
                       const qmcrt_observer *ob, const qmcrt_points_desc *pts, const qmcrt_trace_opts *op,
                       const qmcrt_image *im);

// Launchers (return a cudaError_t from the launch).
cudaError_t launch_trace_batch_f32(const TraceP<float> &p, const NetTables &tab, const qmcrt_instance *inst,
                                   int n_inst, unsigned long long *ws, int block, int ctas, int per_thread,
                                   cudaStream_t s);
cudaError_t launch_trace_batch_f64(const TraceP<double> &p, const NetTables &tab, const qmcrt_instance *inst,
                                   int n_inst, unsigned long long *ws, int block, int ctas, int per_thread,
                                   cudaStream_t s);
cudaError_t launch_batch_reduce(const long long *acc, const qmcrt_instance *inst, int n_inst, size_t per_inst,
                                double frac_scale, double *out, cudaStream_t s);
int batch_occupancy(int block, int precision);

// Forward pass of the learned warp, both conditionals fused on the tensor cores.
cudaError_t launch_warp_forward_fused(const float *params, const __nv_bfloat16 *wb, const float *u, float *x,
                                      float *logj, long long n, float mix, int *error, cudaStream_t s);
cudaError_t launch_generate_points(const PointsP &p, uint64_t first, uint64_t count, int format, void *out,
                                   cudaStream_t s);
cudaError_t launch_pad_grid(const float *k, int nx, int ny, int nz, int pad, float *out, cudaStream_t s);
cudaError_t launch_sky_bound(const float *k, int nx, int ny, int nz, const double lo[3], const double hi[3],
                             double radius, int m, double *map, void *ws, cudaStream_t s);
int sky_dilation(const double lo[3], const double hi[3], int nx, int ny, int nz, double radius);
uint64_t sky_workspace_bytes(int nx, int ny, int nz, int D);

// qmcrt_tail.cu: codes of a tail map (qmcrt_tail_map) for direction k over a padded grid
constexpr int TAIL_BLOCK = 4;  // cells per block edge
uint64_t tail_workspace_bytes(int nx, int ny, int nz);
cudaError_t launch_tail_map(const float *k_padded, int nx, int ny, int nz, int pad, const double lo[3],
                            const double hi[3], const double dir[3], uint8_t *map, void *ws, cudaStream_t s);
// Largest code a walk may stop at for a depth tolerance eps (with kscale): 0 when eps is 0.
__host__ __device__ inline int tail_threshold(double eps, double kscale)
{
    if (!(eps > 0)) return 0;
    int e;
    frexp(eps / kscale, &e);  // eps / kscale = m 2^e, 1/2 <= m < 1: 2^(e-1) <= it
    const int c = e - 1 + 150;
    return c < 0 ? 0 : (c > 254 ? 254 : c);
}
cudaError_t launch_image_reduce(const void *acc, int mode, double frac_scale, size_t elems, int replicas,
                                double scale, double *out, cudaStream_t s);
cudaError_t launch_trace_single_f32(const TraceP<float> &p, int block, cudaStream_t s);
cudaError_t launch_trace_single_f64(const TraceP<double> &p, int block, cudaStream_t s);
cudaError_t launch_trace_multiple_f32(const TraceP<float> &p, int block, cudaStream_t s);
cudaError_t launch_trace_multiple_f64(const TraceP<double> &p, int block, cudaStream_t s);

}  // namespace qmcrt

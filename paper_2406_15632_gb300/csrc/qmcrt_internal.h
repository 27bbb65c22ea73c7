// qmcrt_internal.h -- kernel parameter blocks and launcher declarations shared by the
// host-side ABI (qmcrt_api.cu) and the kernel translation units.  Every block is
// passed to its kernel by value (one constant-bank parameter, no device allocation).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace qmcrt {

// Point set of Sec. 3.1.  Indices are global point indices (>= 1).
struct PointsP {
    int kind;          // QMCRT_SOBOL .. QMCRT_PHILOX
    int dims;
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
    int stride[3];     // linear index step of one cell along x, y, z
    T lo[3], hi[3], h[3];
    T kscale, inv_kscale;
    T sph_r, sph_k;    // analytic sphere: radius, kscale * extinction
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
    T hw;                  // half width of the image
    T pix_x, pix_y;        // pixels per unit sky length: n / (2 hw)
    int nx, ny, splat;
};

struct AccumP {
    void *ptr;         // [n_images][3][ny][nx] int64 or double
    int mode;          // QMCRT_ACCUM_*
    int n_images;
    double scale;      // 2^frac_bits (I64)
    size_t plane;      // nx * ny
};

template <class T>
struct TraceP {
    MediumP<T> med;
    SourceP<T> src;
    DustP<T> dust;
    ObsP<T> obs;
    PointsP pts;
    AccumP acc;
    T tau_min;
    uint64_t first;    // first point index
    uint64_t count;    // packets
    uint64_t stride;   // lane stride: ceil(count / 32); lane l of warp task w traces first + l*stride + w
    double *log;       // optional [count][9]
    int max_orders, force_all, per_order;
    T rr_threshold, rr_survival, inv_rr_survival;
};

// Launchers (return a cudaError_t from the launch).
cudaError_t launch_generate_points(const PointsP &p, uint64_t first, uint64_t count, int format, void *out,
                                   cudaStream_t s);
cudaError_t launch_image_reduce(const void *acc, int mode, double frac_scale, size_t elems, int replicas,
                                double scale, double *out, cudaStream_t s);
cudaError_t launch_trace_single_f32(const TraceP<float> &p, int block, cudaStream_t s);
cudaError_t launch_trace_single_f64(const TraceP<double> &p, int block, cudaStream_t s);
cudaError_t launch_trace_multiple_f32(const TraceP<float> &p, int block, cudaStream_t s);
cudaError_t launch_trace_multiple_f64(const TraceP<double> &p, int block, cudaStream_t s);

}  // namespace qmcrt

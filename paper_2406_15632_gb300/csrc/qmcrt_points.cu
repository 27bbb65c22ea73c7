// qmcrt_points.cu -- point-set generation (Sec. 3.1), the final image reduction
// (Sec. 3.6: sums of all replicas, in units of the source luminosity) and the padded
// copy of a density grid.
#include "qmcrt_device.cuh"

namespace qmcrt {

// One thread per output element of the row-major [count][dims] block: consecutive
// threads write consecutive addresses.
__global__ void __launch_bounds__(256) k_generate_points(const __grid_constant__ PointsP P, uint64_t first,
                                                        uint64_t count, int format, void *out)
{
    const uint64_t total = count * (uint64_t)P.dims;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = e / (uint64_t)P.dims;
        const int d = (int)(e - j * (uint64_t)P.dims);
        const uint64_t i = first + j;
        if (format == QMCRT_FMT_U32) {
            ((uint32_t *)out)[e] = point_u32(P, i, d);
        } else if (format == QMCRT_FMT_F32) {
            ((float *)out)[e] = point<float>(P, i, d);
        } else {
            ((double *)out)[e] = point_f64(P, i, d);
        }
    }
}

__global__ void __launch_bounds__(256) k_image_reduce(const void *acc, int mode, double frac_scale, size_t elems,
                                                     int replicas, double scale, double *out)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < elems; e += (size_t)gridDim.x * blockDim.x) {
        if (mode == QMCRT_ACCUM_I64) {
            const long long *a = (const long long *)acc;
            long long s = 0;
            for (int r = 0; r < replicas; ++r) s += a[(size_t)r * elems + e];
            out[e] = (double)s * frac_scale * scale;
        } else {
            const double *a = (const double *)acc;
            double s = 0.0;
            for (int r = 0; r < replicas; ++r) s += a[(size_t)r * elems + e];
            out[e] = s * scale;
        }
    }
}

// Copy of a grid with `pad` layers of sentinel cells (-1) on every side.
__global__ void __launch_bounds__(256) k_pad_grid(const float *__restrict__ k, int nx, int ny, int nz, int pad,
                                                 float *__restrict__ out)
{
    const int px = nx + 2 * pad, py = ny + 2 * pad, pz = nz + 2 * pad;
    const size_t total = (size_t)px * py * pz;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(e % px) - pad;
        const int y = (int)((e / px) % py) - pad;
        const int z = (int)(e / ((size_t)px * py)) - pad;
        const bool in = x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz;
        // interior: the density, with empty, negative and NaN cells as +0 (no sign bit);
        // padding: the sentinel -0.0, whose sign bit ends a padded walk
        const float v = in ? k[((size_t)z * ny + y) * nx + x] : 0.0f;
        out[e] = in ? (v > 0.0f ? v : 0.0f) : -0.0f;
    }
}

static unsigned grid_for(uint64_t n)
{
    uint64_t g = (n + 255) / 256;
    if (g > 152ull * 64) g = 152ull * 64;  // grid-stride beyond 64 blocks per SM
    return (unsigned)(g ? g : 1);
}

cudaError_t launch_generate_points(const PointsP &p, uint64_t first, uint64_t count, int format, void *out,
                                   cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    k_generate_points<<<grid_for(count * (uint64_t)p.dims), 256, 0, s>>>(p, first, count, format, out);
    return cudaGetLastError();
}

cudaError_t launch_pad_grid(const float *k, int nx, int ny, int nz, int pad, float *out, cudaStream_t s)
{
    const uint64_t total = (uint64_t)(nx + 2 * pad) * (ny + 2 * pad) * (nz + 2 * pad);
    k_pad_grid<<<grid_for(total), 256, 0, s>>>(k, nx, ny, nz, pad, out);
    return cudaGetLastError();
}

cudaError_t launch_image_reduce(const void *acc, int mode, double frac_scale, size_t elems, int replicas,
                                double scale, double *out, cudaStream_t s)
{
    if (elems == 0) return cudaSuccess;
    k_image_reduce<<<grid_for(elems), 256, 0, s>>>(acc, mode, frac_scale, elems, replicas, scale, out);
    return cudaGetLastError();
}

}  // namespace qmcrt

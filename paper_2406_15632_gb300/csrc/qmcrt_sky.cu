// qmcrt_sky_bound: for rays that start within a radius R of the origin (a point source,
// R = 0, or the surface of a star of radius R), an upper bound on the optical depth of every
// ray whose direction falls in each texel of a cube map.  A packet whose direction's bound
// is below the forcing threshold tau_min cannot scatter (Sec. 3.2: rays with tau_1 < tau_min
// are skipped), so the tracer decides that from one lookup instead of walking its ray
// through the grid; the decision, and hence the image, is the walk's.
//
// Cube map: face f = 2 a + (d_a < 0) for the major axis a of the direction (ties to the
// lower axis); on it u, v are the other two components (in increasing axis order) divided
// by |d_a|, in [-1, 1]; texel (iu, iv) = floor((u + 1) / 2 m), floor((v + 1) / 2 m).
#include "qmcrt.h"
#include "qmcrt_internal.h"

namespace qmcrt {

namespace {

// Every cell with kappa rho > 0 adds kappa rho times its longest chord (the diagonal) to
// the texels of all directions from the origin that pass through its box grown by R on
// every side: on each face, the box of (u, v) that grown box subtends, widened by one texel
// on every side (the tracer's float directions and cell faces differ from these double
// values by far less than a texel).  A ray p + t d with |p| <= R that meets the cell at t
// has t d in the cell shifted by -p, inside the grown box: its direction is splatted.
// A cell that reaches the major axis' zero plane subtends directions up to the face's
// edge on the side where its other coordinates lie.  A ray crosses each cell at most once,
// over at most the diagonal, so the sum over the cells it crosses -- all of them splatted
// onto its texel -- bounds its optical depth.
__global__ void __launch_bounds__(256) k_sky_bound(const float *__restrict__ k, int nx, int ny, int nz, double lo0,
                                                   double lo1, double lo2, double h0, double h1, double h2, int m,
                                                   double chord, double grow, double *map)
{
    const long long cells = (long long)nx * ny * nz;
    const double lo[3] = {lo0, lo1, lo2}, h[3] = {h0, h1, h2};
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (long long)gridDim.x * blockDim.x) {
        const float kc = k[c];
        if (!(kc > 0.0f)) continue;
        const int idx[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
        double b0[3], b1[3];
        for (int a = 0; a < 3; ++a) {
            b0[a] = lo[a] + idx[a] * h[a] - grow;
            b1[a] = lo[a] + (idx[a] + 1) * h[a] + grow;
        }
        const double add = (double)kc * chord;
        for (int f = 0; f < 6; ++f) {
            const int a = f >> 1;
            const double s = (f & 1) ? -1.0 : 1.0;
            const double w0 = fmin(s * b0[a], s * b1[a]), w1 = fmax(s * b0[a], s * b1[a]);
            if (w1 <= 0.0) continue;  // the cell lies behind this face's half space
            const int ab = a == 0 ? 1 : 0, ac = a == 2 ? 1 : 2;
            double r[2][2];  // [u, v][min, max] of the component ratio over the cell's part with w > 0
            const int oth[2] = {ab, ac};
            const double inf = __longlong_as_double(0x7ff0000000000000ll);
            for (int q = 0; q < 2; ++q) {
                const int o = oth[q];
                // x_o / w is smallest at the smallest x_o with the largest w if x_o >= 0, else
                // with the smallest w (unbounded when the cell reaches w = 0), and likewise
                // for the largest
                r[q][0] = b0[o] >= 0.0 ? b0[o] / w1 : (w0 > 0.0 ? b0[o] / w0 : -inf);
                r[q][1] = b1[o] <= 0.0 ? b1[o] / w1 : (w0 > 0.0 ? b1[o] / w0 : inf);
            }
            if (r[0][0] > 1.0 || r[0][1] < -1.0 || r[1][0] > 1.0 || r[1][1] < -1.0) continue;
            int lo_t[2], hi_t[2];
            for (int q = 0; q < 2; ++q) {
                const double mn = fmax(r[q][0], -1.0), mx = fmin(r[q][1], 1.0);
                lo_t[q] = max(0, (int)floor((mn + 1.0) * 0.5 * m) - 1);
                hi_t[q] = min(m - 1, (int)floor((mx + 1.0) * 0.5 * m) + 1);
            }
            for (int iv = lo_t[1]; iv <= hi_t[1]; ++iv)
                for (int iu = lo_t[0]; iu <= hi_t[0]; ++iu) atomicAdd(map + ((size_t)f * m + iv) * m + iu, add);
        }
    }
}

}  // namespace

cudaError_t launch_sky_bound(const float *k, int nx, int ny, int nz, const double lo[3], const double hi[3],
                             double radius, int m, double *map, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(map, 0, (size_t)6 * m * m * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const double h0 = (hi[0] - lo[0]) / nx, h1 = (hi[1] - lo[1]) / ny, h2 = (hi[2] - lo[2]) / nz;
    const double chord = sqrt(h0 * h0 + h1 * h1 + h2 * h2);
    const long long cells = (long long)nx * ny * nz;
    const unsigned grid = (unsigned)min((cells + 255) / 256, 152LL * 32);
    k_sky_bound<<<grid, 256, 0, s>>>(k, nx, ny, nz, lo[0], lo[1], lo[2], h0, h1, h2, m, chord, radius, map);
    return cudaGetLastError();
}

}  // namespace qmcrt

// qmcrt_sky.cu -- qmcrt_sky_bound: for rays that start within a radius R of the origin (a
// point source, R = 0, or the surface of a star of radius R), an upper bound on the
// optical depth of every ray whose direction falls in each texel of a cube map.  A packet
// whose direction's bound is below the forcing threshold tau_min cannot scatter (Sec. 3.2:
// rays with tau_1 < tau_min are skipped), so the tracer decides that from one lookup
// instead of walking its ray through the grid; the decision, and hence the image, is the
// walk's.
//
// Cube map: face f = 2 a + (d_a < 0) for the major axis a of the direction (ties to the
// lower axis); on it u, v are the other two components (in increasing axis order) divided
// by |d_a|, in [-1, 1]; texel (iu, iv) = floor((u + 1) / 2 m), floor((v + 1) / 2 m).
//
// Construction.  A ray p + t v with |p| <= R and v in a texel stays within R + t alpha of
// the texel's centre ray t u (alpha: the largest angle between u and the texel's corners),
// so as long as R + t alpha <= D h_min inside the grid, the cell it is in at any t is within
// D cells, in every axis, of the cell the centre ray is in at the same t.  With K_D the grid
// maximised over (2 D + 1)^3 neighbourhoods (on the grid grown by D layers), the ray's
// optical depth is at most the integral of K_D along the centre ray through the grown box:
// one walk per texel.  A texel whose cone outgrows the neighbourhoods gets an infinite bound
// (its rays are always walked).
#include <algorithm>
#include <cmath>

#include "qmcrt.h"
#include "qmcrt_internal.h"

namespace qmcrt {

namespace {

// One pass of the separable maximum filter: out = max over the 2D + 1 values of `in`
// along axis `ax` around each cell of the grown grid [nz + 2D][ny + 2D][nx + 2D].  In the
// first pass `in` is the grid itself (read at the offset -D, zero outside it); only values
// kappa rho > 0 raise the maximum (zero, negative and NaN cells count as empty, as in the
// padded grid the walk reads).
__global__ void __launch_bounds__(256) k_max_filter(const float *__restrict__ in, float *__restrict__ out, int nx,
                                                    int ny, int nz, int D, int ax, int first)
{
    const int gx = nx + 2 * D, gy = ny + 2 * D, gz = nz + 2 * D;
    const long long total = (long long)gx * gy * gz;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % gx), y = (int)((c / gx) % gy), z = (int)(c / ((long long)gx * gy));
        float m = 0.0f;
        for (int o = -D; o <= D; ++o) {
            int q[3] = {x, y, z};
            q[ax] += o;
            float v;
            if (first) {
                const int i = q[0] - D, j = q[1] - D, k = q[2] - D;
                v = (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz) ? in[((long long)k * ny + j) * nx + i]
                                                                                 : 0.0f;
            } else {
                v = (q[0] >= 0 && q[0] < gx && q[1] >= 0 && q[1] < gy && q[2] >= 0 && q[2] < gz)
                        ? in[((long long)q[2] * gy + q[1]) * gx + q[0]]
                        : 0.0f;
            }
            if (v > m) m = v;
        }
        out[c] = m;
    }
}

struct SkyGeom {
    double lo[3], h[3];  // the grid proper
    int n[3], D;
    double hmin, R, tmax;  // smallest cell edge, start radius, longest path inside the grid
    int m;
};

// Direction of face f at face coordinates (u, v), not normalised.
__device__ __forceinline__ void face_dir(int f, double u, double v, double d[3])
{
    const int a = f >> 1;
    const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
    d[a] = (f & 1) ? -1.0 : 1.0;
    d[b] = u;
    d[c] = v;
}

__global__ void __launch_bounds__(256) k_sky_walk(const float *__restrict__ K, SkyGeom g, double *map)
{
    const int m = g.m;
    const long long texels = 6LL * m * m;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    const int gn[3] = {g.n[0] + 2 * g.D, g.n[1] + 2 * g.D, g.n[2] + 2 * g.D};
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < texels;
         t += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(t / ((long long)m * m)), iv = (int)((t / m) % m), iu = (int)(t % m);
        const double du = 2.0 / m, u0 = -1.0 + iu * du, v0 = -1.0 + iv * du;
        double u[3];
        face_dir(f, u0 + 0.5 * du, v0 + 0.5 * du, u);
        const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int a = 0; a < 3; ++a) u[a] /= un;
        // the texel is a convex patch of the face: its directions lie within the largest
        // angle between u and its corners
        double cmin = 1.0;
        for (int k = 0; k < 4; ++k) {
            double w[3];
            face_dir(f, u0 + (k & 1) * du, v0 + (k >> 1) * du, w);
            const double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            cmin = fmin(cmin, (u[0] * w[0] + u[1] * w[1] + u[2] * w[2]) / wn);
        }
        const double alpha = acos(fmax(fmin(cmin, 1.0), -1.0)) * (1.0 + 1e-6) + 1e-12;
        // the walk below runs in float: its cell boundaries (face distances recomputed from
        // the cell index at every step, never accumulated) sit within 1e-6 of the medium of
        // the exact ones, taken off the room the neighbourhoods leave
        if (g.R + g.tmax * alpha > g.D * g.hmin - 1e-6 * (1.0 + g.tmax)) {
            map[t] = inf;
            continue;
        }
        // the centre ray from the origin through the grown box [blo, bhi]
        double blo[3], bhi[3], t0 = 0.0, t1 = inf;
        bool miss = false;
        for (int a = 0; a < 3; ++a) {
            blo[a] = g.lo[a] - g.D * g.h[a];
            bhi[a] = g.lo[a] + (g.n[a] + g.D) * g.h[a];
            if (u[a] != 0.0) {
                double ta = blo[a] / u[a], tb = bhi[a] / u[a];
                if (ta > tb) {
                    const double x = ta;
                    ta = tb;
                    tb = x;
                }
                t0 = fmax(t0, ta);
                t1 = fmin(t1, tb);
            } else if (0.0 < blo[a] || 0.0 >= bhi[a]) {
                miss = true;
            }
        }
        float sum = 0.0f;
        if (!miss && t1 > t0) {
            int c[3], step[3];
            float face0[3], hf[3], iu_[3], next[3];
            for (int a = 0; a < 3; ++a) {
                // a start on a face may pick the cell on either side: K_D of either bounds
                // the other's cell (D >= 1), and a wrong side is left after a zero length
                c[a] = min(max((int)floor((t0 * u[a] - blo[a]) / g.h[a]), 0), gn[a] - 1);
                step[a] = u[a] > 0.0 ? 1 : u[a] < 0.0 ? -1 : 0;
                face0[a] = (float)(blo[a] + (u[a] > 0.0 ? g.h[a] : 0.0));  // exit face of cell 0
                hf[a] = (float)g.h[a];
                iu_[a] = u[a] != 0.0 ? (float)(1.0 / u[a]) : 0.0f;
                next[a] = step[a] ? (face0[a] + (float)c[a] * hf[a]) * iu_[a] : __int_as_float(0x7f800000);
            }
            float tc = (float)t0;
            const float tend = (float)t1;
            while (tc < tend) {
                int a = 0;
                if (next[1] < next[a]) a = 1;
                if (next[2] < next[a]) a = 2;
                const float te = fminf(next[a], tend);
                sum += K[((long long)c[2] * gn[1] + c[1]) * gn[0] + c[0]] * fmaxf(te - tc, 0.0f);
                tc = fmaxf(tc, te);
                c[a] += step[a];
                if (c[a] < 0 || c[a] >= gn[a]) break;
                next[a] = (face0[a] + (float)c[a] * hf[a]) * iu_[a];
            }
        }
        // the cone ray and the centre ray cover equal lengths per t: the margin covers the
        // float rounding of the segments and of the sum (a few hundred terms); the tracer's
        // test keeps a further factor of two
        map[t] = (double)sum * (1.0 + 1e-4);
    }
}

}  // namespace

int sky_dilation(const double lo[3], const double hi[3], int nx, int ny, int nz, double radius)
{
    const double hmin = std::min((hi[0] - lo[0]) / nx, std::min((hi[1] - lo[1]) / ny, (hi[2] - lo[2]) / nz));
    return 1 + (int)std::ceil(radius / hmin);
}

uint64_t sky_workspace_bytes(int nx, int ny, int nz, int D)
{
    const uint64_t cells = (uint64_t)(nx + 2 * D) * (ny + 2 * D) * (nz + 2 * D);
    return 2 * ((cells * 4 + 255) & ~255ull);
}

cudaError_t launch_sky_bound(const float *k, int nx, int ny, int nz, const double lo[3], const double hi[3],
                             double radius, int m, double *map, void *ws, cudaStream_t s)
{
    const int D = sky_dilation(lo, hi, nx, ny, nz, radius);
    const uint64_t cells = (uint64_t)(nx + 2 * D) * (ny + 2 * D) * (nz + 2 * D);
    float *A = (float *)ws;
    float *B = (float *)((char *)ws + ((cells * 4 + 255) & ~255ull));
    const unsigned grid = (unsigned)std::min<uint64_t>((cells + 255) / 256, 152ull * 32);
    k_max_filter<<<grid, 256, 0, s>>>(k, A, nx, ny, nz, D, 0, 1);
    k_max_filter<<<grid, 256, 0, s>>>(A, B, nx, ny, nz, D, 1, 0);
    k_max_filter<<<grid, 256, 0, s>>>(B, A, nx, ny, nz, D, 2, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SkyGeom g;
    g.D = D;
    g.m = m;
    g.R = radius;
    const int n[3] = {nx, ny, nz};
    g.hmin = 1e300;
    double far2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = lo[a];
        g.n[a] = n[a];
        g.h[a] = (hi[a] - lo[a]) / n[a];
        g.hmin = std::min(g.hmin, g.h[a]);
        const double ext = std::max(std::fabs(lo[a]), std::fabs(hi[a])) + radius;
        far2 += ext * ext;
    }
    g.tmax = std::sqrt(far2);  // from within R of the origin to the farthest point of the grid
    const long long texels = 6LL * m * m;
    const unsigned tgrid = (unsigned)std::min<long long>((texels + 255) / 256, 152LL * 32);
    k_sky_walk<<<tgrid, 256, 0, s>>>(A, g, map);
    return cudaGetLastError();
}

}  // namespace qmcrt

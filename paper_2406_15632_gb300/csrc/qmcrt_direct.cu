// qmcrt_direct.cu -- direct (unscattered) light of the source, integrated from the
// source toward the observer (Sec. 3.4), Stokes I only.
//
// Point source: one value e^-tau(0 -> observer) / (4 pi), binned at the sky origin.
// Finite star: one thread per (pixel, subsample) of the pixels the stellar disk can
// touch; each evaluates the limb-darkened surface brightness at its sky point, walks
// the grid from the visible surface point toward the observer, and deposits
// brightness x e^-tau x subpixel area; the subsamples of a pixel are adjacent lanes,
// so the deposits aggregate to one atomic per pixel and warp.
#include "qmcrt_device.cuh"

namespace qmcrt {

template <class T>
__global__ void __launch_bounds__(32) k_direct_point(const __grid_constant__ TraceP<T> P, T weight)
{
    const bool lead = threadIdx.x == 0;
    T S[3] = {T(0), T(0), T(0)};
    if (lead) {
        const T origin[3] = {T(0), T(0), T(0)};
        S[0] = Mth<T>::exp_(-tau_to_edge(P.med, origin, P.obs.k)) * T(0.07957747154594767) * weight;  // 1/(4 pi)
    }
    splat(P, lead, 0, T(0), T(0), S);
}

template <class T>
__global__ void __launch_bounds__(256) k_direct_star(const __grid_constant__ TraceP<T> P, int S, int ix0, int iy0,
                                                    int bw, int bh, T weight)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t per_pix = (uint64_t)S * S, total = (uint64_t)bw * bh * per_pix;
    if ((t & ~31ull) >= total) return;  // uniform per warp
    const ObsP<T> &O = P.obs;
    bool in = false;
    T v = T(0);
    size_t e = 0;
    if (t < total) {
        const uint64_t pix = t / per_pix, sub = t - pix * per_pix;
        const int ix = ix0 + (int)(pix % (uint64_t)bw), iy = iy0 + (int)(pix / (uint64_t)bw);
        const int a = (int)(sub % (uint64_t)S), b = (int)(sub / (uint64_t)S);
        const T px = T(2) * O.hw / T(O.nx), py = T(2) * O.hw / T(O.ny);
        const T x = -O.hw + (T(ix) + (T(a) + T(0.5)) / T(S)) * px;
        const T y = -O.hw + (T(iy) + (T(b) + T(0.5)) / T(S)) * py;
        const T R = P.src.R, rho2 = x * x + y * y;
        if (rho2 < R * R) {
            const T mu = Mth<T>::sqrt_(T(1) - rho2 / (R * R));
            T p[3];
            for (int c = 0; c < 3; ++c) p[c] = x * O.ex[c] + y * O.ey[c] + R * mu * O.k[c];
            const T B = (T(1) - P.src.limb_u + P.src.limb_u * mu) * P.src.limb_norm * T(0.07957747154594767) /
                        (T(3.14159265358979323846) * R * R);
            const T dA = px * py / (T(S) * T(S));
            v = B * Mth<T>::exp_(-tau_to_edge(P.med, p, O.k)) * dA * weight;
            e = (size_t)iy * O.nx + ix;
            in = true;
        }
    }
    deposit<T>(P.acc, in, e, v, T(0), T(0));
}

template <class T>
static cudaError_t launch(const TraceP<T> &p, int S, double weight, cudaStream_t s)
{
    if (p.src.kind != QMCRT_SOURCE_SPHERE) {
        k_direct_point<T><<<1, 32, 0, s>>>(p, (T)weight);
        return cudaGetLastError();
    }
    const double hw = (double)p.obs.hw, R = (double)p.src.R;
    const double px = 2.0 * hw / p.obs.nx, py = 2.0 * hw / p.obs.ny;
    const int ix0 = std::max(0, (int)std::floor((-R + hw) / px)), ix1 = std::min(p.obs.nx - 1, (int)std::floor((R + hw) / px));
    const int iy0 = std::max(0, (int)std::floor((-R + hw) / py)), iy1 = std::min(p.obs.ny - 1, (int)std::floor((R + hw) / py));
    if (ix1 < ix0 || iy1 < iy0) return cudaSuccess;
    const int bw = ix1 - ix0 + 1, bh = iy1 - iy0 + 1;
    const uint64_t total = (uint64_t)bw * bh * S * S;
    const uint64_t grid = (((total + 31) & ~31ull) + 255) / 256;
    k_direct_star<T><<<(unsigned)grid, 256, 0, s>>>(p, S, ix0, iy0, bw, bh, (T)weight);
    return cudaGetLastError();
}

cudaError_t launch_direct_light_f32(const TraceP<float> &p, int S, double weight, cudaStream_t s)
{
    return launch(p, S, weight, s);
}

cudaError_t launch_direct_light_f64(const TraceP<double> &p, int S, double weight, cudaStream_t s)
{
    return launch(p, S, weight, s);
}

}  // namespace qmcrt

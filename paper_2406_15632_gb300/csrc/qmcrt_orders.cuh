// qmcrt_orders.cuh -- the scattering orders of one packet (Sec. 3.5, 3.7), shared by
// the multiple-scattering kernels for one observer and for a set of observers.
//
// Order k reads coordinates 4(k-1) + {0 azimuth, 1 cos Theta, 2 depth, 3 roulette}; a
// finite star reads its two other emission coordinates at 4 max_orders + {0, 1}; with
// a learned warp the first-order coordinates come from a buffer (x = T(u)) and the
// weight starts at |dx/du|.  The order loop is uniform across the warp, so the
// peel-off callback (which bins into images) is reached by all 32 lanes; the warp
// leaves the loop once all its packets are done.
#pragma once

#include "qmcrt_device.cuh"

namespace qmcrt {

// peel(k, alive, pos, n, a, S): peel-offs of order k for a packet at pos travelling
// along n with Stokes S in the frame of axis a; called by every lane of the warp.
template <class T, class Peel>
__device__ __forceinline__ void trace_orders(const TraceP<T> &P, uint64_t i, uint64_t j, bool live_index, Peel &peel)
{
    bool alive = live_index;
    T pos[3] = {T(0), T(0), T(0)}, n[3] = {T(0), T(0), T(1)}, a[3] = {T(1), T(0), T(0)};
    T S[3] = {T(0), T(0), T(0)};
    T wd = T(0);
    if (alive) {
        T wgt;
        if (P.warp_x) {  // learned proposal: first-order coordinates and their Jacobian
            T sp, cp;
            direction_from((T)P.warp_x[3 * j], (T)P.warp_x[3 * j + 1], n, a, sp, cp);
            pos[0] = pos[1] = pos[2] = T(0);
            wd = (T)P.warp_x[3 * j + 2];
            wgt = Mth<T>::exp_((T)P.warp_logj[j]);
        } else {
            // a finite star's two extra emission coordinates follow all orders' coordinates
            const int e = 4 * P.max_orders;
            wd = emit(P, i, pos, n, a, wgt, e, e + 1, 2);
        }
        S[0] = wgt;
    }
    for (int k = 1; k <= P.max_orders; ++k) {
        if (!__any_sync(FULL_MASK, alive)) break;
        const int base = 4 * (k - 1);
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
            }
        }
        peel(k, alive, pos, n, a, S);
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
}

}  // namespace qmcrt

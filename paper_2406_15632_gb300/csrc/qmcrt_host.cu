// qmcrt_host.cu -- host-side entry points around the tracer: the fixed-point scale of an
// accumulation (from a bound on one peel-off contribution), and single scattering with
// host-resident inputs and outputs (copies, padding, maps, trace, reduction and the copy
// back enqueued on one stream).
#include <cmath>
#include <cstring>

#include "qmcrt.h"
#include "qmcrt_internal.h"

namespace {

int bound_args(const qmcrt_source *src, const qmcrt_dust *du, const qmcrt_trace_opts *op)
{
    if (!src || src->struct_size != sizeof(qmcrt_source))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "source is NULL or has the wrong struct_size");
    if (!du || du->struct_size != sizeof(qmcrt_dust))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "dust is NULL or has the wrong struct_size");
    if (!op || op->struct_size != sizeof(qmcrt_trace_opts))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "opts is NULL or has the wrong struct_size");
    if (!(du->albedo >= 0 && du->albedo <= 1)) return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "albedo outside [0, 1]");
    if (!(std::fabs(du->g) < 1)) return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "|g| must be < 1");
    if (!(du->p_l >= 0 && du->p_l <= 1)) return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "p_l outside [0, 1]");
    if (src->kind == QMCRT_SOURCE_SPHERE && !(src->limb_u >= 0 && src->limb_u <= 1))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "limb_u outside [0, 1]");
    if (src->kind != QMCRT_SOURCE_POINT && src->kind != QMCRT_SOURCE_SPHERE)
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "unknown source kind %d", src->kind);
    return QMCRT_OK;
}

// Orders a packet scatters at most (1 for single scattering).
int orders_of(const qmcrt_trace_opts *op, int multiple) { return multiple ? op->max_orders : 1; }

// Largest |I|, |Q|, |U| of one peel-off contribution (Sec. 2.2, 3.5, 3.6).  The weight
// starts at the source weight (the limb-darkening factor is at most 1 / (1 - u/3)).  At
// each scattering the forcing weight is at most 1, the albedo multiplies I, and the
// Mueller matrix divided by P11 multiplies I by 1 + (P12/P11)(Q/I) <= 1 + p_l (the carried
// Stokes vector keeps |Q| <= I); the peel-off of order k adds the phase function, at
// most (1 + |g|) / (4 pi (1 - |g|)^2), and once more at most 1 + p_l.  A roulette
// survivor's weight below the threshold is divided by the survival probability, so it
// is at most threshold / survival.  Order k therefore contributes at most
// limb p_max max(1, thr / surv) (albedo (1 + p_l))^k, taken at its largest k.
double contribution_bound(const qmcrt_source *src, const qmcrt_dust *du, const qmcrt_trace_opts *op, int multiple)
{
    const double g = std::fabs(du->g);
    const double p_max = (1.0 + g) / ((1.0 - g) * (1.0 - g)) / (4.0 * M_PI);
    const double limb = src->kind == QMCRT_SOURCE_SPHERE ? 1.0 / (1.0 - src->limb_u / 3.0) : 1.0;
    const double step = du->albedo * (1.0 + du->p_l);
    const int K = orders_of(op, multiple);
    double growth = 0.0, f = 1.0;
    for (int k = 1; k <= K; ++k) {
        f *= step;
        growth = std::fmax(growth, f);
    }
    const double rr = (multiple && K > 1 && op->rr_threshold > 0) ? std::fmax(1.0, op->rr_threshold / op->rr_survival)
                                                                   : 1.0;
    return limb * p_max * growth * rr;
}

}  // namespace

extern "C" {

int qmcrt_contribution_bound(const qmcrt_source *source, const qmcrt_dust *dust, const qmcrt_trace_opts *opts,
                             int32_t multiple, double *bound)
{
    int rc = bound_args(source, dust, opts);
    if (rc) return rc;
    if (!bound) return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "bound is NULL");
    if (multiple && (opts->max_orders < 1 || opts->max_orders > 64))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "max_orders outside 1..64");
    if (multiple && opts->rr_threshold > 0 && !(opts->rr_survival > 0 && opts->rr_survival <= 1))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "rr_survival outside (0, 1]");
    *bound = contribution_bound(source, dust, opts, multiple);
    return QMCRT_OK;
}

int qmcrt_default_frac_bits(const qmcrt_source *source, const qmcrt_dust *dust, const qmcrt_trace_opts *opts,
                            int32_t multiple, uint64_t n_packets, double weight_bound, int32_t *frac_bits)
{
    double b = 0.0;
    int rc = qmcrt_contribution_bound(source, dust, opts, multiple, &b);
    if (rc) return rc;
    if (!frac_bits) return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "frac_bits is NULL");
    if (!(weight_bound >= 1.0) || !std::isfinite(weight_bound))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "weight_bound must be finite and >= 1");
    // contributions one image pixel can receive per packet: every order, unless each
    // order has its own image
    const double per_packet = (multiple && !opts->per_order) ? (double)orders_of(opts, multiple) : 1.0;
    const double need = std::log2(std::fmax((double)n_packets, 1.0) * per_packet * b * weight_bound);
    *frac_bits = (int32_t)std::fmax(0.0, std::fmin(62.0, std::floor(62.0 - need)));
    return QMCRT_OK;
}

int qmcrt_render_single_host(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                             const qmcrt_observer *obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                             const qmcrt_host_io *io, int32_t frac_bits, double scale, void *stream)
{
    if (!io || io->struct_size != sizeof(qmcrt_host_io))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "io is NULL or has the wrong struct_size");
    if (!medium || medium->struct_size != sizeof(qmcrt_medium))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "medium is NULL or has the wrong struct_size");
    if (!obs || obs->struct_size != sizeof(qmcrt_observer))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "obs is NULL or has the wrong struct_size");
    if (!io->d_accum || !io->d_image || !io->h_image)
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "d_accum, d_image and h_image must be given");
    const bool copy_grid = io->h_k != nullptr;
    if (copy_grid && medium->kind != QMCRT_MEDIUM_GRID)
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "h_k given for a medium without a grid");
    if (copy_grid && medium->pad > 0 && !io->d_k)
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "a padded grid needs d_k to receive h_k");
    if (copy_grid && medium->pad > 0 && io->d_k == medium->d_k)
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "d_k must not be the padded grid medium->d_k");
    if (copy_grid && medium->d_sky) {  // the bound map is rebuilt from the new grid: its workspace first
        const uint64_t need = qmcrt_sky_workspace_bytes(medium->nx, medium->ny, medium->nz, medium->lo, medium->hi,
                                                        medium->sky_r);
        if (!io->d_sky_ws || io->sky_ws_bytes < need || ((uintptr_t)io->d_sky_ws & 255) != 0)
            return qmcrt::set_error(QMCRT_ERR_INVALID_ARG,
                                    "a grid with a bound map needs d_sky_ws of %llu bytes, 256-byte aligned",
                                    (unsigned long long)need);
    }
    if (copy_grid && obs->d_tail) {  // so is the tail map
        const uint64_t need = qmcrt_tail_workspace_bytes(medium->nx, medium->ny, medium->nz);
        if (!io->d_tail_ws || io->tail_ws_bytes < need || ((uintptr_t)io->d_tail_ws & 255) != 0)
            return qmcrt::set_error(QMCRT_ERR_INVALID_ARG,
                                    "an observer with a tail map needs d_tail_ws of %llu bytes, 256-byte aligned",
                                    (unsigned long long)need);
    }
    qmcrt_image im;
    memset(&im, 0, sizeof im);
    im.struct_size = sizeof im;
    im.accum = QMCRT_ACCUM_I64;
    im.d_accum = io->d_accum;
    im.n_images = 1;
    im.frac_bits = frac_bits;
    int rc = qmcrt::check_trace_single(medium, source, dust, obs, pts, opts, &im);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t pixels = (size_t)obs->nx * obs->ny;
    cudaError_t e = cudaSuccess;
    if (copy_grid) {
        const size_t cells = (size_t)medium->nx * medium->ny * medium->nz;
        // unpadded: the grid the walk reads is medium->d_k itself
        float *dst = medium->pad > 0 ? io->d_k : const_cast<float *>(medium->d_k);
        e = cudaMemcpyAsync(dst, io->h_k, cells * sizeof(float), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return qmcrt::set_error(QMCRT_ERR_CUDA, "grid copy: %s", cudaGetErrorString(e));
        if (medium->pad > 0) {
            rc = qmcrt_pad_grid(io->d_k, medium->nx, medium->ny, medium->nz, medium->pad,
                                const_cast<float *>(medium->d_k), stream);
            if (rc) return rc;
        }
        if (medium->d_sky) {  // the bound map follows the new grid
            rc = qmcrt_sky_bound(medium->pad > 0 ? io->d_k : medium->d_k, medium->nx, medium->ny, medium->nz,
                                 medium->lo, medium->hi, medium->sky_r, medium->sky_m,
                                 const_cast<double *>(medium->d_sky), io->d_sky_ws, io->sky_ws_bytes, stream);
            if (rc) return rc;
        }
        if (obs->d_tail) {  // and the tail map
            rc = qmcrt_tail_map(medium, obs, const_cast<uint8_t *>(obs->d_tail), io->d_tail_ws, io->tail_ws_bytes,
                                stream);
            if (rc) return rc;
        }
    }
    e = cudaMemsetAsync(io->d_accum, 0, 3 * pixels * sizeof(long long), s);
    if (e != cudaSuccess) return qmcrt::set_error(QMCRT_ERR_CUDA, "clearing the accumulator: %s", cudaGetErrorString(e));
    rc = qmcrt_trace_single(medium, source, dust, obs, pts, opts, &im, nullptr, stream);
    if (rc) return rc;
    rc = qmcrt_image_reduce(&im, obs->nx, obs->ny, 1, scale, io->d_image, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(io->h_image, io->d_image, 3 * pixels * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return qmcrt::set_error(QMCRT_ERR_CUDA, "image copy: %s", cudaGetErrorString(e));
    return QMCRT_OK;
}

}  // extern "C"

// qmcrt_api.cu -- host side of the C ABI declared in include/qmcrt.h: argument
// validation, kernel parameter blocks, launches.  No device memory is allocated here.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <mutex>
#include <utility>

#include "qmcrt.h"
#include "qmcrt_gemm.cuh"
#include "qmcrt_internal.h"
#include "qmcrt_tables.h"

namespace {

// Host copy of the Sobol direction numbers (the same generated table the kernels
// hold in constant memory), for building the net-order packet mapping.
const uint32_t kSobolV[QMCRT_GEN_DIMS][32] = QMCRT_GEN_SOBOL_V_INIT;
const uint32_t kNiedV[QMCRT_GEN_DIMS][32] = QMCRT_GEN_NIED_V_INIT;

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return QMCRT_OK;
    return fail(QMCRT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CHECK_STRUCT(p, T)                                                                         \
    do {                                                                                           \
        if (!(p)) return fail(QMCRT_ERR_INVALID_ARG, #p " is NULL");                               \
        if ((p)->struct_size != sizeof(T))                                                         \
            return fail(QMCRT_ERR_INVALID_ARG, #p "->struct_size %u != %zu (ABI mismatch)",        \
                        (unsigned)(p)->struct_size, sizeof(T));                                    \
    } while (0)

int check_points(const qmcrt_points_desc *d, uint32_t dims_needed)
{
    CHECK_STRUCT(d, qmcrt_points_desc);
    if (d->kind < QMCRT_SOBOL || d->kind > QMCRT_FAURE) return fail(QMCRT_ERR_INVALID_ARG, "unknown point kind %d", d->kind);
    if (d->dims < 1 || d->dims > QMCRT_MAX_DIMS)
        return fail(QMCRT_ERR_INVALID_ARG, "dims %u outside 1..%d", d->dims, QMCRT_MAX_DIMS);
    if (d->dims < dims_needed)
        return fail(QMCRT_ERR_INVALID_ARG, "dims %u < %u coordinates used per packet", d->dims, dims_needed);
    if (d->first_index == 0) return fail(QMCRT_ERR_INVALID_ARG, "first_index must be >= 1 (the zero point is skipped)");
    const uint64_t last = d->first_index + (d->count ? d->count - 1 : 0);
    if (last < d->first_index) return fail(QMCRT_ERR_INVALID_ARG, "index range overflows");
    if (d->kind != QMCRT_PHILOX && last > 0xffffffffull)
        return fail(QMCRT_ERR_INVALID_ARG, "point index %llu >= 2^32", (unsigned long long)last);
    if (d->kind == QMCRT_HAMMERSLEY && (d->total_n == 0 || last > d->total_n))
        return fail(QMCRT_ERR_INVALID_ARG, "Hammersley index %llu beyond N = %llu", (unsigned long long)last,
                    (unsigned long long)d->total_n);
    return QMCRT_OK;
}

qmcrt::PointsP make_points(const qmcrt_points_desc *d)
{
    qmcrt::PointsP p;
    p.kind = d->kind;
    p.dims = (int)d->dims;
    p.seed = d->seed;
    p.total_n = d->total_n;
    p.inv_total_n = d->total_n ? 1.0 / (double)d->total_n : 0.0;
    uint32_t b = d->dims < 2 ? 2u : d->dims;  // Faure base: smallest prime >= dims
    for (;; ++b) {
        bool prime = true;
        for (uint32_t q = 2; q * q <= b; ++q)
            if (b % q == 0) {
                prime = false;
                break;
            }
        if (prime) break;
    }
    p.faure_b = b;
    return p;
}

// Packet order of a launch (see OrderP): net order for digital base-2 point sets
// (Sobol, scrambled Sobol, Niederreiter) of at least 2^7 packets, linear otherwise.
// Solves y = L g over GF(2) once per call: L maps the digit vector g of an index
// inside a 2^m block (its Gray code for Sobol, its binary digits for Niederreiter) to
// the leading bits of its coordinates 0, 1, 2 (balanced) and, when x0 >= 0, of the two
// further coordinates x0, x1 (xbits each); tt is the smallest value for which L has full
// row rank (the elementary boxes then hold 2^tt points each).  Thread bits go to the
// box bits in Morton order, finest first, over coordinates 0, 1, 2 before x0, x1 (a
// warp's five bits mostly to coordinate 2, kWarpBitOrder): a warp spans the finest bits
// of the ray coordinates and shares the coarser ones, including those of x0, x1.  If no
// tt <= NET_MAX_TT gives full rank with the further coordinates, they are dropped.
// The coordinates whose finest box bits a warp's five thread bits take: four of
// coordinate 2 (the forced scattering depth) and one of coordinate 0 (the azimuth), so a
// warp's 32 packets run along two nearly equal rays to nearby depths.  Measured on the
// 256^3 disk at 2^26 packets (two bits each of coordinates 0 and 1 and one of 2 before):
// 1.3 % faster, and the 256-instance finite-star batch 7 %; the L1 data pipe serves one
// wavefront per distinct 128-byte line a warp-wide density load touches.  Five bits of
// coordinate 2 were 0.9 % slower on the disk.
constexpr int kWarpBitOrder[5] = {2, 2, 2, 2, 0};
void make_order(int kind, uint64_t first, uint64_t count, qmcrt::OrderP &O, int x0 = -1, int x1 = -1, int xbits = 0)
{
    memset(&O, 0, sizeof O);
    O.threads = count;
    if (count == 0 || (kind != QMCRT_SOBOL && kind != QMCRT_SOBOL_OWEN && kind != QMCRT_NIEDERREITER)) return;
    const uint32_t(*V)[32] = kind == QMCRT_NIEDERREITER ? kNiedV : kSobolV;
    int m = 0;
    while (m < qmcrt::NET_MAX_M && (2ull << m) <= count) ++m;
    if (m < 7) return;
    if (x0 < 0 || x1 < 0 || x0 >= QMCRT_GEN_DIMS || x1 >= QMCRT_GEN_DIMS) xbits = 0;
    for (int pass = 0; pass < 2; ++pass, xbits = 0) {
        for (int tt = 0; tt <= qmcrt::NET_MAX_TT; ++tt) {
            const int bits = m - tt;
            // the further coordinates take bits only from blocks large enough that the ray
            // coordinates keep 18 leading bits between them (measured on the 256-instance
            // finite-star batch, R* = 6.4 cells, blocks of 2^18-2^23, with a warp's thread
            // bits on the depth coordinate: 8 % faster than keeping 22; keeping 16 the same)
            const int xb = std::min(xbits, std::max(0, (bits - 18) / 2));
            const int r = bits - 2 * xb;
            const int nb[5] = {(r + 2) / 3, (r + 1) / 3, r / 3, xb, xb};
            const int dims[5] = {0, 1, 2, x0, x1};
            const int order[5] = {2, 1, 0, 3, 4};  // y bits: coordinate 2 lowest, then 1, 0, x0, x1
            uint32_t Lr[qmcrt::NET_MAX_M], Er[qmcrt::NET_MAX_M];
            int off[5], rho = 0;
            for (int oi = 0; oi < 5; ++oi) {
                const int comp = order[oi];
                off[comp] = rho;
                for (int q = 0; q < nb[comp]; ++q, ++rho) {
                    const int bit = 32 - nb[comp] + q;
                    uint32_t row = 0;
                    for (int k = 0; k < m; ++k) row |= ((V[dims[comp]][k] >> bit) & 1u) << k;
                    Lr[rho] = row;
                    Er[rho] = 1u << rho;
                }
            }
            int piv[qmcrt::NET_MAX_M], rank = 0;
            for (int col = 0; col < m && rank < bits; ++col) {
                int sel = -1;
                for (int q = rank; q < bits; ++q)
                    if ((Lr[q] >> col) & 1u) { sel = q; break; }
                if (sel < 0) continue;
                std::swap(Lr[sel], Lr[rank]);
                std::swap(Er[sel], Er[rank]);
                for (int q = 0; q < bits; ++q)
                    if (q != rank && ((Lr[q] >> col) & 1u)) {
                        Lr[q] ^= Lr[rank];
                        Er[q] ^= Er[rank];
                    }
                piv[rank++] = col;
            }
            if (rank < bits) continue;
            O.net = kind == QMCRT_NIEDERREITER ? 2 : 1;
            O.m = m;
            O.bits = bits;
            O.tt = tt;
            for (int q = 0; q < 5; ++q) O.nb[q] = nb[q];
            O.xdim[0] = xb ? x0 : 0;
            O.xdim[1] = xb ? x1 : 0;
            for (int j = 0; j < bits; ++j) {
                uint32_t col = 0;
                for (int q = 0; q < bits; ++q) col |= ((Er[q] >> j) & 1u) << piv[q];
                O.ry[j] = col;
            }
            int nk = 0;
            for (int f = 0; f < m; ++f) {
                bool is_piv = false;
                for (int q = 0; q < bits; ++q) is_piv |= piv[q] == f;
                if (is_piv) continue;
                uint32_t kv = 1u << f;
                for (int q = 0; q < bits; ++q) kv |= ((Lr[q] >> f) & 1u) << piv[q];
                O.k[nk++] = kv;
            }
            // Morton order of the boxes: a warp's thread bits go to the finest bits of the
            // coordinates in kWarpBitOrder (while they have any), the rest round-robin to
            // the finest remaining bit of coordinates 0, 1, 2, then of x0, x1.
            int used[5] = {0, 0, 0, 0, 0}, j = 0;
            for (const int comp : kWarpBitOrder)
                if (used[comp] < nb[comp]) O.rm[j++] = O.ry[off[comp] + used[comp]++];
            for (int group = 0; group < 2; ++group) {
                const int lo = group ? 3 : 0, hi = group ? 5 : 3;
                for (bool any = true; any;) {
                    any = false;
                    for (int comp = lo; comp < hi; ++comp) {
                        if (used[comp] >= nb[comp]) continue;
                        O.rm[j++] = O.ry[off[comp] + used[comp]++];
                        any = true;
                    }
                }
            }
            O.block0 = first >> m;
            const uint64_t nblocks = ((first + count - 1) >> m) - O.block0 + 1;
            O.threads = nblocks << m;
            // The part of g that depends only on the block (the leading bits y of the
            // block start's coordinates), for the first block: the kernels take it from
            // here instead of recomputing it per packet.
            const uint32_t b32 = (uint32_t)(O.block0 << m);
            const uint32_t gb = O.net == 2 ? b32 : b32 ^ (b32 >> 1);
            const int bd[5] = {0, 1, 2, O.xdim[0], O.xdim[1]};
            uint32_t bv[5] = {0, 0, 0, 0, 0};
            for (int k = 0; k < 32; ++k)
                if ((gb >> k) & 1u)
                    for (int c = 0; c < 5; ++c) bv[c] ^= V[bd[c]][k];
            auto lead = [](uint32_t x, int n) { return n ? x >> (32 - n) : 0u; };
            const int s1 = nb[2], s0 = s1 + nb[1], s3 = s0 + nb[0], s4 = s3 + nb[3];
            const uint32_t y = lead(bv[2], nb[2]) | (lead(bv[1], nb[1]) << s1) | (lead(bv[0], nb[0]) << s0) |
                               (lead(bv[3], nb[3]) << s3) | (lead(bv[4], nb[4]) << s4);
            O.g0_block = O.block0;
            O.g0 = 0;
            for (int j = 0; j < bits; ++j)
                if ((y >> j) & 1u) O.g0 ^= O.ry[j];
            return;
        }
        if (xbits == 0) return;  // no full rank even without the further coordinates
    }
}

// Leading bits per further coordinate in the net order of a finite star's packets.
constexpr int kNetExtraBits = 2;

// The further coordinates a net order groups, and how many bits each: those of a finite
// star that place the ray besides its direction and depth (single scattering:
// coordinates 3, 4 -- the local cos theta and the depth in the direct order, the
// emission point in the inverse order; multiple scattering: the star's extras after all
// orders', 4M and 4M + 1).  The inverse order's emission point matters only where the
// star spans several grid cells (measured with two bits each: R* = 6.4 cells gains 7 %,
// R* = 1.3 cells loses 13 %); a point source has none.
int order_extras(int src_kind, int src_order, double R, int med_kind, const double h[3], int max_orders, int &x0,
                 int &x1)
{
    x0 = x1 = -1;
    if (src_kind != QMCRT_SOURCE_SPHERE) return 0;
    x0 = max_orders > 1 ? 4 * max_orders : 3;
    x1 = x0 + 1;
    if (src_order == QMCRT_ORDER_DIRECT) return kNetExtraBits;
    if (med_kind != QMCRT_MEDIUM_GRID) return 0;
    return R >= 4.0 * std::min(h[0], std::min(h[1], h[2])) ? kNetExtraBits : 0;
}

template <class T>
int order_extras(const qmcrt::TraceP<T> &P, int &x0, int &x1)
{
    const double h[3] = {(double)P.med.h[0], (double)P.med.h[1], (double)P.med.h[2]};
    return order_extras(P.src.kind, P.src.order, (double)P.src.R, P.med.kind, h, P.max_orders, x0, x1);
}

// Observer direction k, sky axes e_x, e_y and pixel scale (Sec. 3.6).
template <class T>
int make_obs(const qmcrt_observer *ob, qmcrt::ObsP<T> &O)
{
    if (ob->nx < 1 || ob->ny < 1) return fail(QMCRT_ERR_INVALID_ARG, "image has no pixels");
    if (!(ob->half_width > 0)) return fail(QMCRT_ERR_INVALID_ARG, "half_width must be > 0");
    if (ob->splat != QMCRT_SPLAT_NEAREST && ob->splat != QMCRT_SPLAT_BILINEAR)
        return fail(QMCRT_ERR_INVALID_ARG, "unknown splat mode %d", ob->splat);
    const double st = std::sin(ob->theta), ct = std::cos(ob->theta), sp = std::sin(ob->phi), cp = std::cos(ob->phi);
    const double k[3] = {st * cp, st * sp, ct}, ex[3] = {-sp, cp, 0.0}, ey[3] = {-ct * cp, -ct * sp, st};
    for (int a = 0; a < 3; ++a) {
        O.k[a] = (T)k[a];
        O.ex[a] = (T)ex[a];
        O.ey[a] = (T)ey[a];
        O.inv_k[a] = T(1) / O.k[a];  // IEEE division in T, as on the device (inf for a zero component)
    }
    O.hw = (T)ob->half_width;
    O.pix_x = (T)(ob->nx / (2.0 * ob->half_width));
    O.pix_y = (T)(ob->ny / (2.0 * ob->half_width));
    O.nx = ob->nx;
    O.ny = ob->ny;
    O.splat = ob->splat;
    O.tail = nullptr;
    O.tail_thr = 0;
    return QMCRT_OK;
}

// The observer's tail map (qmcrt_tail_map), if given: valid on a padded grid only; the
// threshold code follows from the tolerance and the medium's kscale.
template <class T>
int attach_tail(const qmcrt_medium *md, const qmcrt_observer *ob, const qmcrt_trace_opts *op, qmcrt::ObsP<T> &O)
{
    if (!ob->d_tail) return QMCRT_OK;
    if (md->kind != QMCRT_MEDIUM_GRID || md->pad < QMCRT_MIN_PAD)
        return fail(QMCRT_ERR_INVALID_ARG, "a tail map needs a padded grid medium");
    if (!(op->tail_eps >= 0) || !std::isfinite(op->tail_eps))
        return fail(QMCRT_ERR_INVALID_ARG, "tail_eps must be finite and >= 0");
    O.tail = ob->d_tail;
    O.tail_thr = qmcrt::tail_threshold(op->tail_eps, md->kscale);
    return QMCRT_OK;
}

template <class T>
int fill_trace(const qmcrt_medium *md, const qmcrt_source *src, const qmcrt_dust *du, const qmcrt_observer *ob,
               const qmcrt_points_desc *pts, const qmcrt_trace_opts *op, const qmcrt_image *im, int multiple,
               qmcrt::TraceP<T> &P)
{
    memset(&P, 0, sizeof P);
    // medium
    P.med.kind = md->kind;
    if (!(md->kscale > 0) || !std::isfinite(md->kscale)) return fail(QMCRT_ERR_INVALID_ARG, "kscale must be > 0");
    P.med.kscale = (T)md->kscale;
    P.med.inv_kscale = (T)(1.0 / md->kscale);
    if (md->kind == QMCRT_MEDIUM_GRID) {
        if (!md->d_k) return fail(QMCRT_ERR_INVALID_ARG, "grid medium with NULL d_k");
        if (md->nx < 1 || md->ny < 1 || md->nz < 1) return fail(QMCRT_ERR_INVALID_ARG, "grid has zero cells");
        if ((double)md->nx * md->ny * md->nz > 2147483647.0)
            return fail(QMCRT_ERR_INVALID_ARG, "grid larger than 2^31 cells");
        const int n[3] = {md->nx, md->ny, md->nz};
        for (int a = 0; a < 3; ++a) {
            if (!(md->hi[a] > md->lo[a])) return fail(QMCRT_ERR_INVALID_ARG, "grid box axis %d is empty", a);
            P.med.n[a] = n[a];
            P.med.lo[a] = (T)md->lo[a];
            P.med.hi[a] = (T)md->hi[a];
            P.med.h[a] = (T)((md->hi[a] - md->lo[a]) / n[a]);
            P.med.inv_h[a] = (T)(n[a] / (md->hi[a] - md->lo[a]));
        }
        if (md->pad != 0 && md->pad < QMCRT_MIN_PAD)
            return fail(QMCRT_ERR_INVALID_ARG, "pad %d: 0 or at least %d", md->pad, QMCRT_MIN_PAD);
        const int px = md->nx + 2 * md->pad, py = md->ny + 2 * md->pad, pz = md->nz + 2 * md->pad;
        if ((double)px * py * pz > 2147483647.0) return fail(QMCRT_ERR_INVALID_ARG, "padded grid larger than 2^31 cells");
        P.med.pad = md->pad;
        if (md->d_sky) {
            if (md->sky_m < 1 || md->sky_m > 4096) return fail(QMCRT_ERR_INVALID_ARG, "sky_m outside 1..4096");
            if (!(md->sky_r >= 0) || !std::isfinite(md->sky_r)) return fail(QMCRT_ERR_INVALID_ARG, "sky_r must be >= 0");
            P.med.sky = md->d_sky;
            P.med.sky_m = md->sky_m;
            // a start point counts as within R if |p|^2 <= R^2 (1 + 1e-5), which takes in the
            // float rounding of a point on the star's surface; the map is built for R (1 + 1e-4)
            P.med.sky_r2 = (T)(md->sky_r * md->sky_r * (1.0 + 1e-5));
        }
        P.med.stride[0] = 1;
        P.med.stride[1] = px;
        P.med.stride[2] = px * py;
        P.med.k = md->d_k;
    } else if (md->kind == QMCRT_MEDIUM_SPHERE) {
        if (!(md->sphere_r > 0) || !(md->sphere_k >= 0)) return fail(QMCRT_ERR_INVALID_ARG, "sphere medium needs r > 0, k >= 0");
        P.med.sph_r = (T)md->sphere_r;
        P.med.sph_k = (T)(md->sphere_k * md->kscale);
    } else {
        return fail(QMCRT_ERR_INVALID_ARG, "unknown medium kind %d", md->kind);
    }
    // source
    if (src->kind == QMCRT_SOURCE_POINT) {
        P.src.kind = src->kind;
        P.src.limb_u = T(0);
        P.src.limb_norm = T(1);
    } else if (src->kind == QMCRT_SOURCE_SPHERE) {
        if (!(src->radius > 0)) return fail(QMCRT_ERR_INVALID_ARG, "sphere source needs radius > 0");
        if (!(src->limb_u >= 0 && src->limb_u <= 1)) return fail(QMCRT_ERR_INVALID_ARG, "limb_u outside [0, 1]");
        if (src->order != QMCRT_ORDER_DIRECT && src->order != QMCRT_ORDER_INVERSE)
            return fail(QMCRT_ERR_INVALID_ARG, "unknown emission order %d", src->order);
        P.src.kind = src->kind;
        P.src.order = src->order;
        P.src.R = (T)src->radius;
        P.src.limb_u = (T)src->limb_u;
        P.src.limb_norm = (T)(1.0 / (1.0 - src->limb_u / 3.0));
    } else {
        return fail(QMCRT_ERR_INVALID_ARG, "unknown source kind %d", src->kind);
    }
    // dust
    if (!(du->albedo >= 0 && du->albedo <= 1)) return fail(QMCRT_ERR_INVALID_ARG, "albedo outside [0, 1]");
    if (!(std::fabs(du->g) < 1)) return fail(QMCRT_ERR_INVALID_ARG, "|g| must be < 1");
    if (!(du->p_l >= 0 && du->p_l <= 1)) return fail(QMCRT_ERR_INVALID_ARG, "p_l outside [0, 1]");
    P.dust.albedo = (T)du->albedo;
    P.dust.g = (T)du->g;
    P.dust.p_l = (T)du->p_l;
    P.dust.one_m_g2 = (T)(1.0 - du->g * du->g);
    P.dust.one_p_g2 = (T)(1.0 + du->g * du->g);
    P.dust.two_g = (T)(2.0 * du->g);
    P.dust.isotropic = std::fabs(du->g) < 1e-6;
    // observer
    {
        int rc = make_obs(ob, P.obs);
        if (!rc) rc = attach_tail(md, ob, op, P.obs);
        if (rc) return rc;
    }
    // options
    if (op->precision != QMCRT_PREC_F32 && op->precision != QMCRT_PREC_F64)
        return fail(QMCRT_ERR_INVALID_ARG, "unknown precision %d", op->precision);
    if (!(op->tau_min >= 0)) return fail(QMCRT_ERR_INVALID_ARG, "tau_min must be >= 0");
    if (op->block_size != 0 && (op->block_size % 32 != 0 || op->block_size < 32 || op->block_size > 256))
        return fail(QMCRT_ERR_INVALID_ARG, "block_size must be a multiple of 32 in 32..256");
    P.tau_min = (T)op->tau_min;
    if (!(op->tail_eps >= 0) || !std::isfinite(op->tail_eps))
        return fail(QMCRT_ERR_INVALID_ARG, "tail_eps must be finite and >= 0");
    P.tail_eps = op->tail_eps;
    P.max_orders = multiple ? op->max_orders : 1;
    if (multiple) {
        if (op->max_orders < 1 || op->max_orders > 64) return fail(QMCRT_ERR_INVALID_ARG, "max_orders outside 1..64");
        if (op->force_mode != QMCRT_FORCE_ALL && op->force_mode != QMCRT_FORCE_FIRST)
            return fail(QMCRT_ERR_INVALID_ARG, "unknown force mode %d", op->force_mode);
        if (!(op->rr_threshold >= 0)) return fail(QMCRT_ERR_INVALID_ARG, "rr_threshold must be >= 0");
        if (!(op->rr_survival > 0 && op->rr_survival <= 1)) return fail(QMCRT_ERR_INVALID_ARG, "rr_survival outside (0, 1]");
        P.force_all = op->force_mode == QMCRT_FORCE_ALL;
        P.per_order = op->per_order != 0;
        P.rr_threshold = (T)op->rr_threshold;
        P.rr_survival = (T)op->rr_survival;
        P.inv_rr_survival = (T)(1.0 / op->rr_survival);
    }
    // points
    const uint32_t need = multiple ? 4u * (uint32_t)op->max_orders + (src->kind == QMCRT_SOURCE_SPHERE ? 2u : 0u)
                                   : (src->kind == QMCRT_SOURCE_SPHERE ? 5u : 3u);
    int rc = check_points(pts, need);
    if (rc) return rc;
    P.pts = make_points(pts);
    P.first = pts->first_index;
    P.count = pts->count;
    {
        int x0, x1;
        const int xb = order_extras(P, x0, x1);
        make_order(pts->kind, pts->first_index, pts->count, P.ord, x0, x1, xb);
    }
    // image
    if (!im->d_accum) return fail(QMCRT_ERR_INVALID_ARG, "image->d_accum is NULL");
    if (im->accum != QMCRT_ACCUM_I64 && im->accum != QMCRT_ACCUM_F64)
        return fail(QMCRT_ERR_INVALID_ARG, "unknown accumulation mode %d", im->accum);
    if (im->accum == QMCRT_ACCUM_I64 && (im->frac_bits < 0 || im->frac_bits > 62))
        return fail(QMCRT_ERR_INVALID_ARG, "frac_bits outside 0..62");
    const int want_images = (multiple && op->per_order) ? op->max_orders : 1;
    if (im->n_images != want_images)
        return fail(QMCRT_ERR_INVALID_ARG, "image->n_images = %d, expected %d", im->n_images, want_images);
    P.acc.ptr = im->d_accum;
    P.acc.mode = im->accum;
    P.acc.n_images = im->n_images;
    P.acc.scale = std::ldexp(1.0, im->frac_bits);
    P.acc.plane = (size_t)ob->nx * ob->ny;
    return QMCRT_OK;
}

struct WarpIO {
    const float *x = nullptr, *logj = nullptr;
    float *log = nullptr;
};

int trace_common(const qmcrt_medium *md, const qmcrt_source *src, const qmcrt_dust *du, const qmcrt_observer *ob,
                 const qmcrt_points_desc *pts, const qmcrt_trace_opts *op, const qmcrt_image *im, double *d_log,
                 void *stream, int multiple, WarpIO wio = WarpIO())
{
    CHECK_STRUCT(md, qmcrt_medium);
    CHECK_STRUCT(src, qmcrt_source);
    CHECK_STRUCT(du, qmcrt_dust);
    CHECK_STRUCT(ob, qmcrt_observer);
    CHECK_STRUCT(op, qmcrt_trace_opts);
    CHECK_STRUCT(im, qmcrt_image);
    const int block = op->block_size ? op->block_size : 256;
    cudaStream_t s = (cudaStream_t)stream;
    if (op->precision == QMCRT_PREC_F64) {
        qmcrt::TraceP<double> P;
        int rc = fill_trace<double>(md, src, du, ob, pts, op, im, multiple, P);
        if (rc) return rc;
        P.log = d_log;
        P.warp_x = wio.x;
        P.warp_logj = wio.logj;
        P.train_log = wio.log;
        return cuda_status(multiple ? qmcrt::launch_trace_multiple_f64(P, block, s)
                                    : qmcrt::launch_trace_single_f64(P, block, s),
                           "trace launch");
    }
    qmcrt::TraceP<float> P;
    int rc = fill_trace<float>(md, src, du, ob, pts, op, im, multiple, P);
    if (rc) return rc;
    P.log = d_log;
    P.warp_x = wio.x;
    P.warp_logj = wio.logj;
    P.train_log = wio.log;
    return cuda_status(multiple ? qmcrt::launch_trace_multiple_f32(P, block, s) : qmcrt::launch_trace_single_f32(P, block, s),
                       "trace launch");
}

// The host-side checks of trace_common without the launch: the status the call would
// return for these arguments, nothing enqueued.
int check_trace(const qmcrt_medium *md, const qmcrt_source *src, const qmcrt_dust *du, const qmcrt_observer *ob,
                const qmcrt_points_desc *pts, const qmcrt_trace_opts *op, const qmcrt_image *im, int multiple)
{
    CHECK_STRUCT(md, qmcrt_medium);
    CHECK_STRUCT(src, qmcrt_source);
    CHECK_STRUCT(du, qmcrt_dust);
    CHECK_STRUCT(ob, qmcrt_observer);
    CHECK_STRUCT(op, qmcrt_trace_opts);
    CHECK_STRUCT(im, qmcrt_image);
    if (op->precision == QMCRT_PREC_F64) {
        qmcrt::TraceP<double> P;
        return fill_trace<double>(md, src, du, ob, pts, op, im, multiple, P);
    }
    qmcrt::TraceP<float> P;
    return fill_trace<float>(md, src, du, ob, pts, op, im, multiple, P);
}

cudaError_t launch_observers(const qmcrt::TraceP<float> &P, const qmcrt::ObsSet<float> &S, int block, cudaStream_t s)
{
    return qmcrt::launch_trace_observers_f32(P, S, block, s);
}

cudaError_t launch_observers(const qmcrt::TraceP<double> &P, const qmcrt::ObsSet<double> &S, int block, cudaStream_t s)
{
    return qmcrt::launch_trace_observers_f64(P, S, block, s);
}

template <class T>
int observers_common(const qmcrt_medium *md, const qmcrt_source *src, const qmcrt_dust *du, const qmcrt_observer *obs,
                     int32_t n_obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *op, const qmcrt_image *im,
                     cudaStream_t s)
{
    const int multiple = op->max_orders > 1;
    qmcrt::TraceP<T> P;
    int rc = fill_trace<T>(md, src, du, &obs[0], pts, op, im, multiple, P);
    if (rc) return rc;
    qmcrt::ObsSet<T> S;
    memset(&S, 0, sizeof S);
    S.n = n_obs;
    S.stack = (size_t)im->n_images * 3 * P.acc.plane;
    for (int o = 0; o < n_obs; ++o) {
        if ((rc = make_obs(&obs[o], S.o[o]))) return rc;
        if ((rc = attach_tail(md, &obs[o], op, S.o[o]))) return rc;
        if (obs[o].nx != obs[0].nx || obs[o].ny != obs[0].ny || obs[o].splat != obs[0].splat)
            return fail(QMCRT_ERR_INVALID_ARG, "observer %d: nx, ny and splat must equal observer 0's", o);
    }
    const int block = op->block_size ? op->block_size : 256;
    return cuda_status(launch_observers(P, S, block, s), "trace_observers launch");
}

cudaError_t launch_wavefront(const qmcrt::TraceP<float> &P, void *ws, uint64_t cap, int sms, cudaStream_t s)
{
    return qmcrt::launch_trace_wavefront_f32(P, ws, cap, sms, s);
}

cudaError_t launch_wavefront(const qmcrt::TraceP<double> &P, void *ws, uint64_t cap, int sms, cudaStream_t s)
{
    return qmcrt::launch_trace_wavefront_f64(P, ws, cap, sms, s);
}

// Runs the wavefront tracer over pts in chunks of the largest power of two of packets the
// workspace holds, each chunk on cap-aligned index blocks (so each keeps whole nets).
template <class T>
int wavefront_run(qmcrt::TraceP<T> P, const qmcrt_points_desc *pts, WarpIO wio, void *ws, uint64_t ws_bytes,
                  int precision, cudaStream_t s)
{
    uint64_t cap = 1;
    while (cap < (1ull << 31) && qmcrt::wavefront_workspace_bytes(cap * 2, precision) <= ws_bytes) cap *= 2;
    if (qmcrt::wavefront_workspace_bytes(cap, precision) > ws_bytes)
        return fail(QMCRT_ERR_INVALID_ARG, "workspace below one packet");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e, "device query");
    const uint64_t first = pts->first_index, count = pts->count;
    for (uint64_t lo = first; lo < first + count;) {
        const uint64_t hi = std::min(first + count, (lo / cap + 1) * cap);
        P.first = lo;
        P.count = hi - lo;
        int x0, x1;
        const int xb = order_extras(P, x0, x1);
        make_order(pts->kind, lo, hi - lo, P.ord, x0, x1, xb);
        const uint64_t off = lo - first;
        P.warp_x = wio.x ? wio.x + 3 * off : nullptr;
        P.warp_logj = wio.logj ? wio.logj + off : nullptr;
        P.train_log = wio.log ? wio.log + 5 * off : nullptr;
        if ((e = launch_wavefront(P, ws, cap, sms, s)) != cudaSuccess) return cuda_status(e, "wavefront launch");
        lo = hi;
    }
    return QMCRT_OK;
}

}  // namespace

namespace qmcrt {

int check_trace_single(const qmcrt_medium *md, const qmcrt_source *src, const qmcrt_dust *du,
                       const qmcrt_observer *ob, const qmcrt_points_desc *pts, const qmcrt_trace_opts *op,
                       const qmcrt_image *im)
{
    return check_trace(md, src, du, ob, pts, op, im, 0);
}

int set_error(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

}  // namespace qmcrt

extern "C" {

int qmcrt_abi_version(void) { return QMCRT_ABI_VERSION; }

const char *qmcrt_last_error(void) { return g_last_error.c_str(); }

int qmcrt_generate_points(const qmcrt_points_desc *d, void *d_out, void *stream)
{
    g_last_error.clear();
    int rc = check_points(d, 1);
    if (rc) return rc;
    if (!d_out) return fail(QMCRT_ERR_INVALID_ARG, "d_out is NULL");
    if (d->format != QMCRT_FMT_U32 && d->format != QMCRT_FMT_F32 && d->format != QMCRT_FMT_F64)
        return fail(QMCRT_ERR_INVALID_ARG, "unknown format %d", d->format);
    if (d->format == QMCRT_FMT_U32 && (d->kind == QMCRT_HALTON || d->kind == QMCRT_HAMMERSLEY || d->kind == QMCRT_FAURE))
        return fail(QMCRT_ERR_INVALID_ARG, "Halton/Hammersley/Faure points have no 32-bit integer form");
    return cuda_status(qmcrt::launch_generate_points(make_points(d), d->first_index, d->count, d->format, d_out,
                                                     (cudaStream_t)stream),
                       "generate_points launch");
}

int qmcrt_trace_single(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                       const qmcrt_observer *obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                       const qmcrt_image *image, double *d_log, void *stream)
{
    g_last_error.clear();
    return trace_common(medium, source, dust, obs, pts, opts, image, d_log, stream, 0);
}

int qmcrt_trace_multiple(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                         const qmcrt_observer *obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                         const qmcrt_image *image, void *stream)
{
    g_last_error.clear();
    return trace_common(medium, source, dust, obs, pts, opts, image, nullptr, stream, 1);
}

int qmcrt_trace_observers(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                          const qmcrt_observer *obs, int32_t n_obs, const qmcrt_points_desc *pts,
                          const qmcrt_trace_opts *opts, const qmcrt_image *image, void *stream)
{
    g_last_error.clear();
    if (!obs) return fail(QMCRT_ERR_INVALID_ARG, "obs is NULL");
    if (n_obs < 1 || n_obs > QMCRT_MAX_OBSERVERS)
        return fail(QMCRT_ERR_INVALID_ARG, "n_obs = %d outside 1..%d", n_obs, QMCRT_MAX_OBSERVERS);
    for (int o = 0; o < n_obs; ++o) CHECK_STRUCT((&obs[o]), qmcrt_observer);
    CHECK_STRUCT(medium, qmcrt_medium);
    CHECK_STRUCT(source, qmcrt_source);
    CHECK_STRUCT(dust, qmcrt_dust);
    CHECK_STRUCT(opts, qmcrt_trace_opts);
    CHECK_STRUCT(image, qmcrt_image);
    cudaStream_t s = (cudaStream_t)stream;
    if (opts->precision == QMCRT_PREC_F64)
        return observers_common<double>(medium, source, dust, obs, n_obs, pts, opts, image, s);
    return observers_common<float>(medium, source, dust, obs, n_obs, pts, opts, image, s);
}

int qmcrt_direct_light(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_observer *obs,
                       int32_t subsamples, double weight, const qmcrt_trace_opts *opts, const qmcrt_image *image,
                       void *stream)
{
    g_last_error.clear();
    CHECK_STRUCT(source, qmcrt_source);
    CHECK_STRUCT(opts, qmcrt_trace_opts);
    if (subsamples < 1 || subsamples > 64) return fail(QMCRT_ERR_INVALID_ARG, "subsamples %d outside 1..64", subsamples);
    if (!(weight >= 0) || !std::isfinite(weight)) return fail(QMCRT_ERR_INVALID_ARG, "weight must be finite, >= 0");
    qmcrt_dust dust;
    memset(&dust, 0, sizeof dust);
    dust.struct_size = sizeof dust;
    dust.albedo = 1.0;
    qmcrt_points_desc pts;
    memset(&pts, 0, sizeof pts);
    pts.struct_size = sizeof pts;
    pts.kind = QMCRT_SOBOL;
    pts.dims = 5;
    pts.first_index = 1;
    pts.count = 0;
    qmcrt_trace_opts o = *opts;
    o.max_orders = 1;
    cudaStream_t s = (cudaStream_t)stream;
    if (opts->precision == QMCRT_PREC_F64) {
        qmcrt::TraceP<double> P;
        int rc = fill_trace<double>(medium, source, &dust, obs, &pts, &o, image, 0, P);
        if (rc) return rc;
        return cuda_status(qmcrt::launch_direct_light_f64(P, subsamples, weight, s), "direct_light launch");
    }
    qmcrt::TraceP<float> P;
    int rc = fill_trace<float>(medium, source, &dust, obs, &pts, &o, image, 0, P);
    if (rc) return rc;
    return cuda_status(qmcrt::launch_direct_light_f32(P, subsamples, weight, s), "direct_light launch");
}

uint64_t qmcrt_batch_workspace_bytes(int32_t n_instances)
{
    if (n_instances < 0) return 0;
    return ((uint64_t)(n_instances + 2) * 8 + 255) & ~255ull;
}

int qmcrt_trace_batch(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_observer *obs,
                      const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts, const qmcrt_instance *d_instances,
                      int32_t n_instances, const qmcrt_batch_config *config, void *d_workspace,
                      uint64_t workspace_bytes, const qmcrt_image *image, void *stream)
{
    g_last_error.clear();
    CHECK_STRUCT(medium, qmcrt_medium);
    CHECK_STRUCT(source, qmcrt_source);
    CHECK_STRUCT(obs, qmcrt_observer);
    CHECK_STRUCT(pts, qmcrt_points_desc);
    CHECK_STRUCT(opts, qmcrt_trace_opts);
    CHECK_STRUCT(config, qmcrt_batch_config);
    CHECK_STRUCT(image, qmcrt_image);
    if (!d_instances || !d_workspace) return fail(QMCRT_ERR_INVALID_ARG, "NULL instance table or workspace");
    if (n_instances < 1) return fail(QMCRT_ERR_INVALID_ARG, "n_instances must be >= 1");
    if (workspace_bytes < qmcrt_batch_workspace_bytes(n_instances))
        return fail(QMCRT_ERR_INVALID_ARG, "workspace of %llu bytes < %llu", (unsigned long long)workspace_bytes,
                    (unsigned long long)qmcrt_batch_workspace_bytes(n_instances));
    if (config->chunk_log2 < 7 || config->chunk_log2 > qmcrt::NET_MAX_M)
        return fail(QMCRT_ERR_INVALID_ARG, "chunk_log2 outside 7..%d", qmcrt::NET_MAX_M);
    if (config->block_size != 64 && config->block_size != 128 && config->block_size != 256)
        return fail(QMCRT_ERR_INVALID_ARG, "block_size must be 64, 128 or 256");
    if (config->packets_per_thread < 1 || config->packets_per_thread > 16)
        return fail(QMCRT_ERR_INVALID_ARG, "packets_per_thread outside 1..16");
    if (config->ctas_per_sm < 0) return fail(QMCRT_ERR_INVALID_ARG, "ctas_per_sm must be >= 0");
    if (image->n_images != 1) return fail(QMCRT_ERR_INVALID_ARG, "a batch has one image per instance");
    // the template problem: instance values replace observer angles, dust, opacity and range
    qmcrt_dust dust;
    memset(&dust, 0, sizeof dust);
    dust.struct_size = sizeof dust;
    dust.albedo = 1.0;
    qmcrt_points_desc p = *pts;
    p.first_index = 1;
    p.count = 1ull << config->chunk_log2;
    p.total_n = p.count;
    qmcrt_trace_opts o = *opts;
    o.max_orders = 1;
    o.per_order = 0;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e, "device query");
    const int occ = qmcrt::batch_occupancy(config->block_size, opts->precision);
    const int per_sm = config->ctas_per_sm ? std::min(config->ctas_per_sm, std::max(occ, 1)) : std::max(occ, 1);
    const int ctas = per_sm * sms;
    cudaStream_t s = (cudaStream_t)stream;
    auto *ws = (unsigned long long *)d_workspace;
    // per point kind, and whether a finite star's coordinates 3, 4 are ordered too,
    // built once (read-only after)
    if (pts->kind < QMCRT_SOBOL || pts->kind > QMCRT_FAURE) return fail(QMCRT_ERR_INVALID_ARG, "unknown point kind %d", pts->kind);
    int x0 = -1, x1 = -1, xb = 0;
    if (medium->kind == QMCRT_MEDIUM_GRID && medium->nx > 0 && medium->ny > 0 && medium->nz > 0) {
        const double h[3] = {(medium->hi[0] - medium->lo[0]) / medium->nx, (medium->hi[1] - medium->lo[1]) / medium->ny,
                             (medium->hi[2] - medium->lo[2]) / medium->nz};
        xb = order_extras(source->kind, source->order, source->radius, medium->kind, h, 1, x0, x1);
    } else {
        const double h[3] = {1.0, 1.0, 1.0};
        xb = order_extras(source->kind, source->order, source->radius, medium->kind, h, 1, x0, x1);
    }
    const int ext = xb > 0 ? 1 : 0;
    static qmcrt::NetTables tabs[QMCRT_FAURE + 1][2];
    static std::once_flag once[QMCRT_FAURE + 1][2];
    std::call_once(once[pts->kind][ext], [&] {
        for (int m = qmcrt::NET_MIN_M; m <= qmcrt::NET_MAX_M; ++m)
            make_order(pts->kind, 0, 1ull << m, tabs[pts->kind][ext].ord[m - qmcrt::NET_MIN_M], ext ? 3 : -1,
                       ext ? 4 : -1, ext ? kNetExtraBits : 0);
    });
    qmcrt::NetTables tab = tabs[pts->kind][ext];
    tab.m_cap = config->chunk_log2;
    if (opts->precision == QMCRT_PREC_F64) {
        qmcrt::TraceP<double> P;
        int rc = fill_trace<double>(medium, source, &dust, obs, &p, &o, image, 0, P);
        if (rc) return rc;
        return cuda_status(qmcrt::launch_trace_batch_f64(P, tab, d_instances, n_instances, ws, config->block_size,
                                                         ctas, config->packets_per_thread, s),
                           "trace_batch launch");
    }
    qmcrt::TraceP<float> P;
    int rc = fill_trace<float>(medium, source, &dust, obs, &p, &o, image, 0, P);
    if (rc) return rc;
    return cuda_status(qmcrt::launch_trace_batch_f32(P, tab, d_instances, n_instances, ws, config->block_size, ctas,
                                                     config->packets_per_thread, s),
                       "trace_batch launch");
}

int qmcrt_batch_reduce(const qmcrt_image *image, const qmcrt_instance *d_instances, int32_t n_instances, int32_t nx,
                       int32_t ny, double *d_out, void *stream)
{
    g_last_error.clear();
    CHECK_STRUCT(image, qmcrt_image);
    if (!image->d_accum || !d_instances || !d_out) return fail(QMCRT_ERR_INVALID_ARG, "NULL buffer");
    if (n_instances < 1 || nx < 1 || ny < 1) return fail(QMCRT_ERR_INVALID_ARG, "sizes must be >= 1");
    if (image->accum != QMCRT_ACCUM_I64 || image->frac_bits < 0 || image->frac_bits > 62)
        return fail(QMCRT_ERR_INVALID_ARG, "batch images use fixed-point accumulation with frac_bits 0..62");
    return cuda_status(qmcrt::launch_batch_reduce((const long long *)image->d_accum, d_instances, n_instances,
                                                  (size_t)3 * nx * ny, std::ldexp(1.0, -image->frac_bits), d_out,
                                                  (cudaStream_t)stream),
                       "batch_reduce launch");
}

int qmcrt_gemm_bf16(const void *d_A, const void *d_B, int32_t M, int32_t N, int32_t K,
                    const qmcrt_gemm_epilogue *epilogue, void *stream)
{
    g_last_error.clear();
    CHECK_STRUCT(epilogue, qmcrt_gemm_epilogue);
    if (!d_A || !d_B) return fail(QMCRT_ERR_INVALID_ARG, "NULL operand");
    if (M < 1 || (N != 32 && N != 64 && N != 128) || K < 32 || K % 32)
        return fail(QMCRT_ERR_INVALID_ARG, "shape M=%d N=%d K=%d: need M >= 1, N in {32, 64, 128}, K a multiple of 32",
                    M, N, K);
    if ((reinterpret_cast<uintptr_t>(d_A) | reinterpret_cast<uintptr_t>(d_B)) & 15)
        return fail(QMCRT_ERR_INVALID_ARG, "operands must be 16-byte aligned");
    const int splits = epilogue->k_splits > 1 ? epilogue->k_splits : 1;
    if (splits > 1 && (epilogue->d_bias || epilogue->relu || epilogue->d_mask || epilogue->d_out_bf16 ||
                       epilogue->d_out_bf16_t || !epilogue->d_out_f32))
        return fail(QMCRT_ERR_INVALID_ARG, "a K split only adds into d_out_f32 (no bias, ReLU, mask or BF16 output)");
    if (epilogue->d_out_bf16_t && epilogue->ldt < M) return fail(QMCRT_ERR_INVALID_ARG, "ldt < M");
    if ((reinterpret_cast<uintptr_t>(epilogue->d_mask) | reinterpret_cast<uintptr_t>(epilogue->d_out_f32) |
         reinterpret_cast<uintptr_t>(epilogue->d_out_bf16)) & 15)
        return fail(QMCRT_ERR_INVALID_ARG, "d_mask, d_out_f32 and d_out_bf16 must be 16-byte aligned");
    qmcrt::GemmEpi ep;
    ep.bias = epilogue->d_bias;
    ep.relu = epilogue->relu;
    ep.mask = static_cast<const __nv_bfloat16 *>(epilogue->d_mask);
    ep.out_f32 = epilogue->d_out_f32;
    ep.out_bf16 = static_cast<__nv_bfloat16 *>(epilogue->d_out_bf16);
    ep.out_bf16_t = static_cast<__nv_bfloat16 *>(epilogue->d_out_bf16_t);
    ep.ldt = epilogue->ldt;
    ep.atomic_f32 = splits > 1;
    ep.error = epilogue->d_error;
    return cuda_status(qmcrt::launch_gemm_bf16(static_cast<const __nv_bfloat16 *>(d_A),
                                               static_cast<const __nv_bfloat16 *>(d_B), M, N, K, splits, ep,
                                               (cudaStream_t)stream),
                       "gemm launch");
}

uint64_t qmcrt_sky_workspace_bytes(int32_t nx, int32_t ny, int32_t nz, const double *lo, const double *hi,
                                   double radius)
{
    if (nx < 1 || ny < 1 || nz < 1 || !lo || !hi || !(radius >= 0) || !std::isfinite(radius)) return 0;
    for (int a = 0; a < 3; ++a)
        if (!(hi[a] > lo[a])) return 0;
    return qmcrt::sky_workspace_bytes(nx, ny, nz, qmcrt::sky_dilation(lo, hi, nx, ny, nz, radius * (1.0 + 1e-4)));
}

int qmcrt_sky_bound(const float *d_k, int32_t nx, int32_t ny, int32_t nz, const double *lo, const double *hi,
                    double radius, int32_t m, double *d_map, void *d_workspace, uint64_t workspace_bytes,
                    void *stream)
{
    g_last_error.clear();
    if (!d_k || !lo || !hi || !d_map || !d_workspace) return fail(QMCRT_ERR_INVALID_ARG, "NULL pointer");
    if (nx < 1 || ny < 1 || nz < 1) return fail(QMCRT_ERR_INVALID_ARG, "grid has zero cells");
    for (int a = 0; a < 3; ++a)
        if (!(hi[a] > lo[a])) return fail(QMCRT_ERR_INVALID_ARG, "grid box axis %d is empty", a);
    if (m < 1 || m > 4096) return fail(QMCRT_ERR_INVALID_ARG, "m outside 1..4096");
    if (!(radius >= 0) || !std::isfinite(radius)) return fail(QMCRT_ERR_INVALID_ARG, "radius must be >= 0");
    if (((uintptr_t)d_workspace & 255) != 0) return fail(QMCRT_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    const uint64_t need = qmcrt_sky_workspace_bytes(nx, ny, nz, lo, hi, radius);
    if (workspace_bytes < need)
        return fail(QMCRT_ERR_INVALID_ARG, "workspace of %llu bytes, need %llu", (unsigned long long)workspace_bytes,
                    (unsigned long long)need);
    // the map is built for a radius slightly above the one the trace tests start points
    // against (|p|^2 <= R^2 (1 + 1e-5)), which absorbs the float rounding of a surface point
    return cuda_status(qmcrt::launch_sky_bound(d_k, nx, ny, nz, lo, hi, radius * (1.0 + 1e-4), m, d_map, d_workspace,
                                               (cudaStream_t)stream),
                       "sky_bound launch");
}

uint64_t qmcrt_tail_map_bytes(int32_t nx, int32_t ny, int32_t nz, int32_t pad)
{
    if (nx < 1 || ny < 1 || nz < 1 || pad < 0) return 0;
    return (uint64_t)(nx + 2 * pad) * (ny + 2 * pad) * (nz + 2 * pad);
}

uint64_t qmcrt_tail_workspace_bytes(int32_t nx, int32_t ny, int32_t nz)
{
    if (nx < 1 || ny < 1 || nz < 1) return 0;
    return qmcrt::tail_workspace_bytes(nx, ny, nz);
}

int qmcrt_tail_map(const qmcrt_medium *medium, const qmcrt_observer *obs, uint8_t *d_map, void *d_workspace,
                   uint64_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    if (!medium || medium->struct_size != sizeof(qmcrt_medium))
        return fail(QMCRT_ERR_INVALID_ARG, "medium is NULL or has the wrong struct_size");
    if (!obs || obs->struct_size != sizeof(qmcrt_observer))
        return fail(QMCRT_ERR_INVALID_ARG, "obs is NULL or has the wrong struct_size");
    if (!d_map || !d_workspace) return fail(QMCRT_ERR_INVALID_ARG, "NULL map or workspace");
    if (medium->kind != QMCRT_MEDIUM_GRID || !medium->d_k || medium->pad < QMCRT_MIN_PAD)
        return fail(QMCRT_ERR_INVALID_ARG, "a tail map needs a padded grid medium (pad >= %d)", QMCRT_MIN_PAD);
    const int nx = medium->nx, ny = medium->ny, nz = medium->nz, pad = medium->pad;
    if (nx < 1 || ny < 1 || nz < 1) return fail(QMCRT_ERR_INVALID_ARG, "grid has zero cells");
    if ((double)(nx + 2 * pad) * (ny + 2 * pad) * (nz + 2 * pad) > 2147483647.0)
        return fail(QMCRT_ERR_INVALID_ARG, "padded grid larger than 2^31 cells");
    for (int a = 0; a < 3; ++a)
        if (!(medium->hi[a] > medium->lo[a]) || !std::isfinite(medium->hi[a] - medium->lo[a]))
            return fail(QMCRT_ERR_INVALID_ARG, "grid box axis %d is empty", a);
    if (!std::isfinite(obs->theta) || !std::isfinite(obs->phi))
        return fail(QMCRT_ERR_INVALID_ARG, "observer direction not finite");
    if (((uintptr_t)d_workspace & 255) != 0) return fail(QMCRT_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    const uint64_t need = qmcrt::tail_workspace_bytes(nx, ny, nz);
    if (workspace_bytes < need)
        return fail(QMCRT_ERR_INVALID_ARG, "workspace of %llu bytes, need %llu", (unsigned long long)workspace_bytes,
                    (unsigned long long)need);
    // the direction as the tracer computes it (make_obs); its zero components are exact
    const double st = std::sin(obs->theta), ct = std::cos(obs->theta), sp = std::sin(obs->phi), cp = std::cos(obs->phi);
    const double k[3] = {st * cp, st * sp, ct};
    return cuda_status(qmcrt::launch_tail_map(medium->d_k, nx, ny, nz, pad, medium->lo, medium->hi, k, d_map,
                                              d_workspace, (cudaStream_t)stream),
                       "tail_map launch");
}

int qmcrt_pad_grid(const float *d_k, int32_t nx, int32_t ny, int32_t nz, int32_t pad, float *d_padded, void *stream)
{
    g_last_error.clear();
    if (!d_k || !d_padded) return fail(QMCRT_ERR_INVALID_ARG, "NULL grid pointer");
    if (nx < 1 || ny < 1 || nz < 1) return fail(QMCRT_ERR_INVALID_ARG, "grid has zero cells");
    if (pad < QMCRT_MIN_PAD) return fail(QMCRT_ERR_INVALID_ARG, "pad %d < %d", pad, QMCRT_MIN_PAD);
    if ((double)(nx + 2 * pad) * (ny + 2 * pad) * (nz + 2 * pad) > 2147483647.0)
        return fail(QMCRT_ERR_INVALID_ARG, "padded grid larger than 2^31 cells");
    return cuda_status(qmcrt::launch_pad_grid(d_k, nx, ny, nz, pad, d_padded, (cudaStream_t)stream), "pad_grid launch");
}

int qmcrt_trace_multiple_warped(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                                const qmcrt_observer *obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                                const float *d_x, const float *d_logj, const qmcrt_image *image, float *d_train_log,
                                void *stream)
{
    g_last_error.clear();
    CHECK_STRUCT(source, qmcrt_source);
    if ((d_x == nullptr) != (d_logj == nullptr)) return fail(QMCRT_ERR_INVALID_ARG, "d_x and d_logj go together");
    if (d_x && source->kind != QMCRT_SOURCE_POINT)
        return fail(QMCRT_ERR_UNSUPPORTED, "the warp replaces point-source coordinates only");
    WarpIO w;
    w.x = d_x;
    w.logj = d_logj;
    w.log = d_train_log;
    return trace_common(medium, source, dust, obs, pts, opts, image, nullptr, stream, 1, w);
}

uint64_t qmcrt_wavefront_workspace_bytes(uint64_t max_packets, int32_t precision)
{
    return qmcrt::wavefront_workspace_bytes(max_packets, precision);
}

int qmcrt_trace_multiple_wavefront(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                                   const qmcrt_observer *obs, const qmcrt_points_desc *pts,
                                   const qmcrt_trace_opts *opts, const float *d_x, const float *d_logj,
                                   const qmcrt_image *image, float *d_train_log, void *d_workspace,
                                   uint64_t workspace_bytes, void *stream)
{
    g_last_error.clear();
    CHECK_STRUCT(source, qmcrt_source);
    CHECK_STRUCT(opts, qmcrt_trace_opts);
    CHECK_STRUCT(pts, qmcrt_points_desc);
    if ((d_x == nullptr) != (d_logj == nullptr)) return fail(QMCRT_ERR_INVALID_ARG, "d_x and d_logj go together");
    if (d_x && source->kind != QMCRT_SOURCE_POINT)
        return fail(QMCRT_ERR_UNSUPPORTED, "the warp replaces point-source coordinates only");
    if (!d_workspace) return fail(QMCRT_ERR_INVALID_ARG, "d_workspace is NULL");
    if (((uintptr_t)d_workspace) & 255) return fail(QMCRT_ERR_INVALID_ARG, "d_workspace must be 256-byte aligned");
    WarpIO w;
    w.x = d_x;
    w.logj = d_logj;
    w.log = d_train_log;
    cudaStream_t s = (cudaStream_t)stream;
    if (opts->precision == QMCRT_PREC_F64) {
        qmcrt::TraceP<double> P;
        int rc = fill_trace<double>(medium, source, dust, obs, pts, opts, image, 1, P);
        if (rc) return rc;
        P.log = nullptr;
        return wavefront_run<double>(P, pts, w, d_workspace, workspace_bytes, QMCRT_PREC_F64, s);
    }
    qmcrt::TraceP<float> P;
    int rc = fill_trace<float>(medium, source, dust, obs, pts, opts, image, 1, P);
    if (rc) return rc;
    P.log = nullptr;
    return wavefront_run<float>(P, pts, w, d_workspace, workspace_bytes, QMCRT_PREC_F32, s);
}

int qmcrt_image_reduce(const qmcrt_image *image, int32_t nx, int32_t ny, int32_t n_replicas, double scale,
                       double *d_out, void *stream)
{
    g_last_error.clear();
    CHECK_STRUCT(image, qmcrt_image);
    if (!image->d_accum || !d_out) return fail(QMCRT_ERR_INVALID_ARG, "NULL buffer");
    if (nx < 1 || ny < 1 || image->n_images < 1 || n_replicas < 1)
        return fail(QMCRT_ERR_INVALID_ARG, "sizes must be >= 1");
    if (image->accum != QMCRT_ACCUM_I64 && image->accum != QMCRT_ACCUM_F64)
        return fail(QMCRT_ERR_INVALID_ARG, "unknown accumulation mode %d", image->accum);
    if (image->accum == QMCRT_ACCUM_I64 && (image->frac_bits < 0 || image->frac_bits > 62))
        return fail(QMCRT_ERR_INVALID_ARG, "frac_bits outside 0..62");
    const size_t elems = (size_t)image->n_images * 3 * nx * ny;
    return cuda_status(qmcrt::launch_image_reduce(image->d_accum, image->accum, std::ldexp(1.0, -image->frac_bits), elems,
                                                  n_replicas, scale, d_out, (cudaStream_t)stream),
                       "image_reduce launch");
}

}  // extern "C"

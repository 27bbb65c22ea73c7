/*
 * qmcrt.h -- C ABI of the GB300 (sm_103a) quasi-Monte Carlo radiative-transfer library.
 *
 * The library traces photon packets driven by low-discrepancy point sets through a
 * dusty medium and accumulates their peel-off contributions into Stokes I/Q/U images,
 * the method of S. G. Shulman, "Quasi-Monte Carlo Radiative Transfer" (arXiv:2406.15632).
 * Section numbers below refer to that paper.
 *
 * Conventions for every entry point:
 *  - Return an int status: QMCRT_OK (0) or a negative QMCRT_ERR_* code.  No C++
 *    exception crosses the ABI.  qmcrt_last_error() returns a message for the last
 *    failure on the calling thread (valid until that thread's next call).
 *  - Pointers named d_* are device pointers owned by the caller; pointers to the
 *    descriptor structs are host pointers read during the call only.  The library
 *    allocates no device memory in any entry point.
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Work is enqueued asynchronously on it; the call returns after the launch.
 *    Argument errors are detected on the host before anything is enqueued.
 *  - Every descriptor starts with struct_size, which must equal sizeof(the struct);
 *    a mismatch is QMCRT_ERR_INVALID_ARG (ABI version check).
 *  - Point index i of a packet is its index in the point set; packets are numbered
 *    from first_index (>= 1: the leading zero point is skipped, Sec. 3.1).
 */
#ifndef QMCRT_H
#define QMCRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QMCRT_ABI_VERSION 3

/* ---- status codes ---- */
#define QMCRT_OK 0
#define QMCRT_ERR_INVALID_ARG (-1)    /* a NULL pointer, a size out of range, a bad enum */
#define QMCRT_ERR_UNSUPPORTED (-2)    /* a valid combination the library does not implement */
#define QMCRT_ERR_CUDA (-3)           /* a CUDA runtime call failed (launch, attribute query) */
#define QMCRT_ERR_DEVICE_TIMEOUT (-4) /* a bounded device-side wait gave up */

/* ---- point sets (Sec. 3.1) ---- */
#define QMCRT_SOBOL 0      /* Sobol, Joe-Kuo direction numbers, Gray-code order */
#define QMCRT_SOBOL_OWEN 1 /* Sobol with a hash-based nested uniform (Owen) scramble */
#define QMCRT_HALTON 2     /* Halton, prime bases 2, 3, 5, ... */
#define QMCRT_HAMMERSLEY 3 /* i/N in the first coordinate, Halton in the others */
#define QMCRT_PHILOX 4     /* Philox4x32-10 pseudo-random numbers (Monte Carlo) */
#define QMCRT_NIEDERREITER 5 /* Niederreiter base 2 (irreducible polynomials over GF(2)), natural order */
#define QMCRT_FAURE 6      /* Faure, base = smallest prime >= dims, Pascal-matrix powers */

#define QMCRT_FMT_U32 0 /* raw 32-bit integers (Sobol, scrambled Sobol, Philox only) */
#define QMCRT_FMT_F32 1 /* the FP64 value rounded toward zero to float */
#define QMCRT_FMT_F64 2 /* integers: x * 2^-32 exactly; Halton: correctly rounded b-adic fraction */

#define QMCRT_MAX_DIMS 256 /* coordinates per point */

typedef struct qmcrt_points_desc {
    uint32_t struct_size;
    int32_t kind;         /* QMCRT_SOBOL .. QMCRT_FAURE */
    uint32_t dims;        /* 1 .. QMCRT_MAX_DIMS */
    int32_t format;       /* QMCRT_FMT_* (used by qmcrt_generate_points only) */
    uint64_t first_index; /* >= 1 */
    uint64_t count;       /* points to produce / packets to trace */
    uint64_t total_n;     /* Hammersley: N of the set (first_index + count - 1 <= total_n) */
    uint64_t seed;        /* Owen scramble seed or Philox key */
} qmcrt_points_desc;

/*
 * qmcrt_generate_points -- points first_index .. first_index+count-1 of the set (Sec. 3.1).
 * d_out: device, row-major [count][dims] of uint32, float or double per d->format.
 * Sobol point i is the XOR of the direction numbers over the set bits of the Gray code
 * of i (random access; equal to the sequential construction of Bratley & Fox).
 * Errors: INVALID_ARG for NULL pointers, dims outside 1..QMCRT_MAX_DIMS,
 * first_index == 0, indices >= 2^32 for Sobol kinds, Halton/Hammersley with
 * QMCRT_FMT_U32, a Hammersley index above total_n.
 */
int qmcrt_generate_points(const qmcrt_points_desc *d, void *d_out, void *stream);

/* ---- medium (Sec. 2.1, 3.4) ---- */
#define QMCRT_MEDIUM_GRID 0   /* Cartesian grid, constant kappa*rho per cell */
#define QMCRT_MEDIUM_SPHERE 1 /* homogeneous sphere centred at the origin (analytic chords) */

#define QMCRT_MIN_PAD 8 /* sentinel layers a padded grid needs (qmcrt_pad_grid) */

typedef struct qmcrt_medium {
    uint32_t struct_size;
    int32_t kind;
    const float *d_k;  /* grid: device [nz][ny][nx] extinction kappa*rho per unit length, x fastest;
                          with pad > 0 the [nz+2pad][ny+2pad][nx+2pad] array of qmcrt_pad_grid */
    int32_t nx, ny, nz; /* cells of the grid proper (without padding) */
    int32_t pad;        /* 0, or >= QMCRT_MIN_PAD sentinel layers (faster walk) */
    double lo[3], hi[3]; /* grid box; every packet starts inside it */
    double kscale;       /* multiplier on every cell (opacity at another wavelength) */
    double sphere_r;     /* sphere medium: radius */
    double sphere_k;     /* sphere medium: extinction per unit length */
    const double *d_sky; /* grid, optional (NULL): device map of qmcrt_sky_bound for this grid; rays that
                            start within sky_r of the origin in a direction whose bound (times kscale) is
                            below tau_min / 2 are known not to scatter without walking the grid (same
                            result) */
    int32_t sky_m;       /* texels per face edge of d_sky (1..4096) */
    int32_t sky_reserved;
    double sky_r;        /* the radius d_sky was built for (0 for a point source, the star's radius) */
} qmcrt_medium;

/* ---- source (Sec. 3.2, 3.3) ---- */
#define QMCRT_SOURCE_POINT 0  /* point source at the origin: 3 coordinates (u, v, w) */
#define QMCRT_SOURCE_SPHERE 1 /* star of radius r at the origin: 5 coordinates */
#define QMCRT_ORDER_DIRECT 0  /* emission point, local direction, depth */
#define QMCRT_ORDER_INVERSE 1 /* direction, depth, emission point relative to it */

typedef struct qmcrt_source {
    uint32_t struct_size;
    int32_t kind;
    double radius;  /* star radius (> 0 for a sphere source) */
    double limb_u;  /* linear limb darkening I(mu) ~ 1 - u + u mu, 0 <= u <= 1 */
    int32_t order;  /* QMCRT_ORDER_* */
    int32_t reserved;
} qmcrt_source;

/* ---- dust (Sec. 2.2, 2.3): albedo, HG asymmetry g (|g| < 1), max linear polarization ---- */
typedef struct qmcrt_dust {
    uint32_t struct_size;
    int32_t reserved;
    double albedo, g, p_l;
} qmcrt_dust;

/* ---- observer and image (Sec. 3.6) ---- */
#define QMCRT_SPLAT_NEAREST 0  /* whole contribution to the pixel that holds the point */
#define QMCRT_SPLAT_BILINEAR 1 /* tent weights over the 4 nearest pixel centres */

typedef struct qmcrt_observer {
    uint32_t struct_size;
    int32_t splat;
    double theta, phi;  /* direction toward the observer, polar and azimuth angles */
    double half_width;  /* the image covers [-hw, hw]^2 of the sky plane */
    int32_t nx, ny;     /* pixels */
    const uint8_t *d_tail; /* optional (NULL): device map of qmcrt_tail_map for the medium's padded grid and
                              this direction; peel-off walks toward this observer then stop once the map
                              bounds the optical depth still ahead by opts->tail_eps */
} qmcrt_observer;
/* Sky axes: ex = (-sin phi, cos phi, 0), ey = (-cos theta cos phi, -cos theta sin phi,
 * sin theta); (ex, ey, k) is right-handed.  Stokes Q > 0 along ey, U > 0 along
 * (ey - ex)/sqrt(2).  Pixel (ix, iy) = floor((x + hw) / (2 hw) * n); image layout
 * [n_images][3 = I, Q, U][ny][nx]. */

/* ---- accumulation buffer ---- */
#define QMCRT_ACCUM_I64 0 /* two's-complement fixed point: value = raw * 2^-frac_bits (order-independent) */
#define QMCRT_ACCUM_F64 1 /* IEEE double atomics */

typedef struct qmcrt_image {
    uint32_t struct_size;
    int32_t accum;      /* QMCRT_ACCUM_* */
    void *d_accum;      /* device [n_images][3][ny][nx] int64 or double; contributions are ADDED */
    int32_t n_images;   /* 1, or max_orders with per-order images */
    int32_t frac_bits;  /* I64: 0..62; pick so that |sum| * 2^frac_bits < 2^63 */
} qmcrt_image;

/* ---- trace options ---- */
#define QMCRT_PREC_F32 0 /* march and phase math in float, compensated optical-depth sums */
#define QMCRT_PREC_F64 1 /* everything in double (reference-grade, slow on this part) */
#define QMCRT_FORCE_ALL 0   /* every order forced (weight 1 - e^-tau_edge) */
#define QMCRT_FORCE_FIRST 1 /* only the first order forced; later depths -ln w (Sec. 3.5) */

typedef struct qmcrt_trace_opts {
    uint32_t struct_size;
    int32_t precision;     /* QMCRT_PREC_* */
    double tau_min;        /* packets with tau_1 below this contribute nothing (Sec. 3.2) */
    int32_t max_orders;    /* qmcrt_trace_multiple: scatterings per packet, 1 .. 64 */
    int32_t force_mode;    /* QMCRT_FORCE_* */
    double rr_threshold;   /* Russian roulette when the weight drops below (0: off) */
    double rr_survival;    /* survival probability (0, 1]; survivors' weight / rr_survival */
    int32_t per_order;     /* 1: image k-1 receives scattering order k */
    int32_t block_size;    /* threads per block, 0 = library default (multiple of 32, <= 1024) */
    double tail_eps;       /* observers with a d_tail map: the optical depth (with kscale) a peel-off walk
                              may leave out, >= 0; e^{-tau_obs} then grows by at most that fraction
                              (0: only what the map bounds by zero) */
} qmcrt_trace_opts;

/*
 * qmcrt_trace_single -- single scattering (Sec. 3.2-3.6).  For each packet i:
 * emission from the first coordinates (Eq. point_source_propagation_direction, or the
 * sphere-source orders of Sec. 3.3 with the limb weight); optical depth tau_1 to the
 * grid edge; if tau_1 >= tau_min the packet is forced to scatter with weight
 * 1 - e^{-tau_1} at depth -ln[1 - w (1 - e^{-tau_1})] (Eq. random_depth); the albedo
 * multiplies the weight; the peel-off packet toward the observer carries
 * W0 e^{-tau_obs} P(Theta_obs)/(4 pi) with the White polarization, is hidden if the
 * star blocks its path, and is added to the pixel under its projection.
 * Coordinates: point source (u, v, w) = dims (0, 1, 2); sphere source dims 0..4.
 * pts->dims must be >= the coordinates used; pts->format is ignored.
 * Speed: digital base-2 point sets are traced in net order, one aligned block of 2^m
 * indices at a time (2^m <= count); a range that starts or ends inside such a block
 * launches the whole block, whose threads outside the range only compute their index.
 * first_index a multiple of a power-of-two count traces no such threads.
 * d_log (optional, NULL to skip): device double [count][9] = scattering x, y, z,
 * peel-off I, Q, U, sky x, y, status (0 contributed, 1 tau_1 < tau_min, 2 occulted).
 * Errors: INVALID_ARG (NULL descriptors, bad sizes or enums, |g| >= 1, albedo outside
 * [0,1], a grid with NULL d_k or zero cells, first_index == 0), CUDA.
 */
int qmcrt_trace_single(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                       const qmcrt_observer *obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                       const qmcrt_image *image, double *d_log, void *stream);

/*
 * qmcrt_trace_multiple -- multiple scattering (Sec. 3.5, 3.7).
 * Order k (1-based) reads coordinates 4(k-1) + {0: azimuth i1 = 2 pi u (emission
 * phi at k = 1), 1: cos Theta from the HG inverse (emission theta at k = 1), 2: depth,
 * 3: roulette}.  After the peel-off of order k the packet is rouletted if its weight
 * is below rr_threshold, then scattered: the direction from HG, the Stokes vector
 * rotated into the scattering plane and multiplied by M(Theta)/P11.  Orders stop at
 * max_orders, at tau_edge < tau_min, on leaving the grid (FORCE_FIRST) or by roulette.
 * A sphere source (the paper treats it in single scattering only, Sec. 7) emits as in
 * qmcrt_trace_single with coordinates 0, 1 (emission point in the direct order,
 * direction in the inverse order) and 2 (first depth); its other two emission
 * coordinates are 4 max_orders and 4 max_orders + 1.  Later flights are not stopped by
 * the star; peel-offs it hides are dropped.  pts->dims must be >= 4 * max_orders (+ 2
 * for a sphere source).  image->n_images must be max_orders when per_order is set,
 * else 1.
 * Errors: as qmcrt_trace_single.
 */
int qmcrt_trace_multiple(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                         const qmcrt_observer *obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                         const qmcrt_image *image, void *stream);

/* ---- batches of problems in one launch ---- */
typedef struct qmcrt_instance {  /* device-resident table entry, 72 bytes */
    double theta, phi;       /* direction toward this instance's observer */
    double albedo, g, p_l;   /* dust at this instance's wavelength (as qmcrt_dust) */
    double kscale;           /* opacity multiplier (times qmcrt_medium.kscale) */
    uint64_t first_index;    /* first point index (>= 1); aligned to count keeps chunks full */
    uint64_t count;          /* packet budget */
    const uint8_t *d_tail;   /* optional (NULL): qmcrt_tail_map of this direction on the medium's padded grid
                                (as qmcrt_observer.d_tail, with opts->tail_eps; unused on a plain grid) */
} qmcrt_instance;

typedef struct qmcrt_batch_config {
    uint32_t struct_size;
    int32_t chunk_log2;          /* largest work chunk, 2^chunk_log2 indices (7..28); an instance
                                    uses chunks of min(2^chunk_log2, largest power of 2 <= budget) */
    int32_t block_size;          /* threads per CTA: 64, 128 or 256 */
    int32_t ctas_per_sm;         /* resident CTAs per SM (0 = as many as fit) */
    int32_t packets_per_thread;  /* packets a thread traces per work tile (1..16) */
    int32_t reserved;
} qmcrt_batch_config;

/* Bytes of device workspace qmcrt_trace_batch needs for n_instances instances. */
uint64_t qmcrt_batch_workspace_bytes(int32_t n_instances);

/*
 * qmcrt_trace_batch -- single scattering (as qmcrt_trace_single, Sec. 3.2-3.6) for
 * n_instances problems that share the medium and the source but differ in observer,
 * dust (wavelength), opacity and packet budget, in one persistent launch: a fixed grid
 * of CTAs pulls work tiles (instance, aligned chunk of indices, tile) from a
 * counter in d_workspace until every budget is traced.  The work order is derived on
 * the device from d_instances, so the call can be captured in a CUDA graph and
 * replayed.  obs gives the image geometry (nx, ny, half_width, splat; theta and phi
 * are taken from the instances); pts gives the point kind, dims, seed (first_index,
 * count and total_n come from the instances: a Hammersley instance uses N = its last
 * index); opts gives precision and tau_min.
 * d_instances: device qmcrt_instance[n_instances] (caller-owned, unchanged).
 * image->d_accum: device [n_instances][3][ny][nx] (n_images must be 1); contributions
 * are added.  d_workspace: device, >= qmcrt_batch_workspace_bytes(n_instances).
 * The instance values are not checked (they live on the device): |g| < 1, albedo and
 * p_l in [0, 1], kscale > 0 and index ranges below 2^32 are the caller's duty.
 * Errors: INVALID_ARG (NULL pointers, bad sizes or config, small workspace),
 * UNSUPPORTED (a multiple-scattering option), CUDA.
 */
int qmcrt_trace_batch(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_observer *obs,
                      const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts, const qmcrt_instance *d_instances,
                      int32_t n_instances, const qmcrt_batch_config *config, void *d_workspace,
                      uint64_t workspace_bytes, const qmcrt_image *image, void *stream);

/*
 * qmcrt_batch_reduce -- d_out[i][s][y][x] = raw[i][s][y][x] * 2^-frac_bits / count_i for
 * every instance i (fixed-point accumulation only): the batch's images in units of
 * the source luminosity.  d_out: device double [n_instances][3][ny][nx].
 * Errors: INVALID_ARG, CUDA.
 */
int qmcrt_batch_reduce(const qmcrt_image *image, const qmcrt_instance *d_instances, int32_t n_instances, int32_t nx,
                       int32_t ny, double *d_out, void *stream);

/* ---- tensor-core GEMM (building block of the learned proposal) ---- */
typedef struct qmcrt_gemm_epilogue {
    uint32_t struct_size;
    int32_t relu;            /* max(0, .) after the bias */
    const float *d_bias;     /* [N] or NULL */
    const void *d_mask;      /* bf16 [M][N] or NULL: zero where mask <= 0 (ReLU backward) */
    float *d_out_f32;        /* [M][N] or NULL */
    void *d_out_bf16;        /* bf16 [M][N] or NULL */
    void *d_out_bf16_t;      /* bf16 [N][ldt] or NULL: the transpose of the result */
    int32_t ldt;             /* row length of d_out_bf16_t, >= M */
    int32_t k_splits;        /* > 1: split K over CTAs and add into d_out_f32 atomically (no bias) */
    int32_t *d_error;        /* set to 1 if a tensor-core wait gives up (NULL: not reported) */
} qmcrt_gemm_epilogue;

/*
 * qmcrt_gemm_bf16 -- D[M][N] = A[M][K] . B[N][K]^T on the tensor cores (BF16 inputs, FP32
 * accumulation), then the epilogue (bias, ReLU, ReLU mask, FP32 / BF16 / transposed
 * BF16 outputs).  A, B: device bf16, row-major, K contiguous, 16-byte aligned; the mask
 * and the FP32 / BF16 outputs 16-byte aligned too.  The paper has no counterpart; it is
 * the building block of the learned warp's network.
 * Errors: INVALID_ARG (NULL pointers, M < 1, N not 32/64/128, K not a positive multiple
 * of 32, ldt < M, bias with k_splits > 1, misaligned pointers), CUDA.
 */
int qmcrt_gemm_bf16(const void *d_A, const void *d_B, int32_t M, int32_t N, int32_t K,
                    const qmcrt_gemm_epilogue *epilogue, void *stream);

/* ---- learned proposal: a trained warp of the first-scattering coordinates ----
 * The paper has no counterpart.  x = T(u) on the unit cube, autoregressive and
 * piecewise linear with QMCRT_WARP_BINS bins per coordinate (after Mueller et al.,
 * "Neural Importance Sampling", 2019): x0 follows the learned pdf softmax(theta0);
 * x1 the pdf given by MLP0(one-blob(x0)); x2 the pdf given by MLP1(one-blob(x0),
 * one-blob(x1)).  Each MLP has 4 layers of width 128 with ReLU (input 128 features:
 * 32 one-blob bins per conditioning coordinate, zero padded; output 32 logits).
 * Parameter vector (FP32, QMCRT_WARP_PARAMS): theta0[32], then for m = 0, 1 and layer
 * l = 0..3 the weight W[m][l] (out x in row-major: 128x128, 128x128, 128x128, 32x128)
 * followed by its bias b[m][l] (out).  The bf16 blobs hold the 8 weight matrices in the
 * same order (QMCRT_WARP_BF16_WEIGHTS values), as is and transposed. */
#define QMCRT_WARP_BINS 32
#define QMCRT_WARP_WIDTH 128
#define QMCRT_WARP_PARAMS 107360
#define QMCRT_WARP_BF16_WEIGHTS 106496

typedef struct qmcrt_warp {
    uint32_t struct_size;
    float uniform_mix;   /* defensive mixture: bin masses (1 - mix) softmax + mix / 32, in [0, 1);
                            bounds |dx/du| by mix^-3 */
    float *d_params;     /* device FP32 [QMCRT_WARP_PARAMS] */
    void *d_weights;     /* device bf16 [QMCRT_WARP_BF16_WEIGHTS] (refreshed by qmcrt_warp_sync) */
    void *d_weights_t;   /* device bf16 [QMCRT_WARP_BF16_WEIGHTS], the transposes */
    int32_t *d_error;    /* device int or NULL: set to 1 if a tensor-core wait gives up */
} qmcrt_warp;

typedef struct qmcrt_adam {
    uint32_t struct_size;
    int32_t step;        /* 1, 2, ... (bias correction) */
    double lr, beta1, beta2, eps;
} qmcrt_adam;

/* Device workspace bytes for the warp calls processing up to `rows` samples per pass. */
uint64_t qmcrt_warp_workspace_bytes(uint64_t rows);

/* Refresh the bf16 weight copies (as is and transposed) from the FP32 parameters. */
int qmcrt_warp_sync(const qmcrt_warp *warp, void *stream);

/*
 * qmcrt_warp_forward -- d_x[n][3] = T(d_u[n][3]) and d_logj[n] = log |det dx/du| =
 * -log q(x), for points u in [0,1]^3 (FP32, row-major).  The MLPs run on the tensor
 * cores (bf16 weights and activations, FP32 accumulation), in passes of as many rows as
 * the workspace holds.  Errors: INVALID_ARG (NULL pointers, workspace below one pass of
 * 128 rows), CUDA.
 */
int qmcrt_warp_forward(const qmcrt_warp *warp, const float *d_u, float *d_x, float *d_logj, uint64_t n,
                       void *d_workspace, uint64_t workspace_bytes, void *stream);

/*
 * qmcrt_warp_grad -- gradient of the cross-entropy loss -sum_j w_j log q(x_j) / sum_j w_j
 * over logged samples (d_x[n][3], weights d_w[n] >= 0: a packet's contribution divided
 * by the density it was drawn from), ADDED into d_grad[QMCRT_WARP_PARAMS]; the loss is
 * added into *d_loss.  Forward and backward passes on the tensor cores.
 * Errors: as qmcrt_warp_forward.
 */
int qmcrt_warp_grad(const qmcrt_warp *warp, const float *d_x, const float *d_w, uint64_t n, float *d_grad,
                    float *d_loss, void *d_workspace, uint64_t workspace_bytes, void *stream);

/* One Adam step on warp->d_params from d_grad (moments d_m, d_v, FP32
 * [QMCRT_WARP_PARAMS]), then qmcrt_warp_sync.  Errors: INVALID_ARG, CUDA. */
int qmcrt_warp_adam(const qmcrt_warp *warp, const float *d_grad, float *d_m, float *d_v, const qmcrt_adam *opt,
                    void *stream);

/*
 * qmcrt_pad_grid -- prepares a grid for the faster walk (Sec. 3.4 optical-depth
 * integration, unchanged in result): writes d_padded, device float
 * [nz+2pad][ny+2pad][nx+2pad], the cells of d_k ([nz][ny][nx]) surrounded by pad layers
 * of the sentinel value -0.0 (negative zero); interior cells that are zero, negative or
 * NaN are written as +0.0, so only sentinels carry a sign bit.  Pass d_padded with
 * qmcrt_medium.pad = pad.
 * Errors: INVALID_ARG (NULL pointers, empty grid, pad < QMCRT_MIN_PAD, more than 2^31
 * padded cells), CUDA.
 */
int qmcrt_pad_grid(const float *d_k, int32_t nx, int32_t ny, int32_t nz, int32_t pad, float *d_padded, void *stream);

/*
 * qmcrt_direct_light -- adds the source's direct (unscattered) light to image 0 of the
 * accumulator, integrated from the source toward the observer (Sec. 3.4), Stokes I
 * only, multiplied by `weight` (images are raw sums over packets: weight = N makes the
 * direct light appear once after qmcrt_image_reduce's 1/N).  Units: source luminosity
 * per steradian.  Point source: e^-tau(0 -> observer) / (4 pi), binned at the sky
 * origin with the observer's splat.  Sphere source (radius R, limb darkening u): the
 * visible disk's surface brightness (1 - u + u mu) / (1 - u/3) / (4 pi) / (pi R^2) per
 * unit sky area, attenuated from the visible surface point, integrated over each pixel
 * by a subsamples x subsamples midpoint rule.  opts: only precision is read.
 * Errors: INVALID_ARG (descriptors as qmcrt_trace_single, subsamples outside 1..64,
 * weight negative or not finite, image->n_images != 1), CUDA.
 */
int qmcrt_direct_light(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_observer *obs,
                       int32_t subsamples, double weight, const qmcrt_trace_opts *opts, const qmcrt_image *image,
                       void *stream);

/*
 * qmcrt_trace_observers -- one trace feeding several observers (Sec. 3.6: the peel-off
 * is repeated toward each observer from the same scattering events).  Emission,
 * forced depths and scattering are done once per packet; the optical depth toward
 * each observer, its peel-off contribution and its binning are done per observer.
 * obs: host array of n_obs (1..QMCRT_MAX_OBSERVERS) observers with equal nx, ny and
 * splat (angles and half widths may differ).  opts->max_orders == 1 gives single
 * scattering with the semantics of qmcrt_trace_single (any source); > 1 gives
 * multiple scattering as qmcrt_trace_multiple (point source).  image->d_accum holds
 * n_obs image stacks one after another: [n_obs][n_images][3][ny][nx]; stack o receives
 * observer o and equals, value for value, what the single-observer call with obs[o]
 * writes.  Errors: as qmcrt_trace_single / qmcrt_trace_multiple; INVALID_ARG for n_obs
 * outside the range or observers of different image shape.
 */
#define QMCRT_MAX_OBSERVERS 16
int qmcrt_trace_observers(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                          const qmcrt_observer *obs, int32_t n_obs, const qmcrt_points_desc *pts,
                          const qmcrt_trace_opts *opts, const qmcrt_image *image, void *stream);

/*
 * qmcrt_trace_multiple_warped -- qmcrt_trace_multiple with the learned proposal: packet
 * j (point index first_index + j) takes its first-order coordinates (emission phi,
 * theta and first depth) from d_x[j][3] (x = T(u) from qmcrt_warp_forward) and
 * multiplies its weight by exp(d_logj[j]) = |dx/du|, which keeps the estimator
 * unbiased; the other orders read the point set as usual.  With d_x = d_logj = NULL
 * it is qmcrt_trace_multiple.  d_train_log (optional, device float [count][5]): per
 * packet the first-order coordinates used, then two norms of the Stokes-I
 * contributions its peel-offs put into the image over all orders: their sum and the
 * square root of their sum of squares -- the samples and weights qmcrt_warp_grad
 * trains on (weights include |dx/du|, i.e. f / q of the proposal that drew them).
 * Errors: as qmcrt_trace_multiple; INVALID_ARG if only one of d_x, d_logj is given;
 * UNSUPPORTED for a warp with a sphere source.
 */
int qmcrt_trace_multiple_warped(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                                const qmcrt_observer *obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                                const float *d_x, const float *d_logj, const qmcrt_image *image, float *d_train_log,
                                void *stream);

/*
 * qmcrt_trace_multiple_wavefront -- qmcrt_trace_multiple_warped computed order by order:
 * every scattering order is one pass over the packets still alive, and between orders
 * the live packets are regrouped by position and direction so that a warp traces
 * similar rays (Sec. 3.5, 3.7; the per-packet arithmetic is the same, so fixed-point
 * images equal qmcrt_trace_multiple's / _warped's bit for bit).  d_x, d_logj,
 * d_train_log: as qmcrt_trace_multiple_warped (may be NULL).  d_workspace: device
 * memory, 256-byte aligned, of workspace_bytes; the packets are processed in chunks of
 * the largest power of two whose qmcrt_wavefront_workspace_bytes fits.
 * Errors: as qmcrt_trace_multiple_warped; INVALID_ARG for a NULL, misaligned or too
 * small workspace.
 */
uint64_t qmcrt_wavefront_workspace_bytes(uint64_t max_packets, int32_t precision);
int qmcrt_trace_multiple_wavefront(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                                   const qmcrt_observer *obs, const qmcrt_points_desc *pts,
                                   const qmcrt_trace_opts *opts, const float *d_x, const float *d_logj,
                                   const qmcrt_image *image, float *d_train_log, void *d_workspace,
                                   uint64_t workspace_bytes, void *stream);

/*
 * qmcrt_image_reduce -- final image in units of the source luminosity (Sec. 3.6):
 * d_out[j] = sum over the n_replicas accumulation buffers (each image->n_images x 3 x
 * ny x nx, consecutive in memory from image->d_accum) of raw[j] * 2^-frac_bits
 * (I64) or raw[j] (F64), times scale (normally 1/N).  d_out: device double, same
 * layout as one buffer.
 * Errors: INVALID_ARG (NULL pointers, sizes <= 0, n_replicas < 1), CUDA.
 */
int qmcrt_image_reduce(const qmcrt_image *image, int32_t nx, int32_t ny, int32_t n_replicas, double scale,
                       double *d_out, void *stream);

/*
 * qmcrt_sky_bound -- for a source at the origin (Sec. 3.2, 3.3: a point, radius 0, or a
 * star of that radius): d_map, device double [6][m][m], receives per cube-map texel an upper
 * bound on the optical depth (kappa rho without kscale) of every ray that starts within
 * `radius` of the origin and whose direction falls in the texel.  Face f = 2 a + (d_a < 0)
 * for the direction's major axis a (ties to the lower axis); u, v are the other two
 * components (increasing axis order) over |d_a|; texel (iu, iv) = (floor((u + 1) m / 2),
 * floor((v + 1) m / 2)).  Construction: such a ray stays within radius + t alpha of the
 * texel's centre ray (alpha: the texel's angular radius), hence, while that is at most D
 * smallest cell edges (D = 1 + ceil(radius / h_min)), within D cells of the centre ray's
 * cell at equal t; the map holds the integral, along the centre ray, of the grid maximised
 * over (2 D + 1)^3 neighbourhoods (times 1 + 1e-6).  A texel whose cone is wider than that
 * (too coarse a map for the grid: m below about 1.2 x the cells per axis) holds +inf.
 * d_k: device [nz][ny][nx] grid (not padded); lo, hi: host [3], the grid box; d_workspace:
 * device, 256-byte aligned, >= qmcrt_sky_workspace_bytes (two grids grown by D layers).
 * Pass the map in qmcrt_medium.d_sky with sky_r = radius: a forced step that starts within
 * that radius of the origin then skips its walks when 2 x bound x kscale < tau_min, which
 * is exactly when the walk's tau_1 would fall below tau_min.  Rebuild the map whenever the
 * grid changes.
 * Errors: INVALID_ARG (NULL pointers, empty grid or box, m outside 1..4096, radius
 * negative or not finite, a small or misaligned workspace), CUDA.
 */
uint64_t qmcrt_sky_workspace_bytes(int32_t nx, int32_t ny, int32_t nz, const double *lo, const double *hi,
                                   double radius);
int qmcrt_sky_bound(const float *d_k, int32_t nx, int32_t ny, int32_t nz, const double *lo, const double *hi,
                    double radius, int32_t m, double *d_map, void *d_workspace, uint64_t workspace_bytes,
                    void *stream);

/*
 * qmcrt_tail_map -- for an observer direction k (Sec. 3.6: the peel-off walks all run
 * along k): d_map, device uint8 [nz+2pad][ny+2pad][nx+2pad] (the padded grid's layout,
 * qmcrt_tail_map_bytes), receives per cell a code c bounding the optical depth (kappa rho
 * without kscale) from any point of the cell along k to the edge of the grid: c = 0, no
 * depth; 1 <= c <= 254, at most 2^(c - 150); 255, no bound.  Padding cells hold 0.
 * Construction: the grid's cells are grouped in 4^3 blocks, each holding the largest value
 * of its cells; slabs of blocks are taken across the axis a of largest |k_a| / h_a, so that
 * along each other axis the walk's cells move by at most one block width per slab (plus one
 * cell of rounding), that is over at most three blocks (one where k has no component); a
 * ray from a block crosses its slab over at most 4 h_a / |k_a| and enters the next slab in
 * one of those lateral blocks, so the bound of a block is that length (times 1 + 1e-6)
 * times the largest value among its slab's lateral blocks, plus the largest bound among
 * the next slab's, summed slab by slab from the side k leaves through (upward roundings).
 * medium: a grid with pad >= QMCRT_MIN_PAD (d_k the padded array of qmcrt_pad_grid);
 * obs: theta and phi give k, as the tracer computes it; d_workspace: device, 256-byte
 * aligned, >= qmcrt_tail_workspace_bytes (two arrays of block values).  Pass the map in
 * qmcrt_observer.d_tail: a peel-off walk toward that observer checks, with the density
 * loads of each batch of cells, the code of the batch's first cell and stops after the
 * batch once 2^(c - 150) kscale <= opts->tail_eps (or c = 0).  Rebuild the map whenever the
 * grid or the direction changes.  The walk's optical depth then falls short of the full
 * walk's by at most tail_eps.
 * Errors: INVALID_ARG (NULL pointers or wrong struct_size, a medium that is not a padded
 * grid, an empty box, a direction that is not finite, a small or misaligned workspace),
 * CUDA.
 */
uint64_t qmcrt_tail_map_bytes(int32_t nx, int32_t ny, int32_t nz, int32_t pad);
uint64_t qmcrt_tail_workspace_bytes(int32_t nx, int32_t ny, int32_t nz);
int qmcrt_tail_map(const qmcrt_medium *medium, const qmcrt_observer *obs, uint8_t *d_map, void *d_workspace,
                   uint64_t workspace_bytes, void *stream);

/*
 * qmcrt_contribution_bound -- *bound = the largest |I|, |Q| or |U| one peel-off
 * contribution can carry (Sec. 2.2, 3.5, 3.6), for the source (limb weight at most
 * 1 / (1 - u/3)), dust and options given; multiple != 0 takes opts->max_orders orders and
 * the roulette (a survivor's weight below rr_threshold grows by 1 / rr_survival), 0 one
 * order.  Each scattering multiplies I by at most albedo (1 + p_l) (forcing weight <= 1,
 * M/P11 with |Q| <= I); the peel-off adds the largest HG value (1 + |g|) / (4 pi
 * (1 - |g|)^2): order k is below limb p_max max(1, thr / surv) (albedo (1 + p_l))^k, and
 * the bound is its largest value over k <= the orders.
 * Errors: INVALID_ARG (NULL pointers or wrong struct_size, dust or limb_u out of range,
 * max_orders outside 1..64 or rr_survival outside (0, 1] when multiple).
 */
int qmcrt_contribution_bound(const qmcrt_source *source, const qmcrt_dust *dust, const qmcrt_trace_opts *opts,
                             int32_t multiple, double *bound);

/*
 * qmcrt_default_frac_bits -- *frac_bits = the largest F in 0..62 for which an int64
 * fixed-point image (QMCRT_ACCUM_I64, value = raw 2^-F) cannot overflow when n_packets
 * packets are added: n_packets x (contributions per packet and pixel: max_orders for
 * multiple scattering into one image, else 1) x qmcrt_contribution_bound x weight_bound
 * x 2^F <= 2^62.  weight_bound (>= 1) bounds an extra factor on every packet's weight:
 * 1 for plain QMC, mix^-3 for a learned warp with uniform mixture mix (|dx/du| <= mix^-3).
 * Errors: as qmcrt_contribution_bound; INVALID_ARG for NULL frac_bits or weight_bound
 * not finite or below 1.
 */
int qmcrt_default_frac_bits(const qmcrt_source *source, const qmcrt_dust *dust, const qmcrt_trace_opts *opts,
                            int32_t multiple, uint64_t n_packets, double weight_bound, int32_t *frac_bits);

/* ---- single scattering with host-resident inputs and outputs ---- */
typedef struct qmcrt_host_io {
    uint32_t struct_size;
    int32_t reserved;
    const float *h_k;   /* host [nz][ny][nx] grid copied in by the call, or NULL to keep the device grid */
    float *d_k;         /* device [nz][ny][nx] receiving h_k when medium->pad > 0 (then padded into
                           medium->d_k); unused when pad == 0 (h_k goes straight to medium->d_k) */
    void *d_accum;      /* device int64 [3][ny][nx]: fixed-point scratch, cleared by the call */
    double *d_image;    /* device [3][ny][nx]: the reduced image */
    double *h_image;    /* host [3][ny][nx]: receives the image (pinned memory keeps the call asynchronous) */
    void *d_sky_ws;     /* device workspace of qmcrt_sky_bound (needed when medium->d_sky is given) */
    uint64_t sky_ws_bytes;
    void *d_tail_ws;    /* device workspace of qmcrt_tail_map (needed when obs->d_tail is given) */
    uint64_t tail_ws_bytes;
} qmcrt_host_io;

/*
 * qmcrt_render_single_host -- one end-to-end single-scattering render for a caller whose
 * inputs and outputs live in host memory (Sec. 3.2-3.6): enqueues on stream the copy of
 * io->h_k to the device (one cudaMemcpyAsync), its sentinel padding (qmcrt_pad_grid,
 * when medium->pad > 0), bound map (qmcrt_sky_bound into medium->d_sky, when given) and
 * tail map (qmcrt_tail_map into obs->d_tail, when given), the clearing of io->d_accum,
 * qmcrt_trace_single with fixed-point
 * accumulation at frac_bits, qmcrt_image_reduce with scale (normally 1/N) into
 * io->d_image, and the copy of that image to io->h_image (one cudaMemcpyAsync).  The
 * call returns after enqueuing: synchronize the stream before reading h_image.  The
 * device buffers are the caller's; the library allocates nothing.
 * Errors: as qmcrt_trace_single; INVALID_ARG for a NULL or mis-sized io, NULL d_accum,
 * d_image or h_image, h_k for a sphere medium, a padded medium without d_k or with
 * d_k == medium->d_k, a medium with a bound map without a large enough, 256-byte aligned
 * d_sky_ws, an observer with a tail map without such a d_tail_ws; CUDA for a failed copy.
 */
int qmcrt_render_single_host(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                             const qmcrt_observer *obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                             const qmcrt_host_io *io, int32_t frac_bits, double scale, void *stream);

/*
 * qmcrt_trace_single_noalloc -- qmcrt_trace_single followed by qmcrt_image_reduce for
 * one image, for callers that cannot allocate device memory: code embedded in a host
 * application that owns every device allocation through its own pool, or code that
 * must not allocate once running (an allocation can synchronize the device, or fail
 * under memory pressure at a bad moment).  The paper has no counterpart; this is a
 * convenience of the library.
 * The fixed-point accumulation scratch is a device array inside the library (3 x
 * QMCRT_NOALLOC_MAX_PIXELS int64 values, 6 MiB, held on every GPU that loads the
 * library until the process exits); nothing is allocated.  The caller passes the
 * descriptors of qmcrt_trace_single, the fixed-point scale frac_bits (as in
 * qmcrt_image), the final scale (normally 1/N) and d_image: device double
 * [3][ny][nx], overwritten with the image.
 * Every call clears the part of the scratch it uses, then traces and reduces on
 * stream.  All calls share the one scratch array: calls whose work overlaps on the
 * GPU (other streams, other host threads) race and corrupt each other's images.
 * Every call looks up the scratch's device address with the caller's device current
 * (after a cudaDeviceReset the array has a new address, so none is cached); the first
 * lookup on a device may load the library's kernels, so make the first call before
 * any stream capture.  All arguments are checked before anything is enqueued.
 * Errors: as qmcrt_trace_single; INVALID_ARG for NULL d_image or an image of more than
 * QMCRT_NOALLOC_MAX_PIXELS pixels; CUDA if the scratch address cannot be found.
 */
#define QMCRT_NOALLOC_MAX_PIXELS (512 * 512)
int qmcrt_trace_single_noalloc(const qmcrt_medium *medium, const qmcrt_source *source, const qmcrt_dust *dust,
                               const qmcrt_observer *obs, const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                               int32_t frac_bits, double scale, double *d_image, void *stream);

/* Thread-local message describing the last error (empty if none). */
const char *qmcrt_last_error(void);

/* QMCRT_ABI_VERSION of the loaded library. */
int qmcrt_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QMCRT_H */

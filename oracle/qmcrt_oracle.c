/*
 * qmcrt_oracle.c -- plain FP64 CPU oracle for quasi-Monte Carlo radiative transfer
 * (S. G. Shulman, "Quasi-Monte Carlo Radiative Transfer", arXiv:2406.15632).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file: it is
 * loaded by the tests, by the smoke check and by the benchmark's CPU-baseline leg.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Every routine is written to be checked against the paper by eye: one packet at a
 * time, one grid cell at a time, in double precision, in the order the paper gives
 * the steps.  Speed is not a goal; the only concession is that independent packet
 * ranges may run on separate threads, each with its own image, summed in a fixed
 * order at the end.
 *
 * Sections of the paper followed:
 *   Sec. 3.1  point generators (Sobol, Halton, Hammersley; leading zeros skipped)
 *   Sec. 3.2  point source emission (Eq. point_source_propagation_direction) and the
 *             forced first scattering (Eq. random_depth)
 *   Sec. 3.3  sphere source, direct and inverse number order
 *   Sec. 3.4  optical depth along a ray through a Cartesian grid; march to a depth
 *   Sec. 3.5  Henyey-Greenstein scattering angle and azimuth; unforced depth -ln w
 *   Sec. 3.6  peel-off weight W = W0 exp(-tau_obs) p_obs and image binning
 *   Sec. 3.7  one long quasi-random vector per packet, fixed coordinate per purpose
 *   Sec. 2.2  Stokes vector, Mueller matrix with the White (1979) approximation
 * Readings where the paper is silent are listed in the design notes; the ones that
 * matter for a line of code are repeated at that line.
 *
 * Parity pins: every function here is pinned by a CPU test against something other
 * than itself (closed forms, library routines, brute force, invariants).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------ */
/* Point generators (Sec. 3.1)                                                      */
/* ------------------------------------------------------------------------------ */

enum { OR_SOBOL = 0, OR_SOBOL_OWEN = 1, OR_HALTON = 2, OR_HAMMERSLEY = 3, OR_PHILOX = 4, OR_NIEDERREITER = 5,
       OR_FAURE = 6 };

/*
 * Sobol direction numbers after Bratley & Fox (1988) with the Joe & Kuo (2008)
 * primitive polynomials and initial values.  poly[d] holds the polynomial
 * x^s + a_1 x^(s-1) + ... + a_(s-1) x + 1 as the integer whose bits are
 * 1 a_1 ... a_(s-1) 1; minit[d*stride + j] is m_(j+1).  Dimension 0 is the
 * van der Corput sequence (all m_k = 1).  V[d*32 + k] is the direction number used
 * by bit k of the Gray-code index: V = m_(k+1) * 2^(31-k).
 * m_k = 2 a_1 m_(k-1) ^ 4 a_2 m_(k-2) ^ ... ^ 2^(s-1) a_(s-1) m_(k-s+1)
 *       ^ 2^s m_(k-s) ^ m_(k-s).
 */
int or_sobol_directions(int dims, const int64_t *poly, const int64_t *minit, int stride,
                        uint32_t *V)
{
    for (int d = 0; d < dims; ++d) {
        uint64_t m[33];
        if (d == 0) {
            for (int k = 1; k <= 32; ++k) m[k] = 1;
        } else {
            int64_t p = poly[d];
            int s = 0;
            while ((p >> (s + 1)) != 0) ++s; /* degree = bit length - 1 */
            if (s < 1 || s > stride) return -1;
            for (int k = 1; k <= s && k <= 32; ++k) m[k] = (uint64_t)minit[(int64_t)d * stride + (k - 1)];
            for (int k = s + 1; k <= 32; ++k) {
                uint64_t v = m[k - s] ^ (m[k - s] << s);
                for (int j = 1; j <= s - 1; ++j) {
                    int a_j = (int)((p >> (s - j)) & 1);
                    if (a_j) v ^= m[k - j] << j;
                }
                m[k] = v;
            }
        }
        for (int k = 1; k <= 32; ++k) {
            if ((m[k] & 1) == 0 || m[k] >= ((uint64_t)1 << k)) return -2; /* m_k odd, < 2^k */
            V[d * 32 + (k - 1)] = (uint32_t)(m[k] << (32 - k));
        }
    }
    return 0;
}

/* Sobol point i, dimension d, as a 32-bit integer: XOR of the direction numbers over
 * the set bits of the Gray code g = i ^ (i >> 1).  Point i of this ordering equals the
 * i-th point of the sequential Antonov-Saleev recurrence. */
uint32_t or_sobol_u32(const uint32_t *V, int d, uint64_t i)
{
    uint64_t g = i ^ (i >> 1);
    uint32_t x = 0;
    for (int k = 0; k < 32; ++k)
        if ((g >> k) & 1) x ^= V[d * 32 + k];
    return x;
}

static uint32_t or_reverse32(uint32_t x)
{
    uint32_t r = 0;
    for (int b = 0; b < 32; ++b)
        if ((x >> b) & 1) r |= 1u << (31 - b);
    return r;
}

/* ---- Niederreiter base 2 (Niederreiter 1988; Bratley, Fox & Niederreiter 1992) ----
 * Polynomials over GF(2) are integers, bit i = coefficient of x^i.  Dimension j uses the
 * j-th irreducible polynomial p_j in the order of degree, then value (x, x + 1,
 * x^2 + x + 1, x^3 + x + 1, ...).  With e = deg p_j, the generator matrix entry for
 * output digit r (weight 2^-(r+1)) and input digit k (weight 2^k) is the coefficient
 * of x^-(k+1) in the Laurent expansion of x^(e - u - 1) / p_j(x)^(q+1), r = q e + u,
 * 0 <= u < e.  Substituting t = 1/x, that coefficient is the coefficient of t^(k - r)
 * in the power series of prev(t)^-(q+1), prev(t) = t^e p_j(1/t) (constant term 1). */
static int or_gf2_degree(uint64_t p)
{
    int d = -1;
    while (p) { ++d; p >>= 1; }
    return d;
}

static uint64_t or_gf2_rem(uint64_t a, uint64_t b)
{
    int db = or_gf2_degree(b);
    for (int da = or_gf2_degree(a); da >= db; da = or_gf2_degree(a)) a ^= b << (da - db);
    return a;
}

static int or_gf2_irreducible(uint64_t p)
{
    int d = or_gf2_degree(p);
    if (d < 1) return 0;
    for (uint64_t q = 2; or_gf2_degree(q) <= d / 2; ++q)
        if (or_gf2_rem(p, q) == 0) return 0;
    return 1;
}

/* V[d*32 + k]: column k of the generator matrix of dimension d, output digit r at
 * bit 31 - r. */
int or_niederreiter_columns(int dims, uint32_t *V)
{
    uint64_t p = 1;
    for (int d = 0; d < dims; ++d) {
        do { ++p; } while (!or_gf2_irreducible(p));
        int e = or_gf2_degree(p);
        uint32_t rev = 0; /* prev(t): coefficient of t^i is that of x^(e-i) in p */
        for (int i = 0; i <= e; ++i)
            if ((p >> (e - i)) & 1) rev |= 1u << i;
        /* inv: series of 1/prev to 32 terms (prev(0) = 1), by long division */
        uint8_t inv[32], pw[32], nx[32];
        for (int n = 0; n < 32; ++n) {
            int c = n == 0 ? 1 : 0;
            for (int i = 1; i <= n && i <= e; ++i)
                if ((rev >> i) & 1) c ^= inv[n - i];
            inv[n] = (uint8_t)c;
        }
        for (int n = 0; n < 32; ++n) pw[n] = inv[n]; /* prev^-(q+1), q = 0 */
        int q_have = 0;
        for (int k = 0; k < 32; ++k) V[d * 32 + k] = 0;
        for (int r = 0; r < 32; ++r) {
            int q = r / e;
            while (q_have < q) { /* pw *= inv */
                for (int n = 0; n < 32; ++n) {
                    int c = 0;
                    for (int i = 0; i <= n; ++i) c ^= pw[i] & inv[n - i];
                    nx[n] = (uint8_t)c;
                }
                for (int n = 0; n < 32; ++n) pw[n] = nx[n];
                ++q_have;
            }
            for (int k = r; k < 32; ++k)
                if (pw[k - r]) V[d * 32 + k] |= 1u << (31 - r);
        }
    }
    return 0;
}

/* Niederreiter point i, dimension d: XOR of the generator columns over the set bits
 * of i (natural order). */
uint32_t or_niederreiter_u32(const uint32_t *V, int d, uint64_t i)
{
    uint32_t x = 0;
    for (int k = 0; k < 32; ++k)
        if ((i >> k) & 1) x ^= V[d * 32 + k];
    return x;
}

/* ---- Faure (1982): base b = the smallest prime >= the number of dimensions.
 * Dimension j applies the j-th power of the Pascal matrix mod b to the base-b digits
 * n_k of the index: output digit r = sum over k >= r of C(k, r) j^(k - r) n_k mod b
 * (j^0 = 1).  The value is the exact fraction sum_r y_r b^(K-1-r) / b^K (K digits of
 * the index), rounded once to double. */
uint32_t or_faure_base(int dims)
{
    uint32_t b = dims < 2 ? 2u : (uint32_t)dims;
    for (;; ++b) {
        int is_p = 1;
        for (uint32_t q = 2; q * q <= b; ++q)
            if (b % q == 0) { is_p = 0; break; }
        if (is_p) return b;
    }
}

double or_faure(uint64_t i, int d, uint32_t b)
{
    uint32_t n[64], y[64];
    int K = 0;
    while (i > 0) { n[K++] = (uint32_t)(i % b); i /= b; }
    /* binomials mod b by Pascal's rule */
    uint32_t C[64][64];
    for (int k = 0; k < K; ++k) {
        C[k][0] = 1 % b;
        C[k][k] = 1 % b;
        for (int r = 1; r < k; ++r) C[k][r] = (C[k - 1][r - 1] + C[k - 1][r]) % b;
    }
    uint64_t jmod = (uint64_t)d % b;
    for (int r = 0; r < K; ++r) {
        uint64_t acc = 0, pw = 1; /* pw = j^(k - r) mod b */
        for (int k = r; k < K; ++k) {
            acc = (acc + (uint64_t)C[k][r] * pw % b * n[k]) % b;
            pw = pw * jmod % b;
        }
        y[r] = (uint32_t)acc;
    }
    uint64_t num = 0, den = 1;
    for (int r = 0; r < K; ++r) {
        num = num * b + y[r];
        den *= b;
    }
    return (double)num / (double)den;
}

/* MurmurHash3 32-bit finaliser (Appleby), used only to derive per-dimension seeds. */
static uint32_t or_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

uint32_t or_owen_seed(uint64_t seed, int d)
{
    uint32_t hi = (uint32_t)(seed >> 32), lo = (uint32_t)seed;
    return or_fmix32(lo ^ or_fmix32(hi + 0x9e3779b9u * (uint32_t)(d + 1)));
}

/*
 * Nested uniform (Owen 1997) scramble of a base-2 digit string, in the hash form
 * (Laine-Karras style, as used by Burley 2020): reverse the bits so that the most
 * significant digit of the point becomes bit 0, apply a bijection in which output
 * bit j is input bit j XOR a function of bits 0..j-1 and the seed, reverse back.
 * Each step below has that triangular form: adding the seed (carries move upward)
 * and x ^= x * even (bit j of x*even depends on bits below j only).  The multipliers
 * are the first SHA-256 initial hash words with their low bit cleared.
 */
uint32_t or_owen_scramble(uint32_t x, uint32_t seed_d)
{
    uint32_t r = or_reverse32(x);
    r += seed_d;
    r ^= r * 0x6a09e666u;
    r ^= r * 0xbb67ae84u;
    r ^= r * 0x3c6ef372u;
    r ^= r * 0xa54ff53au;
    return or_reverse32(r);
}

/* Radical inverse of i in base b: the base-b digits of i mirrored about the point,
 * formed exactly as the integer fraction num / b^k and rounded once to double. */
double or_radical_inverse(uint64_t i, uint32_t b)
{
    uint64_t num = 0, den = 1;
    while (i > 0) {
        num = num * b + (i % b);
        den *= b;
        i /= b;
    }
    return (double)num / (double)den;
}

/* The n-th prime (n = 0 -> 2), by trial division. */
uint32_t or_prime(int n)
{
    int found = -1;
    for (uint32_t c = 2;; ++c) {
        int is_p = 1;
        for (uint32_t q = 2; q * q <= c; ++q)
            if (c % q == 0) { is_p = 0; break; }
        if (is_p && ++found == n) return c;
    }
}

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011): ten rounds of two 32x32->64
 * multiplications with the Weyl key schedule. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k[0];
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k[1];
        uint32_t n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    memcpy(out, c, sizeof c);
}

typedef struct {
    int kind;
    int dims;
    uint64_t seed;
    uint64_t total_n;   /* N of the Hammersley set */
    const uint32_t *V;  /* [dims][32] Sobol direction numbers, or Niederreiter generator columns */
} or_points;

/* 32-bit integer value of point i, dimension d (Sobol, scrambled Sobol, Philox). */
static uint32_t or_point_u32(const or_points *P, uint64_t i, int d)
{
    if (P->kind == OR_PHILOX) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), (uint32_t)(d / 4), 0};
        uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
        uint32_t out[4];
        or_philox4x32_10(ctr, key, out);
        return out[d % 4];
    }
    if (P->kind == OR_NIEDERREITER) return or_niederreiter_u32(P->V, d, i);
    uint32_t x = or_sobol_u32(P->V, d, i);
    if (P->kind == OR_SOBOL_OWEN) x = or_owen_scramble(x, or_owen_seed(P->seed, d));
    return x;
}

/* FP64 value of point i, dimension d, in [0, 1].  Integer generators: x * 2^-32
 * (exact).  Halton: exact radical inverse.  Hammersley: i/N in the first dimension
 * (the paper's variant), Halton of i with bases 2, 3, 5, ... in the others. */
double or_point_f64(const or_points *P, uint64_t i, int d)
{
    switch (P->kind) {
    case OR_HALTON:
        return or_radical_inverse(i, or_prime(d));
    case OR_HAMMERSLEY:
        if (d == 0) return (double)i / (double)P->total_n;
        return or_radical_inverse(i, or_prime(d - 1));
    case OR_FAURE:
        return or_faure(i, d, or_faure_base(P->dims));
    default:
        return (double)or_point_u32(P, i, d) * (1.0 / 4294967296.0);
    }
}

/* Double rounded toward zero to float: the single-precision value of a point. */
static float or_to_f32_rz(double v)
{
    float f = (float)v;
    if ((double)f > v) f = nextafterf(f, 0.0f);
    return f;
}

/* Row-major [count][dims] block of points starting at index first. */
int or_generate_points(int kind, int dims, uint64_t seed, uint64_t total_n, const uint32_t *V,
                       uint64_t first, uint64_t count, int format, void *out)
{
    or_points P = {kind, dims, seed, total_n, V};
    for (uint64_t j = 0; j < count; ++j) {
        uint64_t i = first + j;
        for (int d = 0; d < dims; ++d) {
            size_t o = (size_t)(j * (uint64_t)dims + (uint64_t)d);
            if (format == 0) {
                if (kind == OR_HALTON || kind == OR_HAMMERSLEY || kind == OR_FAURE) return -1;
                ((uint32_t *)out)[o] = or_point_u32(&P, i, d);
            } else if (format == 1) {
                ((float *)out)[o] = or_to_f32_rz(or_point_f64(&P, i, d));
            } else {
                ((double *)out)[o] = or_point_f64(&P, i, d);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Small vector helpers                                                             */
/* ------------------------------------------------------------------------------ */

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double a[3])
{
    double n = sqrt(dot3(a, a));
    a[0] /= n; a[1] /= n; a[2] /= n;
}
/* sin and cos of the angle 2 pi u, exact at quarter turns: the turn splits into a
 * quadrant (4u and its floor are exact in double) and an angle below pi/2, and
 * sin/cos of the whole follow from the quadrant's symmetry.  (A direct cos(2 pi u)
 * would give cos(pi/2) = 6e-17 instead of 0, tilting rays that start on a cell face
 * into a neighbouring row of cells.) */
static void sincos_2pi(double u, double *s, double *c)
{
    double x = 4.0 * u;
    double q = floor(x);
    double a = 0.5 * OR_PI * (x - q);
    double s0 = sin(a), c0 = cos(a);
    int quadrant = (int)(q - 4.0 * floor(q / 4.0));
    if (quadrant == 0) { *s = s0; *c = c0; }
    else if (quadrant == 1) { *s = c0; *c = -s0; }
    else if (quadrant == 2) { *s = -s0; *c = -c0; }
    else { *s = -c0; *c = s0; }
}

/* Unit vector with polar angle theta (cos given) and azimuth phi = 2 pi u (Sec. 3
 * convention). */
static void from_angles(double cos_t, double u, double n[3])
{
    double sin_t = sqrt(fmax(0.0, 1.0 - cos_t * cos_t));
    double sp, cp;
    sincos_2pi(u, &sp, &cp);
    n[0] = sin_t * cp;
    n[1] = sin_t * sp;
    n[2] = cos_t;
}
/* The local basis e_theta, e_phi of a unit vector n (spherical-coordinate unit vectors). */
static void sph_basis(const double n[3], double et[3], double ep[3])
{
    double s = sqrt(n[0] * n[0] + n[1] * n[1]);
    double cp = 1.0, sp = 0.0;
    if (s > 0) { cp = n[0] / s; sp = n[1] / s; }
    et[0] = n[2] * cp; et[1] = n[2] * sp; et[2] = -s;
    ep[0] = -sp; ep[1] = cp; ep[2] = 0.0;
}

/* ------------------------------------------------------------------------------ */
/* Medium: Cartesian grid of constant-density cells or an analytic sphere (Sec. 3.4) */
/* ------------------------------------------------------------------------------ */

enum { OR_MEDIUM_GRID = 0, OR_MEDIUM_SPHERE = 1 };

typedef struct {
    int kind;
    const float *k;    /* grid: extinction kappa*rho per unit length, [nz][ny][nx] */
    int n[3];          /* nx, ny, nz */
    double lo[3], hi[3];
    double kscale;     /* opacity multiplier applied to every cell */
    double sphere_r;   /* analytic: homogeneous sphere of radius r ... */
    double sphere_k;   /* ... and extinction k, centred at the origin */
} or_medium;

/* Cell index of coordinate x along one axis; a point exactly on a face belongs to the
 * cell the ray enters (the lower one when moving in the negative direction). */
static int or_start_cell(double x, double lo, double h, double dir)
{
    double f = (x - lo) / h;
    double fl = floor(f);
    int c = (int)fl;
    if (f == fl && dir < 0) c -= 1;
    return c;
}

/*
 * Walk the ray p + t d (t >= 0, d unit) through the grid, one cell at a time.
 * In each cell the optical depth is tau_cell = d_cell * kappa * rho (Sec. 3.4).
 * If target >= 0 and the running sum reaches target inside a cell, the walk stops
 * there: *t_hit = t_entry + (target - tau_before) / k_cell, return 1.
 * Otherwise it ends where the ray leaves the grid: *tau_sum is the total and
 * *t_last the far end of the last segment with nonzero density; return 0.
 * Ties between faces step x first, then y, then z (zero-length segments add 0).
 */
/* Cells visited by the walks of the packet being traced on this thread (a count of the
 * algorithm's work, reported in the packet log). */
static _Thread_local long long or_cells_visited;
static _Thread_local long long or_cells_marched; /* of those, visited by forced-step marches */
/* optional record of each cell's optical depth along one walk (or_ray_cells) */
static _Thread_local double *or_dtau_log;
static _Thread_local long long or_dtau_cap, or_dtau_n;

static int or_grid_walk(const or_medium *M, const double p[3], const double d[3], double target,
                        double *tau_sum, double *t_hit, double *t_last)
{
    double h[3];
    int c[3];
    for (int a = 0; a < 3; ++a) {
        h[a] = (M->hi[a] - M->lo[a]) / M->n[a];
        c[a] = or_start_cell(p[a], M->lo[a], h[a], d[a]);
    }
    *tau_sum = 0.0;
    *t_last = 0.0;
    for (int a = 0; a < 3; ++a)
        if (c[a] < 0 || c[a] >= M->n[a]) return 0;
    double t = 0.0, tau = 0.0;
    for (;;) {
        double tn[3];
        for (int a = 0; a < 3; ++a) {
            if (d[a] > 0) tn[a] = (M->lo[a] + (c[a] + 1) * h[a] - p[a]) / d[a];
            else if (d[a] < 0) tn[a] = (M->lo[a] + c[a] * h[a] - p[a]) / d[a];
            else tn[a] = INFINITY;
        }
        int a = 0;
        if (tn[1] < tn[a]) a = 1;
        if (tn[2] < tn[a]) a = 2;
        double te = tn[a] > t ? tn[a] : t;
        double kc = M->kscale * (double)M->k[((size_t)c[2] * M->n[1] + c[1]) * M->n[0] + c[0]];
        double dtau = (te - t) * kc;
        ++or_cells_visited;
        if (or_dtau_log && or_dtau_n < or_dtau_cap) or_dtau_log[or_dtau_n++] = dtau;
        if (target >= 0 && kc > 0 && tau + dtau >= target) {
            *t_hit = t + (target - tau) / kc;
            *tau_sum = target;
            return 1;
        }
        tau += dtau;
        if (kc > 0 && te > t) *t_last = te;
        t = te;
        c[a] += d[a] > 0 ? 1 : -1;
        if (c[a] < 0 || c[a] >= M->n[a]) break;
    }
    *tau_sum = tau;
    return 0;
}

/* Distance from p (inside) along unit d to the sphere |x| = r. */
static double or_sphere_exit(const double p[3], const double d[3], double r)
{
    double b = dot3(p, d);
    double c = dot3(p, p) - r * r;
    double disc = b * b - c;
    if (disc < 0) disc = 0;
    double s = -b + sqrt(disc);
    return s > 0 ? s : 0;
}

/* Optical depth from p along d to the edge of the medium (tau_1 and tau_obs). */
double or_tau_to_edge(const or_medium *M, const double p[3], const double d[3])
{
    if (M->kind == OR_MEDIUM_SPHERE) {
        if (dot3(p, p) > M->sphere_r * M->sphere_r) return 0.0;
        return M->kscale * M->sphere_k * or_sphere_exit(p, d, M->sphere_r);
    }
    double tau, th, tl;
    or_grid_walk(M, p, d, -1.0, &tau, &th, &tl);
    return tau;
}

/* Move from p along d through optical depth tau (Sec. 3.4).  Returns 1 with the
 * position if the depth is reached inside the medium, 0 if the ray leaves first
 * (then q is the far end of the last nonempty segment). */
int or_march(const or_medium *M, const double p[3], const double d[3], double tau, double q[3])
{
    double t;
    int hit;
    if (M->kind == OR_MEDIUM_SPHERE) {
        double s = or_sphere_exit(p, d, M->sphere_r);
        double k = M->kscale * M->sphere_k;
        if (k > 0 && tau < k * s) { t = tau / k; hit = 1; }
        else { t = s; hit = 0; }
    } else {
        double ts, th, tl;
        hit = or_grid_walk(M, p, d, tau, &ts, &th, &tl);
        t = hit ? th : tl;
    }
    for (int a = 0; a < 3; ++a) q[a] = p[a] + t * d[a];
    return hit;
}

/* ------------------------------------------------------------------------------ */
/* Scattering physics (Sec. 2.2, 3.5, 3.6)                                          */
/* ------------------------------------------------------------------------------ */

typedef struct {
    double albedo, g, p_l;
} or_dust;

/* Henyey-Greenstein x_HG and the White (1979) polarization elements (p_c = 0). */
static void or_mueller(const or_dust *D, double mu, double *P11, double *P12, double *P33)
{
    double g = D->g;
    double den = 1.0 + g * g - 2.0 * g * mu;
    *P11 = (1.0 - g * g) / (den * sqrt(den));
    *P12 = -D->p_l * *P11 * (1.0 - mu * mu) / (1.0 + mu * mu);
    *P33 = 2.0 * *P11 * mu / (1.0 + mu * mu);
}

/* Scattering angle cosine from v (Sec. 3.5); isotropic when |g| < 1e-6. */
double or_hg_cos(double g, double v)
{
    double c;
    if (fabs(g) < 1e-6) {
        c = 2.0 * v - 1.0;
    } else {
        double f = (1.0 - g * g) / (1.0 - g + 2.0 * g * v);
        c = (1.0 + g * g - f * f) / (2.0 * g);
    }
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return c;
}

/* Rotate the Stokes reference axis by psi (cos, sin given) about the propagation
 * direction: Q' = Q cos 2psi + U sin 2psi, U' = -Q sin 2psi + U cos 2psi. */
static void or_rotate_stokes(double cps, double sps, double *Q, double *U)
{
    double c2 = cps * cps - sps * sps, s2 = 2.0 * cps * sps;
    double q = *Q * c2 + *U * s2;
    double u = -*Q * s2 + *U * c2;
    *Q = q; *U = u;
}

/* ------------------------------------------------------------------------------ */
/* Observer and image (Sec. 3.6)                                                    */
/* ------------------------------------------------------------------------------ */

typedef struct {
    double theta, phi;   /* direction toward the observer */
    double half_width;   /* image covers [-hw, hw]^2 in the sky plane */
    int nx, ny;
    int splat;           /* 0 nearest pixel, 1 bilinear (tent) over 4 pixels */
} or_observer;

typedef struct {
    double k[3], ex[3], ey[3];
} or_view;

static void or_make_view(const or_observer *O, or_view *v)
{
    double st = sin(O->theta), ct = cos(O->theta), sp = sin(O->phi), cp = cos(O->phi);
    v->k[0] = st * cp; v->k[1] = st * sp; v->k[2] = ct;
    v->ex[0] = -sp; v->ex[1] = cp; v->ex[2] = 0.0;
    v->ey[0] = -ct * cp; v->ey[1] = -ct * sp; v->ey[2] = st;
}

/* Add (I, Q, U) at sky position (x, y) to image[3][ny][nx]. */
static void or_splat(const or_observer *O, double *img, double x, double y, const double S[3])
{
    double fx = (x + O->half_width) / (2.0 * O->half_width) * O->nx;
    double fy = (y + O->half_width) / (2.0 * O->half_width) * O->ny;
    size_t plane = (size_t)O->nx * O->ny;
    if (O->splat == 0) {
        double flx = floor(fx), fly = floor(fy);
        if (flx < 0 || flx >= O->nx || fly < 0 || fly >= O->ny) return;
        size_t p = (size_t)fly * O->nx + (size_t)flx;
        for (int s = 0; s < 3; ++s) img[s * plane + p] += S[s];
        return;
    }
    fx -= 0.5;
    fy -= 0.5;
    double x0 = floor(fx), y0 = floor(fy);
    double ax = fx - x0, ay = fy - y0;
    for (int dy = 0; dy < 2; ++dy) {
        for (int dx = 0; dx < 2; ++dx) {
            double ix = x0 + dx, iy = y0 + dy;
            if (ix < 0 || ix >= O->nx || iy < 0 || iy >= O->ny) continue;
            double w = (dx ? ax : 1.0 - ax) * (dy ? ay : 1.0 - ay);
            size_t p = (size_t)iy * O->nx + (size_t)ix;
            for (int s = 0; s < 3; ++s) img[s * plane + p] += w * S[s];
        }
    }
}

/* ------------------------------------------------------------------------------ */
/* Source (Sec. 3.2, 3.3)                                                           */
/* ------------------------------------------------------------------------------ */

typedef struct {
    int kind;          /* 0 point source at the origin, 1 sphere of radius r at the origin */
    double r;
    double limb_u;     /* linear limb darkening coefficient (0: isotropic surface) */
    int order;         /* sphere: 0 direct number order, 1 inverse number order */
} or_source;

/* Emission: position, direction, Stokes reference axis and weight from the first
 * coordinates of the point.  Returns the coordinate that sets the first depth.
 * Coordinates 0, 1 give the emission point (direct order) or the direction (inverse
 * order); c0, c1 the other pair and cw the depth (single scattering: the paper's order,
 * direct c0, c1, cw = 2, 3, 4 and inverse 3, 4, 2). */
static double or_emit(const or_source *S, const or_points *P, uint64_t i, double pos[3], double dir[3],
                      double eref[3], double *weight, int c0, int c1, int cw)
{
    double et[3], ep[3];
    *weight = 1.0;
    if (S->kind == 0) {
        /* Eq. point_source_propagation_direction: phi = 2 pi u, theta = arccos(2v - 1). */
        double u = or_point_f64(P, i, 0), v = or_point_f64(P, i, 1);
        from_angles(2.0 * v - 1.0, u, dir);
        pos[0] = pos[1] = pos[2] = 0.0;
        sph_basis(dir, eref, ep);
        return or_point_f64(P, i, 2);
    }
    double mu;
    if (S->order == 0) {
        /* Direct order: v1, v2 the emission point (Eq. sphere_source_emit_point);
         * v3, v4 the local direction, phi_l = 2 pi v3 and (reading of the garbled
         * theta_l = sqrt(v4)) cos theta_l = sqrt(v4), the cosine-weighted outward
         * hemisphere of an isotropically radiating surface; v5 the depth. */
        double ne[3];
        from_angles(2.0 * or_point_f64(P, i, 1) - 1.0, or_point_f64(P, i, 0), ne);
        for (int a = 0; a < 3; ++a) pos[a] = S->r * ne[a];
        double spl, cpl;
        sincos_2pi(or_point_f64(P, i, c0), &spl, &cpl);
        mu = sqrt(or_point_f64(P, i, c1));
        double sl = sqrt(fmax(0.0, 1.0 - mu * mu));
        sph_basis(ne, et, ep);
        for (int a = 0; a < 3; ++a) dir[a] = sl * cpl * et[a] + sl * spl * ep[a] + mu * ne[a];
        normalize3(dir);
        sph_basis(dir, eref, ep);
        if (S->limb_u != 0) *weight = (1.0 - S->limb_u + S->limb_u * mu) / (1.0 - S->limb_u / 3.0);
        return or_point_f64(P, i, cw);
    }
    /* Inverse order: v1, v2 the direction as for a point source, v3 the depth, v4, v5
     * the emission point relative to the direction.  Reading: the point is uniform on
     * the star's disk projected across the direction (radius R sqrt(v4), angle
     * 2 pi v5) lifted onto the hemisphere facing the direction, which gives the same
     * joint density of (point, direction) as the direct order. */
    from_angles(2.0 * or_point_f64(P, i, 1) - 1.0, or_point_f64(P, i, 0), dir);
    double w = or_point_f64(P, i, cw);
    double v4 = or_point_f64(P, i, c0), v5 = or_point_f64(P, i, c1);
    double rho = S->r * sqrt(v4), sps, cps;
    sincos_2pi(v5, &sps, &cps);
    double lift = sqrt(fmax(0.0, S->r * S->r - rho * rho));
    sph_basis(dir, et, ep);
    for (int a = 0; a < 3; ++a) pos[a] = rho * cps * et[a] + rho * sps * ep[a] + lift * dir[a];
    for (int a = 0; a < 3; ++a) eref[a] = et[a];
    mu = sqrt(fmax(0.0, 1.0 - v4));
    if (S->limb_u != 0) *weight = (1.0 - S->limb_u + S->limb_u * mu) / (1.0 - S->limb_u / 3.0);
    return w;
}

/* Emission with the single-scattering coordinate order of Sec. 3.3. */
static double or_emit_single(const or_source *S, const or_points *P, uint64_t i, double pos[3], double dir[3],
                             double eref[3], double *weight)
{
    int direct = S->order == 0;
    return or_emit(S, P, i, pos, dir, eref, weight, direct ? 2 : 3, direct ? 3 : 4, direct ? 4 : 2);
}

/* ------------------------------------------------------------------------------ */
/* Tracing                                                                          */
/* ------------------------------------------------------------------------------ */

typedef struct {
    or_medium medium;
    or_source source;
    or_dust dust;
    or_observer obs;
    or_points points;
    double tau_min;
    int max_orders;       /* trace_multiple */
    double rr_threshold;  /* Russian roulette below this weight (0: off) */
    double rr_survival;
    int force_all;        /* 1: every order forced; 0: only the first (paper's variant) */
    int per_order;        /* 1: one image per scattering order */
} or_problem;

/* Peel-off toward the observer (Sec. 3.6): the incoming packet (direction n, Stokes
 * S in the frame of eref) scatters at pos toward k; its weight is
 * W0 exp(-tau_obs) P(Theta_obs) / (4 pi).  Writes the image-frame Stokes of the new
 * packet to out and its sky coordinates; returns 0 if the star hides the path. */
static int or_peel(const or_problem *Pr, const or_view *V, const double pos[3], const double n[3],
                   const double eref[3], const double S[3], double out[3], double *x, double *y)
{
    out[0] = out[1] = out[2] = 0.0;
    *x = dot3(pos, V->ex);
    *y = dot3(pos, V->ey);
    if (Pr->source.kind == 1) {
        /* Star occultation: the segment toward the observer must miss the star. */
        double b = dot3(pos, V->k), c = dot3(pos, pos) - Pr->source.r * Pr->source.r;
        if (c <= 0 || (b < 0 && b * b - c > 0)) return 0;
    }
    double tau_obs = or_tau_to_edge(&Pr->medium, pos, V->k);
    double mu = dot3(n, V->k);
    double P11, P12, P33;
    or_mueller(&Pr->dust, mu, &P11, &P12, &P33);
    /* Normal of the scattering plane; for forward/backward scattering any normal. */
    double m[3], b2[3];
    cross3(n, V->k, m);
    cross3(n, eref, b2);
    if (sqrt(dot3(m, m)) < 1e-12) {
        for (int a = 0; a < 3; ++a) m[a] = b2[a];
    }
    normalize3(m);
    double pin[3], pout[3];
    cross3(m, n, pin);
    double I = S[0], Q = S[1], U = S[2];
    or_rotate_stokes(dot3(eref, pin), dot3(b2, pin), &Q, &U);
    double f = exp(-tau_obs) / (4.0 * OR_PI);
    double Io = f * (P11 * I + P12 * Q);
    double Qo = f * (P12 * I + P11 * Q);
    double Uo = f * (P33 * U);
    /* From the scattering frame (pout, m, k) to the image frame (ey, -ex, k). */
    cross3(m, V->k, pout);
    or_rotate_stokes(dot3(pout, V->ey), dot3(m, V->ey), &Qo, &Uo);
    out[0] = Io; out[1] = Qo; out[2] = Uo;
    return 1;
}

/* Forced scattering (Sec. 3.2): tau_1 to the edge; stop if below tau_min; weight
 * 1 - exp(-tau_1); depth -ln[1 - w (1 - exp(-tau_1))]; march to it. */
static int or_forced_step(const or_problem *Pr, double pos[3], const double dir[3], double w,
                          double *W1_out, double *tau1_out)
{
    double tau1 = or_tau_to_edge(&Pr->medium, pos, dir);
    *tau1_out = tau1;
    if (!(tau1 >= Pr->tau_min)) return 0;
    double W1 = -expm1(-tau1);
    double tau = -log1p(-w * W1);
    double q[3];
    const long long before = or_cells_visited;
    or_march(&Pr->medium, pos, dir, tau, q); /* a miss only by rounding: q = last nonempty end */
    or_cells_marched += or_cells_visited - before;
    for (int a = 0; a < 3; ++a) pos[a] = q[a];
    *W1_out = W1;
    return 1;
}

#define OR_LOG_COLS 11

typedef struct {
    const or_problem *Pr;
    uint64_t first, count;
    double *img;
    double *log;
    int multiple;
    const double *wx, *wlogj; /* optional learned warp: first-order coordinates, log |dx/du| */
    double *tlog;             /* optional [count][5]: coordinates used, sum and L2 norm of in-image I */
} or_job;

static void or_trace_single_range(const or_problem *Pr, uint64_t first, uint64_t count, double *img,
                                  double *log)
{
    or_view V;
    or_make_view(&Pr->obs, &V);
    for (uint64_t j = 0; j < count; ++j) {
        uint64_t i = first + j;
        double pos[3], dir[3], eref[3], wgt, W1 = 0, tau1 = 0, S[3], out[3], x = 0, y = 0;
        or_cells_visited = 0;
        or_cells_marched = 0;
        double w = or_emit_single(&Pr->source, &Pr->points, i, pos, dir, eref, &wgt);
        int status = 0;
        out[0] = out[1] = out[2] = 0;
        if (!or_forced_step(Pr, pos, dir, w, &W1, &tau1)) {
            status = 1;
        } else {
            S[0] = wgt * W1 * Pr->dust.albedo;
            S[1] = S[2] = 0.0;
            if (!or_peel(Pr, &V, pos, dir, eref, S, out, &x, &y)) status = 2;
            else or_splat(&Pr->obs, img, x, y, out);
        }
        if (log) {
            double *r = log + j * OR_LOG_COLS;
            r[0] = pos[0]; r[1] = pos[1]; r[2] = pos[2];
            r[3] = out[0]; r[4] = out[1]; r[5] = out[2];
            r[6] = x; r[7] = y; r[8] = status;
            r[9] = (double)or_cells_visited;
            r[10] = (double)or_cells_marched;
        }
    }
}

/* New direction after a Henyey-Greenstein scattering (Sec. 3.5): Theta from v,
 * azimuth i1 = 2 pi u measured from the packet's Stokes reference axis a about n.
 * The Stokes vector is rotated into the scattering plane (angle i1), multiplied by
 * M(Theta)/P11 (the direction was sampled from P11 alone) and referred to the new
 * in-plane axis. */
static void or_scatter(const or_dust *D, double u, double v, double n[3], double a[3], double S[3])
{
    double ct = or_hg_cos(D->g, v);
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double b[3];
    cross3(n, a, b);
    double ci, si;
    sincos_2pi(u, &si, &ci); /* i1 = 2 pi u */
    double nn[3], m[3];
    for (int k = 0; k < 3; ++k) {
        nn[k] = ct * n[k] + st * (ci * a[k] + si * b[k]);
        m[k] = ci * b[k] - si * a[k];
    }
    normalize3(nn);
    double Q = S[1], U = S[2];
    or_rotate_stokes(ci, si, &Q, &U);
    double P11, P12, P33;
    or_mueller(D, ct, &P11, &P12, &P33);
    double I = S[0];
    S[0] = I + (P12 / P11) * Q;
    S[1] = (P12 / P11) * I + Q;
    S[2] = (P33 / P11) * U;
    double anew[3];
    cross3(m, nn, anew);
    normalize3(anew);
    for (int k = 0; k < 3; ++k) { n[k] = nn[k]; a[k] = anew[k]; }
}

/* Multiple scattering, point source.  Coordinates of order k (1-based) are
 * 4(k-1) + {0, 1, 2, 3}: azimuth (or emission phi), cos Theta (or emission
 * theta), depth, roulette. */
static void or_trace_multiple_range(const or_problem *Pr, uint64_t first, uint64_t count, double *img,
                                    const double *wx, const double *wlogj, double *tlog, double *cells)
{
    or_view V;
    or_make_view(&Pr->obs, &V);
    size_t img_size = (size_t)3 * Pr->obs.nx * Pr->obs.ny;
    for (uint64_t j = 0; j < count; ++j) {
        uint64_t i = first + j;
        double pos[3], n[3], a[3], wgt, w, total = 0.0, total2 = 0.0;
        or_cells_visited = 0;
        or_cells_marched = 0;
        double x0 = or_point_f64(&Pr->points, i, 0), x1 = or_point_f64(&Pr->points, i, 1);
        if (wx) {
            /* Learned proposal: the first-order coordinates are x = T(u), and the
             * weight carries the Jacobian |dx/du| = 1 / q(x), so the estimate of the
             * integral over x stays unbiased. */
            double ep[3];
            x0 = wx[3 * j];
            x1 = wx[3 * j + 1];
            from_angles(2.0 * x1 - 1.0, x0, n);
            pos[0] = pos[1] = pos[2] = 0.0;
            sph_basis(n, a, ep);
            w = wx[3 * j + 2];
            wgt = exp(wlogj[j]);
        } else {
            /* a finite star's two other emission coordinates follow all orders' ones */
            int e = 4 * Pr->max_orders;
            w = or_emit(&Pr->source, &Pr->points, i, pos, n, a, &wgt, e, e + 1, 2);
        }
        const double w_first = w;
        double S[3] = {wgt, 0.0, 0.0};
        for (int k = 1; k <= Pr->max_orders; ++k) {
            int base = 4 * (k - 1);
            if (k > 1) {
                or_scatter(&Pr->dust, or_point_f64(&Pr->points, i, base + 0),
                           or_point_f64(&Pr->points, i, base + 1), n, a, S);
                w = or_point_f64(&Pr->points, i, base + 2);
            }
            if (k == 1 || Pr->force_all) {
                double W1, tau1;
                if (!or_forced_step(Pr, pos, n, w, &W1, &tau1)) break;
                for (int s = 0; s < 3; ++s) S[s] *= W1;
            } else {
                double q[3];
                if (!or_march(&Pr->medium, pos, n, -log(w), q)) break;
                for (int s = 0; s < 3; ++s) pos[s] = q[s];
            }
            for (int s = 0; s < 3; ++s) S[s] *= Pr->dust.albedo;
            double out[3], x, y;
            if (or_peel(Pr, &V, pos, n, a, S, out, &x, &y)) {
                or_splat(&Pr->obs, img + (Pr->per_order ? (size_t)(k - 1) * img_size : 0), x, y, out);
                double hw = Pr->obs.half_width;
                if (x >= -hw && x < hw && y >= -hw && y < hw) {
                    total += out[0];
                    total2 += out[0] * out[0];
                }
            }
            if (k == Pr->max_orders) break;
            if (S[0] < Pr->rr_threshold) {
                double r = or_point_f64(&Pr->points, i, base + 3);
                if (r < Pr->rr_survival) {
                    for (int s = 0; s < 3; ++s) S[s] /= Pr->rr_survival;
                } else {
                    break;
                }
            }
        }
        if (tlog) {
            tlog[5 * j] = x0;
            tlog[5 * j + 1] = x1;
            tlog[5 * j + 2] = w_first;
            tlog[5 * j + 3] = total;
            tlog[5 * j + 4] = sqrt(total2);
        }
        if (cells) {
            cells[2 * j] = (double)or_cells_visited;
            cells[2 * j + 1] = (double)or_cells_marched;
        }
    }
}

static void *or_worker(void *arg)
{
    or_job *J = (or_job *)arg;
    if (J->multiple) or_trace_multiple_range(J->Pr, J->first, J->count, J->img, J->wx, J->wlogj, J->tlog, NULL);
    else or_trace_single_range(J->Pr, J->first, J->count, J->img, J->log);
    return NULL;
}

/* Trace packets first .. first+count-1 on nthreads threads; adds the raw sums
 * (not divided by N) to image; log (optional, single only) gets OR_LOG_COLS doubles per
 * packet: scattering position, peel-off I, Q, U, sky x, y, status (0 ok, 1 tau_1 <
 * tau_min, 2 occulted), grid cells visited by the packet's walks, and of those the cells
 * visited by the march to the scattering point (a second pass over cells of the first walk). */
static int or_trace(const or_problem *Pr, uint64_t first, uint64_t count, double *image, double *log,
                    int nthreads, int multiple, const double *wx, const double *wlogj, double *tlog)
{
    size_t img_size = (size_t)3 * Pr->obs.nx * Pr->obs.ny * (multiple && Pr->per_order ? Pr->max_orders : 1);
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > count) nthreads = count > 0 ? (int)count : 1;
    or_job *jobs = calloc((size_t)nthreads, sizeof *jobs);
    pthread_t *th = calloc((size_t)nthreads, sizeof *th);
    if (!jobs || !th) return -1;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t a = count * (uint64_t)t / (uint64_t)nthreads, b = count * (uint64_t)(t + 1) / (uint64_t)nthreads;
        jobs[t].Pr = Pr;
        jobs[t].first = first + a;
        jobs[t].count = b - a;
        jobs[t].img = calloc(img_size, sizeof(double));
        jobs[t].log = log ? log + a * OR_LOG_COLS : NULL;
        jobs[t].multiple = multiple;
        jobs[t].wx = wx ? wx + 3 * a : NULL;
        jobs[t].wlogj = wlogj ? wlogj + a : NULL;
        jobs[t].tlog = tlog ? tlog + 5 * a : NULL;
        if (!jobs[t].img) return -1;
        pthread_create(&th[t], NULL, or_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t) {
        for (size_t p = 0; p < img_size; ++p) image[p] += jobs[t].img[p];
        free(jobs[t].img);
    }
    free(jobs);
    free(th);
    return 0;
}

int or_trace_single(const or_problem *Pr, uint64_t first, uint64_t count, double *image, double *log,
                    int nthreads)
{
    return or_trace(Pr, first, count, image, log, nthreads, 0, NULL, NULL, NULL);
}

int or_trace_multiple(const or_problem *Pr, uint64_t first, uint64_t count, double *image, int nthreads)
{
    return or_trace(Pr, first, count, image, NULL, nthreads, 1, NULL, NULL, NULL);
}

/* Multiple scattering with the first-order coordinates of packet j given (x[j][3],
 * weight exp(logj[j])); either may be NULL together (plain points).  train_log
 * (optional) gets per packet the first-order coordinates used, the sum of the
 * intensities its peel-offs put into the image (all orders) and the square root of
 * their sum of squares. */
int or_trace_multiple_warped(const or_problem *Pr, uint64_t first, uint64_t count, const double *x,
                             const double *logj, double *image, double *train_log, int nthreads)
{
    if (Pr->source.kind != 0 && x) return -3; /* the warp replaces point-source coordinates only */
    if ((x == NULL) != (logj == NULL)) return -2;
    return or_trace(Pr, first, count, image, NULL, nthreads, 1, x, logj, train_log);
}

/* Direct (unscattered) light of the source, integrated separately from the source
 * toward the observer (Sec. 3.4), Stokes I only, added to image[0] times `weight`
 * (raw images are sums over packets, so weight = N makes it appear once after the
 * 1/N scaling).  Values are in units of the source luminosity per steradian.
 *   Point source: e^-tau(0 -> observer) / (4 pi), binned at the sky origin like a
 *   peel-off contribution.
 *   Sphere source of radius R and linear limb darkening u: surface brightness
 *   (1 - u + u mu) / (1 - u/3) / (4 pi) / (pi R^2) per unit sky area at projected
 *   radius rho, mu = sqrt(1 - rho^2 / R^2) (it integrates to 1 / (4 pi) over the disk),
 *   attenuated by e^-tau from the visible surface point rho-offset on the facing
 *   hemisphere toward the observer; each pixel is integrated by an S x S midpoint rule
 *   over its area. */
int or_direct_light(const or_problem *Pr, int S, double weight, double *img)
{
    const or_observer *O = &Pr->obs;
    or_view V;
    or_make_view(O, &V);
    if (Pr->source.kind == 0) {
        double origin[3] = {0.0, 0.0, 0.0};
        double f = exp(-or_tau_to_edge(&Pr->medium, origin, V.k)) / (4.0 * OR_PI) * weight;
        double out[3] = {f, 0.0, 0.0};
        or_splat(O, img, 0.0, 0.0, out);
        return 0;
    }
    if (S < 1) return -1;
    double R = Pr->source.r, u = Pr->source.limb_u;
    double px = 2.0 * O->half_width / O->nx, py = 2.0 * O->half_width / O->ny;
    double dA = px * py / ((double)S * S);
    for (int iy = 0; iy < O->ny; ++iy) {
        for (int ix = 0; ix < O->nx; ++ix) {
            double sum = 0.0;
            for (int b = 0; b < S; ++b) {
                for (int a = 0; a < S; ++a) {
                    double x = -O->half_width + (ix + (a + 0.5) / S) * px;
                    double y = -O->half_width + (iy + (b + 0.5) / S) * py;
                    double rho2 = x * x + y * y;
                    if (!(rho2 < R * R)) continue;
                    double mu = sqrt(1.0 - rho2 / (R * R));
                    double p[3];
                    for (int c = 0; c < 3; ++c) p[c] = x * V.ex[c] + y * V.ey[c] + R * mu * V.k[c];
                    double B = (1.0 - u + u * mu) / (1.0 - u / 3.0) / (4.0 * OR_PI) / (OR_PI * R * R);
                    sum += B * exp(-or_tau_to_edge(&Pr->medium, p, V.k)) * dA;
                }
            }
            img[(size_t)iy * O->nx + ix] += sum * weight;
        }
    }
    return 0;
}

/* Grid cells visited by all walks of each packet of the multiple-scattering tracer
 * (one thread), and of those the cells visited by the marches of forced steps:
 * cells[2 j], cells[2 j + 1]; the image goes to `image`.  The per-unit work figure of the
 * multiple-scattering kernel's roofline. */
int or_trace_multiple_cells(const or_problem *Pr, uint64_t first, uint64_t count, double *image, double *cells)
{
    or_trace_multiple_range(Pr, first, count, image, NULL, NULL, NULL, cells);
    return 0;
}

/* Exposed for pins: tau along a ray and the position after a march. */
double or_tau_ray(const or_problem *Pr, const double p[3], const double d[3])
{
    return or_tau_to_edge(&Pr->medium, p, d);
}
/* Cells the walk from p along d to the edge of a grid visits (out[0]), and how many of them
 * come before the optical depth still ahead falls to eps or below (out[1]): the cells a walk
 * that may leave out eps of its depth must visit.  Returns -1 for a sphere medium. */
int or_ray_cells(const or_problem *Pr, const double p[3], const double d[3], double eps, double out[2])
{
    const or_medium *M = &Pr->medium;
    if (M->kind != OR_MEDIUM_GRID) return -1;
    or_dtau_cap = (long long)M->n[0] + M->n[1] + M->n[2] + 3;
    or_dtau_log = malloc((size_t)or_dtau_cap * sizeof(double));
    if (!or_dtau_log) return -1;
    or_dtau_n = 0;
    or_tau_to_edge(M, p, d);
    long long n = or_dtau_n, needed = n;
    double rest = 0.0;
    for (long long j = n - 1; j >= 0; --j) {
        rest += or_dtau_log[j];
        if (!(rest <= eps)) break;
        needed = j;
    }
    free(or_dtau_log);
    or_dtau_log = NULL;
    out[0] = (double)n;
    out[1] = (double)needed;
    return 0;
}
int or_march_ray(const or_problem *Pr, const double p[3], const double d[3], double tau, double q[3])
{
    return or_march(&Pr->medium, p, d, tau, q);
}
/* Exposed for pins: one scattering of a packet (direction n, axis a, Stokes S). */
void or_scatter_packet(const or_problem *Pr, double u, double v, double n[3], double a[3], double S[3])
{
    or_scatter(&Pr->dust, u, v, n, a, S);
}
/* Exposed for pins: the peel-off of one packet (returns 0 if occulted). */
int or_peel_packet(const or_problem *Pr, const double pos[3], const double n[3], const double a[3],
                   const double S[3], double out[5])
{
    or_view V;
    or_make_view(&Pr->obs, &V);
    double x, y;
    int ok = or_peel(Pr, &V, pos, n, a, S, out, &x, &y);
    out[3] = x;
    out[4] = y;
    return ok;
}
/* Exposed for pins: emission of packet i. */
double or_emit_packet(const or_problem *Pr, uint64_t i, double pos[3], double dir[3], double eref[3],
                      double *weight)
{
    return or_emit_single(&Pr->source, &Pr->points, i, pos, dir, eref, weight);
}

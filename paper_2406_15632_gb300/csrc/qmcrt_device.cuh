// qmcrt_device.cuh -- device building blocks of the tracer: point generators (Sec. 3.1),
// sources (Sec. 3.2, 3.3), the cell walk (Sec. 3.4), Henyey-Greenstein / White
// scattering (Sec. 2.2, 3.5), peel-off (Sec. 3.6) and warp-aggregated image deposits.
//
// Everything is templated on the arithmetic type T: float is the production path
// (compensated optical-depth sums, FP64 or fixed-point images), double the
// reference-grade path.  One thread traces one packet.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "qmcrt.h"
#include "qmcrt_internal.h"
#include "qmcrt_tables.h"

namespace qmcrt {

// Sobol direction numbers V[d][k] for bit k of the Gray-code index, and Halton bases.
static __constant__ uint32_t c_sobol_v[QMCRT_GEN_DIMS][32] = QMCRT_GEN_SOBOL_V_INIT;
static __constant__ uint32_t c_primes[QMCRT_GEN_DIMS] = QMCRT_GEN_PRIMES_INIT;
static __device__ const uint32_t d_nied_v[QMCRT_GEN_DIMS][32] = QMCRT_GEN_NIED_V_INIT;
// The same direction numbers of the leading dimensions grouped by bytes of the Gray code:
// entry [d][b][v] is the XOR of V[d][8 b + k] over the set bits k of v.
static __device__ const uint32_t d_sobol_byte[QMCRT_GEN_SOBOL_BYTE_DIMS][4][256] = QMCRT_GEN_SOBOL_BYTE_INIT;

constexpr unsigned FULL_MASK = 0xffffffffu;

// ------------------------------------------------------------------------------------
// Math in T
// ------------------------------------------------------------------------------------
template <class T>
struct Mth;

template <>
struct Mth<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
    static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    static __device__ __forceinline__ void sincospi_(float x, float *s, float *c) { sincospif(x, s, c); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
    static __device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
    static __device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
    // value of a 32-bit point coordinate: x * 2^-32 rounded toward zero
    static __device__ __forceinline__ float from_u32(uint32_t x) { return __uint2float_rz(x) * 0x1p-32f; }
    static __device__ __forceinline__ float from_f64(double v) { return __double2float_rz(v); }
    // lo + c h with the product and the sum rounded separately (never fused): the face
    // coordinates of the oracle, bit for bit in double
    static __device__ __forceinline__ float face(float lo, int c, float h) { return __fadd_rn(lo, __fmul_rn((float)c, h)); }
    // explicitly rounded operations: the compiler neither fuses nor splits them, so every
    // kernel that inlines a walk computes its sums with the same roundings
    static __device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ long long to_fixed(float v, double scale)
    {
        return __float2ll_rn(v * (float)scale);  // exact power-of-two scaling, one rounding
    }
};

template <>
struct Mth<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double expm1_(double x) { return expm1(x); }
    static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    static __device__ __forceinline__ void sincospi_(double x, double *s, double *c) { sincospi(x, s, c); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
    static __device__ __forceinline__ double min_(double a, double b) { return fmin(a, b); }
    static __device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    static __device__ __forceinline__ double from_u32(uint32_t x) { return (double)x * 0x1p-32; }
    static __device__ __forceinline__ double from_f64(double v) { return v; }
    static __device__ __forceinline__ double face(double lo, int c, double h) { return __dadd_rn(lo, __dmul_rn((double)c, h)); }
    static __device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ long long to_fixed(double v, double scale) { return __double2ll_rn(v * scale); }
};

template <class T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

template <class T>
__device__ __forceinline__ void cross3(const T a[3], const T b[3], T c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

template <class T>
__device__ __forceinline__ void normalize3(T a[3])
{
    T inv = T(1) / Mth<T>::sqrt_(dot3(a, a));
    a[0] *= inv;
    a[1] *= inv;
    a[2] *= inv;
}

// ------------------------------------------------------------------------------------
// Point generators (Sec. 3.1)
// ------------------------------------------------------------------------------------

// Sobol: XOR of the direction numbers over the set bits of gray(i).  The leading
// dimensions take it a byte at a time from the grouped table (four independent loads);
// the rest loop over the bits, uniform across the warp so every constant load is a
// broadcast.
__device__ __forceinline__ uint32_t sobol_u32(uint32_t i, int d)
{
    const uint32_t g = i ^ (i >> 1);
    if (d < QMCRT_GEN_SOBOL_BYTE_DIMS)
        return __ldg(&d_sobol_byte[d][0][g & 255u]) ^ __ldg(&d_sobol_byte[d][1][(g >> 8) & 255u]) ^
               __ldg(&d_sobol_byte[d][2][(g >> 16) & 255u]) ^ __ldg(&d_sobol_byte[d][3][g >> 24]);
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) x ^= (g & (1u << k)) ? c_sobol_v[d][k] : 0u;
    return x;
}

// Niederreiter point i, dimension d (natural order): XOR of the generator columns over
// the set bits of i.
__device__ __forceinline__ uint32_t niederreiter_u32(uint32_t i, int d)
{
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) x ^= (i & (1u << k)) ? __ldg(&d_nied_v[d][k]) : 0u;
    return x;
}

// Faure point (Faure 1982): output digit r = sum over k >= r of C(k, r) j^(k-r) n_k mod b
// (n_k the base-b digits of i, j the dimension), i.e. the coefficients of N(X + j) for
// N(X) = sum n_k X^k, computed by the Taylor shift (repeated synthetic division) mod b;
// the value is the exact fraction y / b^K rounded once.
static __device__ __noinline__ double faure_f64(uint32_t i, int d, uint32_t b)  // off the hot path (own frame)
{
    uint32_t a[32];
    int K = 0;
    while (i) {
        const uint32_t q = i / b;
        a[K++] = i - q * b;
        i = q;
    }
    const uint32_t j = (uint32_t)d % b;
    for (int s = 0; s + 1 < K; ++s)
        for (int k = K - 2; k >= s; --k) a[k] = (a[k] + j * a[k + 1]) % b;
    uint64_t num = 0, den = 1;
    for (int r = 0; r < K; ++r) {
        num = num * b + a[r];
        den *= b;
    }
    return (double)num / (double)den;
}

// MurmurHash3 finaliser, for per-dimension scramble seeds.
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint32_t owen_seed(uint64_t seed, int d)
{
    return fmix32((uint32_t)seed ^ fmix32((uint32_t)(seed >> 32) + 0x9e3779b9u * (uint32_t)(d + 1)));
}

// Hash-based nested uniform scramble (Owen 1997, in the Laine-Karras / Burley 2020
// form): in bit-reversed order, output bit j = input bit j XOR f(bits below j, seed).
__device__ __forceinline__ uint32_t owen_scramble(uint32_t x, uint32_t s)
{
    uint32_t r = __brev(x);
    r += s;
    r ^= r * 0x6a09e666u;
    r ^= r * 0xbb67ae84u;
    r ^= r * 0x3c6ef372u;
    r ^= r * 0xa54ff53au;
    return __brev(r);
}

// Philox4x32-10 (Salmon et al. 2011).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t philox_u32(uint64_t seed, uint64_t i, int d)
{
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)(d >> 2), 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const int s = d & 3;
    return s == 0 ? w.x : s == 1 ? w.y : s == 2 ? w.z : w.w;
}

// Radical inverse in base b as the exact fraction num / b^k, one correctly rounded
// division (b^k < 2^53 for every index < 2^32 and base in the table).
__device__ __forceinline__ double radical_inverse(uint32_t i, uint32_t b)
{
    if (b == 2) return (double)__brev(i) * 0x1p-32;
    uint64_t num = 0, den = 1;
    while (i) {
        const uint32_t q = i / b;
        num = num * b + (i - q * b);
        den *= b;
        i = q;
    }
    return (double)num / (double)den;
}

__device__ __forceinline__ bool is_integer_kind(int kind)
{
    return kind == QMCRT_SOBOL || kind == QMCRT_SOBOL_OWEN || kind == QMCRT_PHILOX || kind == QMCRT_NIEDERREITER;
}

__device__ __forceinline__ uint32_t point_u32(const PointsP &P, uint64_t i, int d)
{
    if (P.kind == QMCRT_PHILOX) return philox_u32(P.seed, i, d);
    if (P.kind == QMCRT_NIEDERREITER) return niederreiter_u32((uint32_t)i, d);
    uint32_t x = sobol_u32((uint32_t)i, d);
    if (P.kind == QMCRT_SOBOL_OWEN) x = owen_scramble(x, owen_seed(P.seed, d));
    return x;
}

__device__ __forceinline__ double point_f64(const PointsP &P, uint64_t i, int d)
{
    if (P.kind == QMCRT_HALTON) return radical_inverse((uint32_t)i, c_primes[d]);
    if (P.kind == QMCRT_HAMMERSLEY) {
        if (d == 0) return (double)i / (double)P.total_n;
        return radical_inverse((uint32_t)i, c_primes[d - 1]);
    }
    if (P.kind == QMCRT_FAURE) return faure_f64((uint32_t)i, d, P.faure_b);
    return (double)point_u32(P, i, d) * 0x1p-32;
}

template <class T>
__device__ __forceinline__ T point(const PointsP &P, uint64_t i, int d)
{
    if (is_integer_kind(P.kind)) return Mth<T>::from_u32(point_u32(P, i, d));
    return Mth<T>::from_f64(point_f64(P, i, d));
}

// Inverse of the Gray code g = i ^ (i >> 1).
__device__ __forceinline__ uint32_t gray_inverse(uint32_t g)
{
    g ^= g >> 1;
    g ^= g >> 2;
    g ^= g >> 4;
    g ^= g >> 8;
    g ^= g >> 16;
    return g;
}

__device__ __forceinline__ uint32_t lead_bits(uint32_t x, int n) { return n ? x >> (32 - n) : 0u; }

// The part of the GF(2) combination that depends only on the block starting at base (a
// multiple of 2^m): the columns ry of the leading bits y of the block start's coordinates.
__device__ __forceinline__ uint32_t block_columns(const OrderP &O, uint64_t base)
{
    const bool nied = O.net == 2;
    const bool extra = O.nb[3] + O.nb[4] > 0;  // uniform: the order also groups xdim[0], xdim[1]
    // The block start is a multiple of 2^m, so its digit vector (Gray code for Sobol)
    // has set bits only from m - 1 up: XOR the columns of those bits alone.
    uint32_t b0 = 0, b1 = 0, b2 = 0, b3 = 0, b4 = 0;
    const uint32_t b32 = (uint32_t)base;
    for (uint32_t gb = nied ? b32 : b32 ^ (b32 >> 1); gb; gb &= gb - 1u) {
        const int k = __ffs(gb) - 1;
        if (nied) {
            b0 ^= __ldg(&d_nied_v[0][k]);
            b1 ^= __ldg(&d_nied_v[1][k]);
            b2 ^= __ldg(&d_nied_v[2][k]);
            if (extra) {
                b3 ^= __ldg(&d_nied_v[O.xdim[0]][k]);
                b4 ^= __ldg(&d_nied_v[O.xdim[1]][k]);
            }
        } else {
            b0 ^= c_sobol_v[0][k];
            b1 ^= c_sobol_v[1][k];
            b2 ^= c_sobol_v[2][k];
            if (extra) {
                b3 ^= c_sobol_v[O.xdim[0]][k];
                b4 ^= c_sobol_v[O.xdim[1]][k];
            }
        }
    }
    // y: the leading bits of coordinates 2, 1, 0, xdim[0], xdim[1], least significant first
    const int s1 = O.nb[2], s0 = s1 + O.nb[1], s3 = s0 + O.nb[0], s4 = s3 + O.nb[3];
    const uint32_t y = lead_bits(b2, O.nb[2]) | (lead_bits(b1, O.nb[1]) << s1) | (lead_bits(b0, O.nb[0]) << s0) |
                       (lead_bits(b3, O.nb[3]) << s3) | (lead_bits(b4, O.nb[4]) << s4);
    uint32_t g = 0;
#pragma unroll
    for (int j = 0; j < NET_MAX_M; ++j) g ^= ((y >> j) & 1u) ? O.ry[j] : 0u;  // y < 2^bits
    return g;
}

// Point index traced by thread tid: with the net order, thread t of a block traces the
// point in elementary box t (Morton order); the block's own term comes from the host
// (O.g0) for the block O.g0_block and is computed here for any other.  False if the
// index lies outside the range.
__device__ __forceinline__ bool packet_index(const OrderP &O, uint64_t first, uint64_t count, uint64_t tid,
                                             uint64_t &i)
{
    if (!O.net) {
        i = first + tid;
        return tid < count;
    }
    const uint64_t base = (O.block0 + (tid >> O.m)) << O.m;
    const uint32_t tl = (uint32_t)(tid & ((1ull << O.m) - 1));
    const uint32_t box = tl >> O.tt;                 // < 2^bits
    const uint32_t kt = tl & ((1u << O.tt) - 1u);   // < 2^tt
    // Unrolled over the largest sizes: the bits of box, kt and y above bits (tt) are zero,
    // so the columns past them (zero-filled) never enter.
    uint32_t g = 0;
#pragma unroll
    for (int j = 0; j < NET_MAX_M; ++j) g ^= ((box >> j) & 1u) ? O.rm[j] : 0u;
#pragma unroll
    for (int j = 0; j < NET_MAX_TT; ++j) g ^= ((kt >> j) & 1u) ? O.k[j] : 0u;
    const bool nied = O.net == 2;
    g ^= base >> O.m == O.g0_block ? O.g0 : block_columns(O, base);
    i = base + (nied ? g : gray_inverse(g));
    return i >= first && i < first + count;
}

// ------------------------------------------------------------------------------------
// Optical depth along a ray (Sec. 3.4)
// ------------------------------------------------------------------------------------

// Cell of coordinate x; on a face, the cell the ray enters.  (x - lo) drops the low
// digits of a coordinate much smaller than lo (in float a point 2e-8 below the face
// through the origin becomes a point on it), so the estimate (x - lo) / h, taken with
// the reciprocal, is settled against the face coordinates themselves: the result does
// not depend on the rounding of the estimate.  The faces are lo + c h rounded step by
// step (Mth::face), never fused into one rounding: where h is inexact (200 cells over
// [-1, 1]) a fused lo + 100 h lies 2e-17 above the face through the origin, and a
// source there that sends a ray along that face would walk the neighbouring slab.
template <class T>
__device__ __forceinline__ int start_cell(T x, T lo, T h, T inv_h, T d)
{
    int c = (int)Mth<T>::floor_((x - lo) * inv_h);
    if (x < Mth<T>::face(lo, c, h)) --c;
    else if (x >= Mth<T>::face(lo, c + 1, h)) ++c;
    if (d < T(0) && x == Mth<T>::face(lo, c, h)) --c;
    return c;
}

template <class T>
struct AxisWalk {
    T s, dt;   // distance along the ray to this axis's next face; length of one cell crossing
    int step, left;
};

// r = 1 / d, computed once per direction by the caller (the forced step's two walks
// share it; a launch's observer direction has it precomputed on the host).
template <class T>
__device__ __forceinline__ AxisWalk<T> axis_setup(T p, T d, T r, int c, T lo, T h, int n, int stride)
{
    AxisWalk<T> a;
    a.s = Mth<T>::inf();
    a.dt = T(0);
    a.step = 0;
    a.left = 0;
    if (d > T(0)) {
        a.s = (Mth<T>::face(lo, c + 1, h) - p) * r;
        a.dt = h * r;
        a.step = stride;
        a.left = n - 1 - c;
    } else if (d < T(0)) {
        a.s = (Mth<T>::face(lo, c, h) - p) * r;
        a.dt = -h * r;
        a.step = -stride;
        a.left = c;
    }
    if (!(d != T(0) && a.s < Mth<T>::inf() && a.dt < Mth<T>::inf())) {
        // an axis the ray never crosses (zero component, or a face distance beyond
        // float range): never the nearest face
        a.s = Mth<T>::inf();
        a.dt = T(0);
        a.step = 0;
        a.left = 0;
    }
    return a;
}

// A walk needs a finite start and direction and at least one axis it crosses; with
// those every step reaches the nearest face of a crossed axis and moves one cell, so
// both walks below end after at most nx + ny + nz steps (plus one batch).
template <class T>
__device__ __forceinline__ bool walkable(const T p[3], const T d[3])
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) ok &= (p[a] - p[a] == T(0)) && (d[a] - d[a] == T(0));  // finite
    return ok && (d[0] != T(0) || d[1] != T(0) || d[2] != T(0));
}

// Walk through the grid cells from p along unit d.
//   TARGET = false: returns the optical depth to the grid edge in tau_raw.
//   TARGET = true : stops where the optical depth reaches target (true, t_out = path
//                   length), or leaves the grid first (false, t_out = far end of the
//                   last segment with nonzero density).
// Each axis keeps the distance to its own next face, so a segment length is the
// smallest of three cell-sized numbers rather than a difference of two path
// lengths of order one: in float this keeps every segment, and hence every cell's
// optical depth, to a few units in the last place.  Sums run over raw cell values
// (the caller scales by kscale) with Kahan compensation.
//
// The geometry of a walk does not depend on the densities, so it runs WALK_UNROLL
// cells ahead: one batch computes the segments and cell indices of the next cells,
// issues their density loads together (independent loads in flight at once instead
// of one dependent load per cell), then accumulates their optical depths in order.
// After the ray leaves the grid the rest of the batch repeats the last cell with
// zero length, so no load leaves the grid.
constexpr int WALK_UNROLL = 4;
static_assert(QMCRT_MIN_PAD >= WALK_UNROLL, "a padded walk steps up to WALK_UNROLL - 1 cells past the first sentinel");

template <class T, bool TARGET>
__device__ __forceinline__ bool grid_walk(const MediumP<T> &G, const T p[3], const T d[3], const T r[3], T target_raw,
                                          T &tau_raw, T &t_out)
{
    const int cx = start_cell(p[0], G.lo[0], G.h[0], G.inv_h[0], d[0]);
    const int cy = start_cell(p[1], G.lo[1], G.h[1], G.inv_h[1], d[1]);
    const int cz = start_cell(p[2], G.lo[2], G.h[2], G.inv_h[2], d[2]);
    tau_raw = T(0);
    t_out = T(0);
    if (!walkable(p, d)) return false;
    if (cx < 0 || cx >= G.n[0] || cy < 0 || cy >= G.n[1] || cz < 0 || cz >= G.n[2]) return false;
    AxisWalk<T> X = axis_setup(p[0], d[0], r[0], cx, G.lo[0], G.h[0], G.n[0], G.stride[0]);
    AxisWalk<T> Y = axis_setup(p[1], d[1], r[1], cy, G.lo[1], G.h[1], G.n[1], G.stride[1]);
    AxisWalk<T> Z = axis_setup(p[2], d[2], r[2], cz, G.lo[2], G.h[2], G.n[2], G.stride[2]);
    if (X.step == 0 && Y.step == 0 && Z.step == 0) return false;
    int idx = cx * G.stride[0] + cy * G.stride[1] + cz * G.stride[2];
    const float *__restrict__ K = G.k;
    T t = T(0), acc = TARGET ? target_raw : T(0), comp = T(0), t_last = T(0);
    bool done = false;
    for (;;) {
        T L[WALK_UNROLL];
        int cell[WALK_UNROLL];
#pragma unroll
        for (int u = 0; u < WALK_UNROLL; ++u) {
            cell[u] = idx;
            const T l = done ? T(0) : Mth<T>::min_(X.s, Mth<T>::min_(Y.s, Z.s));
            L[u] = l;
            X.s -= l;  // exact (zero) for the axis whose face is reached
            Y.s -= l;
            Z.s -= l;
            if (!done) {
                if (X.s == T(0)) {  // ties step x, then y, then z
                    done = X.left-- == 0;
                    if (!done) {
                        idx += X.step;
                        X.s = X.dt;
                    }
                } else if (Y.s == T(0)) {
                    done = Y.left-- == 0;
                    if (!done) {
                        idx += Y.step;
                        Y.s = Y.dt;
                    }
                } else {
                    done = Z.left-- == 0;
                    if (!done) {
                        idx += Z.step;
                        Z.s = Z.dt;
                    }
                }
            }
        }
        T kc[WALK_UNROLL];
#pragma unroll
        for (int u = 0; u < WALK_UNROLL; ++u) kc[u] = (T)__ldg(K + cell[u]);
#pragma unroll
        for (int u = 0; u < WALK_UNROLL; ++u) {
            const T dtau = L[u] * kc[u];
            if (TARGET) {
                const T rem = acc - comp;
                if (kc[u] > T(0) && dtau >= rem) {
                    t_out = t + rem / kc[u];
                    tau_raw = target_raw;
                    return true;
                }
                const T y = -dtau - comp;  // acc -= dtau, compensated
                const T s = acc + y;
                comp = (s - acc) - y;
                acc = s;
                t += L[u];
                if (kc[u] > T(0) && L[u] > T(0)) t_last = t;
            } else {
                const T y = dtau - comp;  // acc += dtau, compensated
                const T s = acc + y;
                comp = (s - acc) - y;
                acc = s;
            }
        }
        if (done) break;
    }
    if (TARGET) {
        t_out = t_last;
        tau_raw = target_raw - (acc - comp);
    } else {
        tau_raw = acc - comp;
    }
    return false;
}

// The same walk over a padded grid (QMCRT pad >= WALK_UNROLL): the grid is
// surrounded by `pad` layers of sentinel cells holding -0.0, and the interior holds no
// negative zero (qmcrt_pad_grid writes +0 for empty, negative or NaN cells).  The walk
// needs no per-axis cell counters: a batch of WALK_UNROLL cells is stepped blindly (at
// most WALK_UNROLL cells past the box, still inside the padding), a sentinel adds
// L * (-0) = -0, nothing, and the walk ends after the first batch in which a loaded
// value has its sign bit set.  The box is convex and axis-aligned, so once a step
// leaves it along any axis every later cell of the ray is outside too.  The optical
// depths of a batch are summed in order and the batch sum enters the compensated
// total; the march tests the batch sum against the remaining depth and only then
// looks for the stopping cell inside the batch.
// State of a padded walk between batches: each axis's face distance and step, and the
// element index of the next cell.
template <class T>
struct PaddedRay {
    AxisWalk<T> X, Y, Z;
    unsigned idx;
};

// A batch boundary of a padded walk, from which a later walk along the same ray resumes
// with the same arithmetic: the state there, the path length and the compensated raw
// optical depth from the start.
template <class T>
struct WalkMark {
    T s[3], tau;
    unsigned idx;
};

template <class T>
__device__ __forceinline__ void mark_at(WalkMark<T> &M, const PaddedRay<T> &R, T tau)
{
    M.s[0] = R.X.s;
    M.s[1] = R.Y.s;
    M.s[2] = R.Z.s;
    M.tau = tau;
    M.idx = R.idx;
}

// Path length from the walk's start p to the boundary of a mark: the distance along d to
// the next face of the mark's cell on the axis a with the largest |d| (the face as the walk
// set it up, from the cell index), less the remaining face distance the walk carried there.
template <class T>
__device__ __forceinline__ T mark_length(const MediumP<T> &G, const WalkMark<T> &M, const T p[3], const T d[3],
                                         const T r[3])
{
    unsigned q = M.idx;
    const unsigned iz = q / (unsigned)G.stride[2];
    q -= iz * (unsigned)G.stride[2];
    const unsigned iy = q / (unsigned)G.stride[1];
    const unsigned ix = q - iy * (unsigned)G.stride[1];
    const int c[3] = {(int)ix - G.pad, (int)iy - G.pad, (int)iz - G.pad};
    const T ad[3] = {Mth<T>::max_(d[0], -d[0]), Mth<T>::max_(d[1], -d[1]), Mth<T>::max_(d[2], -d[2])};
    const int a = (ad[0] >= ad[1] && ad[0] >= ad[2]) ? 0 : (ad[1] >= ad[2] ? 1 : 2);
    const T face = Mth<T>::face(G.lo[a], d[a] > T(0) ? c[a] + 1 : c[a], G.h[a]);
    return Mth<T>::mul_(face - p[a], r[a]) - M.s[a];
}

// Start of a walk over a padded grid; false if p is outside the grid or not finite, or d
// crosses no axis (the walk then has zero depth and zero length).
template <class T>
__device__ __forceinline__ bool padded_start(const MediumP<T> &G, const T p[3], const T d[3], const T r[3],
                                             PaddedRay<T> &R)
{
    const int cx = start_cell(p[0], G.lo[0], G.h[0], G.inv_h[0], d[0]);
    const int cy = start_cell(p[1], G.lo[1], G.h[1], G.inv_h[1], d[1]);
    const int cz = start_cell(p[2], G.lo[2], G.h[2], G.inv_h[2], d[2]);
    if (!walkable(p, d)) return false;
    if (cx < 0 || cx >= G.n[0] || cy < 0 || cy >= G.n[1] || cz < 0 || cz >= G.n[2]) return false;
    R.X = axis_setup(p[0], d[0], r[0], cx, G.lo[0], G.h[0], G.n[0], G.stride[0]);
    R.Y = axis_setup(p[1], d[1], r[1], cy, G.lo[1], G.h[1], G.n[1], G.stride[1]);
    R.Z = axis_setup(p[2], d[2], r[2], cz, G.lo[2], G.h[2], G.n[2], G.stride[2]);
    if (R.X.step == 0 && R.Y.step == 0 && R.Z.step == 0) return false;
    // Cells are addressed by an unsigned 32-bit element index (one wide multiply-add per
    // load; padded grids hold at most 2^31 cells, and steps are added modulo 2^32).
    R.idx = (unsigned)((cx + G.pad) * G.stride[0] + (cy + G.pad) * G.stride[1] + (cz + G.pad) * G.stride[2]);
    return true;
}

// One batch: the segment lengths and cell values of the next WALK_UNROLL cells; returns
// the OR of the values' bits (sign bit set: the ray has left the grid).
template <class T>
__device__ __forceinline__ unsigned padded_batch(const float *__restrict__ K, PaddedRay<T> &R, T L[WALK_UNROLL],
                                                 float kf[WALK_UNROLL])
{
    unsigned cell[WALK_UNROLL];
#pragma unroll
    for (int u = 0; u < WALK_UNROLL; ++u) {
        cell[u] = R.idx;
        const T l = Mth<T>::min_(R.X.s, Mth<T>::min_(R.Y.s, R.Z.s));
        L[u] = l;
        R.X.s -= l;  // exact (zero) for the axis whose face is reached
        R.Y.s -= l;
        R.Z.s -= l;
        if (R.X.s == T(0)) {  // ties step x, then y, then z
            R.idx += R.X.step;
            R.X.s = R.X.dt;
        } else if (R.Y.s == T(0)) {
            R.idx += R.Y.step;
            R.Y.s = R.Y.dt;
        } else {
            R.idx += R.Z.step;
            R.Z.s = R.Z.dt;
        }
    }
    unsigned sign = 0u;
#pragma unroll
    for (int u = 0; u < WALK_UNROLL; ++u) {
        kf[u] = __ldg(K + cell[u]);
        sign |= __float_as_uint(kf[u]);
    }
    return sign;
}

// Raw optical depth from the state R to the edge of the grid.
template <class T>
__device__ __forceinline__ T padded_depth(const float *__restrict__ K, PaddedRay<T> &R)
{
    T acc = T(0), comp = T(0);
    for (;;) {
        T L[WALK_UNROLL];
        float kf[WALK_UNROLL];
        const unsigned sign = padded_batch(K, R, L, kf);
        T Bs = T(0);  // the batch's optical depth, one fused multiply-add per cell
#pragma unroll
        for (int u = 0; u < WALK_UNROLL; ++u) Bs = Mth<T>::fma_(L[u], (T)kf[u], Bs);
        const T y = Bs - comp;  // acc += Bs, compensated
        const T s2 = acc + y;
        comp = (s2 - acc) - y;
        acc = s2;
        if (sign & 0x80000000u) break;
    }
    return acc - comp;
}

// The same depth toward an observer with a tail map (qmcrt_tail_map): the code of each
// batch's first cell, loaded with the batch's densities, bounds the optical depth from that
// cell to the edge; once it is at most thr the walk ends after the batch, leaving out at
// most the bound the threshold stands for.
template <class T>
__device__ __forceinline__ T padded_depth_tail(const float *__restrict__ K, PaddedRay<T> &R,
                                               const uint8_t *__restrict__ tail, int thr)
{
    T acc = T(0), comp = T(0);
    for (;;) {
        const int code = __ldg(tail + R.idx);
        T L[WALK_UNROLL];
        float kf[WALK_UNROLL];
        const unsigned sign = padded_batch(K, R, L, kf);
        T Bs = T(0);
#pragma unroll
        for (int u = 0; u < WALK_UNROLL; ++u) Bs = Mth<T>::fma_(L[u], (T)kf[u], Bs);
        const T y = Bs - comp;
        const T s2 = acc + y;
        comp = (s2 - acc) - y;
        acc = s2;
        if ((sign & 0x80000000u) || code <= thr) break;
    }
    return acc - comp;
}

// The same depth, keeping two batch boundaries for a march to the forced depth
// tau(tau_1) = -ln[1 - w (1 - e^{-tau_1})] along the same ray: a candidate B, and A, the
// candidate last promoted (initially the start), in mk[ia ^ 1] and mk[ia] (local memory:
// written at promotions only).  B is promoted once the depth x walked so far gives
// w x / (1 + x) >= B's depth, that is once x reaches b / (w - b) (physical units): since
// w x / (1 + x) <= w (1 - e^{-x}) <= tau(x) <= tau(tau_1), A then lies before the stopping
// point; B is renewed at the same boundary.  Between promotions a batch costs the plain
// depth loop's work and a comparison.  Which boundaries are kept is a heuristic only:
// the caller resumes from one whose depth it has checked against the target.
// Promotions are considered at every MARK_GAP-th batch boundary only: the lanes of a warp
// walk their batches in step, so a promotion in any lane holds up the others, and where
// the depth grows by large factors per batch (the edge of an atmosphere whose density
// falls off as a Gaussian) every boundary would qualify.  Measured on the flared disk
// (2^26 packets): 15.5 ms without marks; 14.1, 13.5, 13.3, 13.2 and 13.4 ms with gaps of 1,
// 2, 4, 8 and 16 batches (the finite star and the batch gain most from 8 to 16).
constexpr unsigned MARK_GAP = 8;

template <class T>
__device__ __forceinline__ T padded_depth_marks(const float *__restrict__ K, PaddedRay<T> &R, T w, T kscale,
                                                WalkMark<T> mk[2], int &ia, bool &has_b)
{
    T acc = T(0), comp = T(0), thr = T(0);
    unsigned nb = 0;  // batches walked: promotions are considered at every MARK_GAP-th
    ia = 0;
    has_b = false;
    mark_at(mk[0], R, T(0));
    for (;;) {
        T L[WALK_UNROLL];
        float kf[WALK_UNROLL];
        const unsigned sign = padded_batch(K, R, L, kf);
        T Bs = T(0);
#pragma unroll
        for (int u = 0; u < WALK_UNROLL; ++u) Bs = Mth<T>::fma_(L[u], (T)kf[u], Bs);
        const T y = Bs - comp;
        const T s2 = acc + y;
        comp = (s2 - acc) - y;
        acc = s2;
        if (sign & 0x80000000u) break;
        if (++nb % MARK_GAP == 0 && acc >= thr) {  // the same batches in every lane of a warp
            if (has_b) ia ^= 1;  // A = B
            const T b = acc - comp;
            mark_at(mk[ia ^ 1], R, b);
            has_b = true;
            const T den = w - Mth<T>::mul_(kscale, b);
            thr = den > T(0) ? b / den : Mth<T>::inf();
        }
    }
    return acc - comp;
}

// March from the state R (path length t0 and raw depth tau0 from the walk's start, tau0
// below target_raw) until the optical depth reaches target_raw (true, t_out = path length
// from the start) or the ray leaves the grid (false, t_out = far end of the last segment
// with nonzero density, at least t0).  From the start (t0 = tau0 = 0) this is the walk's
// own march; from a kept boundary it walks the same cells with the same segments.
template <class T>
__device__ __forceinline__ bool padded_march(const float *__restrict__ K, PaddedRay<T> &R, T t0, T tau0,
                                             T target_raw, T &tau_raw, T &t_out)
{
    T t = t0, acc = target_raw - tau0, comp = T(0), t_last = t0;
    for (;;) {
        T L[WALK_UNROLL];
        float kf[WALK_UNROLL];
        const unsigned sign = padded_batch(K, R, L, kf);
        T dtau[WALK_UNROLL];  // each cell's optical depth, and their sum in order
        T Bs = T(0);
#pragma unroll
        for (int u = 0; u < WALK_UNROLL; ++u) {
            dtau[u] = Mth<T>::mul_(L[u], (T)kf[u]);
            Bs = Mth<T>::add_(Bs, dtau[u]);
        }
        T rem = acc - comp;
        if (Bs >= rem) {  // the stopping cell is in this batch (or rounding says so)
#pragma unroll
            for (int u = 0; u < WALK_UNROLL; ++u) {
                if (dtau[u] > T(0) && dtau[u] >= rem) {
                    t_out = t + rem / (T)kf[u];
                    tau_raw = target_raw;
                    return true;
                }
                rem -= dtau[u];
                t += L[u];
                if (dtau[u] > T(0)) t_last = t;
            }
            acc = rem;
            comp = T(0);
        } else {
            const T y = -Bs - comp;  // acc -= Bs, compensated
            const T s2 = acc + y;
            comp = (s2 - acc) - y;
            acc = s2;
#pragma unroll
            for (int u = 0; u < WALK_UNROLL; ++u) {
                t += L[u];
                if (dtau[u] > T(0)) t_last = t;
            }
        }
        if (sign & 0x80000000u) break;
    }
    t_out = t_last;
    tau_raw = target_raw - (acc - comp);
    return false;
}

// The same walk over a padded grid (QMCRT pad >= WALK_UNROLL): the grid is
// surrounded by `pad` layers of sentinel cells holding -0.0, and the interior holds no
// negative zero (qmcrt_pad_grid writes +0 for empty, negative or NaN cells).  The walk
// needs no per-axis cell counters: a batch of WALK_UNROLL cells is stepped blindly (at
// most WALK_UNROLL cells past the box, still inside the padding), a sentinel adds
// L * (-0) = -0, nothing, and the walk ends after the first batch in which a loaded
// value has its sign bit set.  The box is convex and axis-aligned, so once a step
// leaves it along any axis every later cell of the ray is outside too.  The optical
// depths of a batch are summed in order and the batch sum enters the compensated
// total; the march tests the batch sum against the remaining depth and only then
// looks for the stopping cell inside the batch.
template <class T, bool TARGET>
__device__ __forceinline__ bool grid_walk_padded(const MediumP<T> &G, const T p[3], const T d[3], const T r[3],
                                                 T target_raw, T &tau_raw, T &t_out)
{
    tau_raw = T(0);
    t_out = T(0);
    PaddedRay<T> R;
    if (!padded_start(G, p, d, r, R)) return false;
    if (TARGET) return padded_march(G.k, R, T(0), T(0), target_raw, tau_raw, t_out);
    tau_raw = padded_depth(G.k, R);
    return false;
}

// Distance from p (inside) along unit d to the sphere of radius r at the origin.
template <class T>
__device__ __forceinline__ T sphere_exit(const T p[3], const T d[3], T r)
{
    const T b = dot3(p, d);
    const T c = dot3(p, p) - r * r;
    const T disc = Mth<T>::max_(b * b - c, T(0));
    return Mth<T>::max_(-b + Mth<T>::sqrt_(disc), T(0));
}

// The reciprocals 1 / d of a direction's components (the walks' face distances).
template <class T>
__device__ __forceinline__ void reciprocals(const T d[3], T r[3])
{
    r[0] = T(1) / d[0];
    r[1] = T(1) / d[1];
    r[2] = T(1) / d[2];
}

// Optical depth from p along d (r = 1 / d) to the edge of the medium.
template <class T>
__device__ __forceinline__ T tau_to_edge(const MediumP<T> &G, const T p[3], const T d[3], const T r[3])
{
    if (G.kind == QMCRT_MEDIUM_SPHERE) {
        if (dot3(p, p) > G.sph_r * G.sph_r) return T(0);
        return G.sph_k * sphere_exit(p, d, G.sph_r);
    }
    T raw, t;
    if (G.pad) grid_walk_padded<T, false>(G, p, d, r, T(0), raw, t);
    else grid_walk<T, false>(G, p, d, r, T(0), raw, t);
    return Mth<T>::mul_(raw, G.kscale);
}

// Optical depth from p toward observer O (the peel-off walk), ended early by O's tail map
// where the observer has one.
template <class T>
__device__ __forceinline__ T tau_toward(const MediumP<T> &G, const ObsP<T> &O, const T p[3])
{
    if (O.tail && G.kind == QMCRT_MEDIUM_GRID && G.pad) {
        PaddedRay<T> R;
        if (!padded_start(G, p, O.k, O.inv_k, R)) return T(0);
        return Mth<T>::mul_(padded_depth_tail(G.k, R, O.tail, O.tail_thr), G.kscale);
    }
    return tau_to_edge(G, p, O.k, O.inv_k);
}

template <class T>
__device__ __forceinline__ T tau_to_edge(const MediumP<T> &G, const T p[3], const T d[3])
{
    T r[3];
    reciprocals(d, r);
    return tau_to_edge(G, p, d, r);
}

// Move pos along d (r = 1 / d) through optical depth tau; false if the ray leaves first
// (pos is then the far end of the last nonempty segment).
template <class T>
__device__ __forceinline__ bool march(const MediumP<T> &G, T pos[3], const T d[3], const T r[3], T tau)
{
    T t;
    bool hit;
    if (G.kind == QMCRT_MEDIUM_SPHERE) {
        const T s = sphere_exit(pos, d, G.sph_r);
        hit = G.sph_k > T(0) && tau < G.sph_k * s;
        t = hit ? tau / G.sph_k : s;
    } else {
        T raw;
        const T target_raw = Mth<T>::mul_(tau, G.inv_kscale);
        hit = G.pad ? grid_walk_padded<T, true>(G, pos, d, r, target_raw, raw, t)
                    : grid_walk<T, true>(G, pos, d, r, target_raw, raw, t);
    }
    pos[0] += t * d[0];
    pos[1] += t * d[1];
    pos[2] += t * d[2];
    return hit;
}

template <class T>
__device__ __forceinline__ bool march(const MediumP<T> &G, T pos[3], const T d[3], T tau)
{
    T r[3];
    reciprocals(d, r);
    return march(G, pos, d, r, tau);
}

// The bound of qmcrt_sky_bound on the optical depth (without kscale) of a ray along d that
// starts within the map's radius of the origin: one cube-map texel (face of the major
// axis, ties to the lower axis).
template <class T>
__device__ __forceinline__ double sky_bound(const MediumP<T> &G, const T d[3])
{
    const T ax = Mth<T>::max_(d[0], -d[0]), ay = Mth<T>::max_(d[1], -d[1]), az = Mth<T>::max_(d[2], -d[2]);
    int a;
    T w, u, v;
    if (ax >= ay && ax >= az) {
        a = 0; w = ax; u = d[1]; v = d[2];
    } else if (ay >= az) {
        a = 1; w = ay; u = d[0]; v = d[2];
    } else {
        a = 2; w = az; u = d[0]; v = d[1];
    }
    const int m = G.sky_m;
    const int f = 2 * a + (d[a] < T(0) ? 1 : 0);
    const int iu = min(m - 1, max(0, (int)Mth<T>::floor_((u / w + T(1)) * T(0.5) * T(m))));
    const int iv = min(m - 1, max(0, (int)Mth<T>::floor_((v / w + T(1)) * T(0.5) * T(m))));
    return __ldg(G.sky + ((size_t)f * m + iv) * m + iu);
}

// Forced scattering (Sec. 3.2): weight 1 - e^{-tau_1}, depth -ln[1 - w (1 - e^{-tau_1})].
// A ray from within the bound map's radius whose direction's bound (qmcrt_sky_bound, with
// a factor of two for the float walk's rounding) lies below tau_min cannot reach it: the
// packet is skipped as the walk would skip it, without walking.
template <class T>
__device__ __forceinline__ bool forced_step(const TraceP<T> &P, T pos[3], const T d[3], T w, T &W1)
{
    if (P.med.sky && dot3(pos, pos) <= P.med.sky_r2 &&
        2.0 * sky_bound(P.med, d) * (double)P.med.kscale < (double)P.tau_min)
        return false;
    T r[3];  // both walks run along d
    reciprocals(d, r);
    PaddedRay<T> R;
    if (P.med.kind != QMCRT_MEDIUM_GRID || !P.med.pad || !padded_start(P.med, pos, d, r, R)) {
        const T tau1 = tau_to_edge(P.med, pos, d, r);
        if (!(tau1 >= P.tau_min)) return false;
        W1 = -Mth<T>::expm1_(-tau1);
        const T tau = -Mth<T>::log1p_(-w * W1);
        march(P.med, pos, d, r, tau);
        return true;
    }
    // The march to the forced depth resumes from the latest boundary kept by the first
    // walk whose depth lies below the target (and below tau_1, so that cells of nonzero
    // density follow it): the cells before it hold less than the target, so the march
    // from the start would cross them without stopping.
    WalkMark<T> mk[2];
    int ia;
    bool has_b;
    const T raw1 = padded_depth_marks(P.med.k, R, w, P.med.kscale, mk, ia, has_b);
    const T tau1 = Mth<T>::mul_(raw1, P.med.kscale);
    if (!(tau1 >= P.tau_min)) return false;
    W1 = -Mth<T>::expm1_(-tau1);
    const T tau = -Mth<T>::log1p_(-Mth<T>::mul_(w, W1));
    const T target_raw = Mth<T>::mul_(tau, P.med.inv_kscale);
    int im = ia;  // B if it lies before the target, else A (the start until promoted)
    if (has_b && mk[ia ^ 1].tau < target_raw && mk[ia ^ 1].tau < raw1) im = ia ^ 1;
    T raw, t;
    const bool usable = mk[im].tau < target_raw && mk[im].tau < raw1;
    bool hit = false, resumed = false;
    if (usable) {
        const WalkMark<T> &M = mk[im];
        R.X.s = M.s[0];
        R.Y.s = M.s[1];
        R.Z.s = M.s[2];
        R.idx = M.idx;
        const T t0 = mark_length(P.med, M, pos, d, r);  // exactly 0 at the start
        resumed = t0 > T(0);
        hit = padded_march(P.med.k, R, t0, M.tau, target_raw, raw, t);
    }
    // From the start when rounding put both kept boundaries past the target, or when a
    // resumed march left the grid (then the last segment of nonzero density may lie
    // before the boundary, and the walk's own result is the march from the start).
    if (!hit && (resumed || !usable)) {
        padded_start(P.med, pos, d, r, R);
        padded_march(P.med.k, R, T(0), T(0), target_raw, raw, t);
    }
    pos[0] = Mth<T>::fma_(t, d[0], pos[0]);
    pos[1] = Mth<T>::fma_(t, d[1], pos[1]);
    pos[2] = Mth<T>::fma_(t, d[2], pos[2]);
    return true;
}

// ------------------------------------------------------------------------------------
// Sources (Sec. 3.2, 3.3)
// ------------------------------------------------------------------------------------

// Unit vector from cos(theta) = c and phi = 2 pi u, with its e_theta axis.
template <class T>
__device__ __forceinline__ void direction_from(T u, T v, T d[3], T et[3], T &sp, T &cp)
{
    Mth<T>::sincospi_(T(2) * u, &sp, &cp);
    const T ct = T(2) * v - T(1);
    const T st = T(2) * Mth<T>::sqrt_(Mth<T>::max_(v * (T(1) - v), T(0)));
    d[0] = st * cp;
    d[1] = st * sp;
    d[2] = ct;
    et[0] = ct * cp;
    et[1] = ct * sp;
    et[2] = -st;
}

// e_theta of a unit vector given by components.
template <class T>
__device__ __forceinline__ void e_theta_of(const T d[3], T et[3])
{
    const T s = Mth<T>::sqrt_(d[0] * d[0] + d[1] * d[1]);
    T cp = T(1), sp = T(0);
    if (s > T(0)) {
        cp = d[0] / s;
        sp = d[1] / s;
    }
    et[0] = d[2] * cp;
    et[1] = d[2] * sp;
    et[2] = -s;
}

// Emission of packet i (Sec. 3.2, 3.3): position, direction, Stokes axis, weight;
// returns the depth coordinate w.  Coordinates 0, 1 set the emission point (direct order) or
// the direction (inverse order); c0, c1 the other pair (local direction, or the point
// on the projected disk); cw the first depth.  Single scattering reads them in the
// paper's order (direct: c0 = 2, c1 = 3, cw = 4; inverse: cw = 2, c0 = 3, c1 = 4).
template <class T>
__device__ __forceinline__ T emit(const TraceP<T> &P, uint64_t i, T pos[3], T d[3], T a[3], T &wgt, int c0, int c1,
                                  int cw)
{
    wgt = T(1);
    T sp, cp;
    if (P.src.kind == QMCRT_SOURCE_POINT) {
        direction_from(point<T>(P.pts, i, 0), point<T>(P.pts, i, 1), d, a, sp, cp);
        pos[0] = pos[1] = pos[2] = T(0);
        return point<T>(P.pts, i, 2);
    }
    const T R = P.src.R;
    T mu, w;
    if (P.src.order == QMCRT_ORDER_DIRECT) {
        // v1, v2: emission point; v3, v4: local direction (cos theta_l = sqrt(v4),
        // cosine-weighted outward hemisphere); v5: depth.
        T ne[3], et[3];
        direction_from(point<T>(P.pts, i, 0), point<T>(P.pts, i, 1), ne, et, sp, cp);
        const T ep[3] = {-sp, cp, T(0)};
        T spl, cpl;
        Mth<T>::sincospi_(T(2) * point<T>(P.pts, i, c0), &spl, &cpl);
        const T v4 = point<T>(P.pts, i, c1);
        mu = Mth<T>::sqrt_(v4);
        const T sl = Mth<T>::sqrt_(Mth<T>::max_(T(1) - v4, T(0)));
        for (int q = 0; q < 3; ++q) {
            pos[q] = R * ne[q];
            d[q] = sl * cpl * et[q] + sl * spl * ep[q] + mu * ne[q];
        }
        normalize3(d);
        e_theta_of(d, a);
        w = point<T>(P.pts, i, cw);
    } else {
        // v1, v2: direction; v3: depth; v4, v5: emission point uniform on the star's
        // projected disk across the direction, lifted onto the facing hemisphere.
        direction_from(point<T>(P.pts, i, 0), point<T>(P.pts, i, 1), d, a, sp, cp);
        const T ep[3] = {-sp, cp, T(0)};
        w = point<T>(P.pts, i, cw);
        const T v4 = point<T>(P.pts, i, c0);
        T sps, cps;
        Mth<T>::sincospi_(T(2) * point<T>(P.pts, i, c1), &sps, &cps);
        const T rho = R * Mth<T>::sqrt_(v4);
        mu = Mth<T>::sqrt_(Mth<T>::max_(T(1) - v4, T(0)));
        const T lift = R * mu;
        for (int q = 0; q < 3; ++q) pos[q] = rho * (cps * a[q] + sps * ep[q]) + lift * d[q];
    }
    wgt = (T(1) - P.src.limb_u + P.src.limb_u * mu) * P.src.limb_norm;
    return w;
}

template <class T>
__device__ __forceinline__ T emit(const TraceP<T> &P, uint64_t i, T pos[3], T d[3], T a[3], T &wgt)
{
    const bool direct = P.src.order == QMCRT_ORDER_DIRECT;
    return emit(P, i, pos, d, a, wgt, direct ? 2 : 3, direct ? 3 : 4, direct ? 4 : 2);
}

// ------------------------------------------------------------------------------------
// Scattering and peel-off (Sec. 2.2, 3.5, 3.6)
// ------------------------------------------------------------------------------------

// Henyey-Greenstein function x_HG(mu) = P11.
template <class T>
__device__ __forceinline__ T hg_p11(const DustP<T> &D, T mu)
{
    const T den = D.one_p_g2 - D.two_g * mu;
    return D.one_m_g2 / (den * Mth<T>::sqrt_(den));
}

// cos Theta from v by inverting the HG distribution (Sec. 3.5).
template <class T>
__device__ __forceinline__ T hg_cos(const DustP<T> &D, T v)
{
    T c;
    if (D.isotropic) {
        c = T(2) * v - T(1);
    } else {
        const T f = D.one_m_g2 / (T(1) - D.g + D.two_g * v);
        c = (D.one_p_g2 - f * f) / D.two_g;
    }
    return Mth<T>::min_(Mth<T>::max_(c, T(-1)), T(1));
}

// Q' = Q cos 2psi + U sin 2psi, U' = -Q sin 2psi + U cos 2psi for a reference axis
// turned by psi (given cos psi, sin psi up to a common positive factor s: c2, s2 are
// then scaled by s^2; callers pass unit values or divide).
template <class T>
__device__ __forceinline__ void rotate_stokes(T cps, T sps, T &Q, T &U)
{
    const T c2 = cps * cps - sps * sps, s2 = T(2) * cps * sps;
    const T q = Q * c2 + U * s2;
    U = -Q * s2 + U * c2;
    Q = q;
}

template <class T>
__device__ __forceinline__ bool occulted(const TraceP<T> &P, const ObsP<T> &O, const T pos[3])
{
    if (P.src.kind != QMCRT_SOURCE_SPHERE) return false;
    const T b = dot3(pos, O.k);
    const T c = dot3(pos, pos) - P.src.R * P.src.R;
    return c <= T(0) || (b < T(0) && b * b - c > T(0));
}

// Peel-off of an unpolarized packet of weight W0 travelling along d, scattering at
// pos.  In the image frame the White polarization is perpendicular to the scattering
// plane; with (dx, dy) the sky projection of d this is
//   Q = W p_l (dx^2 - dy^2) / (1 + mu^2),  U = W p_l 2 dx dy / (1 + mu^2).
template <class T>
__device__ __forceinline__ bool peel_unpolarized(const TraceP<T> &P, const ObsP<T> &O, const T pos[3], const T d[3],
                                                 T W0, T S[3], T &x, T &y)
{
    x = dot3(pos, O.ex);
    y = dot3(pos, O.ey);
    if (occulted(P, O, pos)) return false;
    const T tau_obs = tau_toward(P.med, O, pos);
    const T mu = dot3(d, O.k);
    const T f = W0 * Mth<T>::exp_(-tau_obs) * hg_p11(P.dust, mu) * T(0.07957747154594767);  // 1/(4 pi)
    const T dx = dot3(d, O.ex), dy = dot3(d, O.ey);
    const T q = f * P.dust.p_l / (T(1) + mu * mu);
    S[0] = f;
    S[1] = q * (dx * dx - dy * dy);
    S[2] = q * T(2) * dx * dy;
    return true;
}

// Peel-off of a polarized packet (direction n, Stokes S in the frame of axis a).
template <class T>
__device__ __forceinline__ bool peel_polarized(const TraceP<T> &P, const ObsP<T> &O, const T pos[3], const T n[3],
                                               const T a[3], const T S[3], T out[3], T &x, T &y)
{
    x = dot3(pos, O.ex);
    y = dot3(pos, O.ey);
    if (occulted(P, O, pos)) return false;
    const T tau_obs = tau_toward(P.med, O, pos);
    const T mu = dot3(n, O.k);
    const T inv1pm2 = T(1) / (T(1) + mu * mu);
    const T r12 = -P.dust.p_l * (T(1) - mu * mu) * inv1pm2;
    const T r33 = T(2) * mu * inv1pm2;
    T b[3], m[3], pin[3];
    cross3(n, a, b);
    cross3(n, O.k, m);
    if (dot3(m, m) < T(1e-24)) {
        m[0] = b[0];
        m[1] = b[1];
        m[2] = b[2];
    }
    normalize3(m);
    cross3(m, n, pin);
    T Q = S[1], U = S[2];
    rotate_stokes(dot3(a, pin), dot3(b, pin), Q, U);
    const T f = Mth<T>::exp_(-tau_obs) * hg_p11(P.dust, mu) * T(0.07957747154594767);
    T Io = f * (S[0] + r12 * Q);
    T Qo = f * (r12 * S[0] + Q);
    T Uo = f * r33 * U;
    // scattering frame (m x k, m, k) -> image frame (ey, -ex, k): cos psi = -m.ex, sin psi = m.ey
    rotate_stokes(-dot3(m, O.ex), dot3(m, O.ey), Qo, Uo);
    out[0] = Io;
    out[1] = Qo;
    out[2] = Uo;
    return true;
}

// The peel-offs toward the problem's own observer.
template <class T>
__device__ __forceinline__ bool peel_unpolarized(const TraceP<T> &P, const T pos[3], const T d[3], T W0, T S[3],
                                                 T &x, T &y)
{
    return peel_unpolarized(P, P.obs, pos, d, W0, S, x, y);
}

template <class T>
__device__ __forceinline__ bool peel_polarized(const TraceP<T> &P, const T pos[3], const T n[3], const T a[3],
                                               const T S[3], T out[3], T &x, T &y)
{
    return peel_polarized(P, P.obs, pos, n, a, S, out, x, y);
}

// HG scattering of a polarized packet (Sec. 3.5): Theta from v, azimuth 2 pi u from
// axis a; Stokes rotated into the scattering plane and multiplied by M/P11.
template <class T>
__device__ __forceinline__ void scatter(const DustP<T> &D, T u, T v, T n[3], T a[3], T S[3])
{
    const T ct = hg_cos(D, v);
    const T st = Mth<T>::sqrt_(Mth<T>::max_((T(1) - ct) * (T(1) + ct), T(0)));
    T si, ci;
    Mth<T>::sincospi_(T(2) * u, &si, &ci);
    T b[3], nn[3], m[3], an[3];
    cross3(n, a, b);
    for (int q = 0; q < 3; ++q) {
        nn[q] = ct * n[q] + st * (ci * a[q] + si * b[q]);
        m[q] = ci * b[q] - si * a[q];
    }
    normalize3(nn);
    T Q = S[1], U = S[2];
    rotate_stokes(ci, si, Q, U);
    const T inv1pm2 = T(1) / (T(1) + ct * ct);
    const T r12 = -D.p_l * (T(1) - ct * ct) * inv1pm2;
    const T r33 = T(2) * ct * inv1pm2;
    const T I = S[0];
    S[0] = I + r12 * Q;
    S[1] = r12 * I + Q;
    S[2] = r33 * U;
    cross3(m, nn, an);
    normalize3(an);
    for (int q = 0; q < 3; ++q) {
        n[q] = nn[q];
        a[q] = an[q];
    }
}

// ------------------------------------------------------------------------------------
// Image deposits
// ------------------------------------------------------------------------------------

// Add (I, Q, U) at accumulation element e (I plane; Q, U one and two planes further).
// Lanes of a warp that hit the same pixel are summed with shuffles first (exactly, in
// fixed point) so that a coherent warp issues one atomic per Stokes component; warps
// spread over many pixels add directly.  Must be called by all 32 lanes.
template <class T>
__device__ __forceinline__ void deposit(const AccumP &A, bool valid, size_t e, T I, T Q, T U)
{
    const int lane = threadIdx.x & 31;
    const unsigned vmask = __ballot_sync(FULL_MASK, valid);
    if (vmask == 0) return;
    const unsigned long long key = valid ? (unsigned long long)e : ~0ull;
    const unsigned peers = __match_any_sync(FULL_MASK, key);
    const bool leader = valid && ((peers & ((1u << lane) - 1u)) == 0u);
    unsigned leaders = __ballot_sync(FULL_MASK, leader);
    const bool aggregate = __popc(leaders) <= 4;
    if (A.mode == QMCRT_ACCUM_I64) {
        unsigned long long *dst = (unsigned long long *)A.ptr;
        long long qi = valid ? Mth<T>::to_fixed(I, A.scale) : 0;
        long long qq = valid ? Mth<T>::to_fixed(Q, A.scale) : 0;
        long long qu = valid ? Mth<T>::to_fixed(U, A.scale) : 0;
        if (!aggregate) {
            if (valid) {
                atomicAdd(dst + e, (unsigned long long)qi);
                atomicAdd(dst + e + A.plane, (unsigned long long)qq);
                atomicAdd(dst + e + 2 * A.plane, (unsigned long long)qu);
            }
            return;
        }
        while (leaders) {
            const int l = __ffs(leaders) - 1;
            const unsigned grp = __shfl_sync(FULL_MASK, peers, l);
            const bool in = (grp >> lane) & 1u;
            long long a = in ? qi : 0, b = in ? qq : 0, c = in ? qu : 0;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                a += __shfl_xor_sync(FULL_MASK, a, o);
                b += __shfl_xor_sync(FULL_MASK, b, o);
                c += __shfl_xor_sync(FULL_MASK, c, o);
            }
            if (lane == l) {
                atomicAdd(dst + e, (unsigned long long)a);
                atomicAdd(dst + e + A.plane, (unsigned long long)b);
                atomicAdd(dst + e + 2 * A.plane, (unsigned long long)c);
            }
            leaders &= leaders - 1u;
        }
    } else {
        double *dst = (double *)A.ptr;
        if (!aggregate) {
            if (valid) {
                atomicAdd(dst + e, (double)I);
                atomicAdd(dst + e + A.plane, (double)Q);
                atomicAdd(dst + e + 2 * A.plane, (double)U);
            }
            return;
        }
        while (leaders) {
            const int l = __ffs(leaders) - 1;
            const unsigned grp = __shfl_sync(FULL_MASK, peers, l);
            const bool in = (grp >> lane) & 1u;
            double a = in ? (double)I : 0.0, b = in ? (double)Q : 0.0, c = in ? (double)U : 0.0;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                a += __shfl_xor_sync(FULL_MASK, a, o);
                b += __shfl_xor_sync(FULL_MASK, b, o);
                c += __shfl_xor_sync(FULL_MASK, c, o);
            }
            if (lane == l) {
                atomicAdd(dst + e, a);
                atomicAdd(dst + e + A.plane, b);
                atomicAdd(dst + e + 2 * A.plane, c);
            }
            leaders &= leaders - 1u;
        }
    }
}

// Bin a peel-off contribution at sky (x, y) of observer O into image img of the image
// stack that starts `stack` values into the accumulator (Sec. 3.6).  Must be called
// by all 32 lanes.
template <class T>
__device__ __forceinline__ void splat(const ObsP<T> &O, const AccumP &acc, size_t stack, bool valid, int img, T x, T y,
                                      const T S[3])
{
    const size_t img_base = stack + (size_t)img * 3 * acc.plane;
    if (O.splat == QMCRT_SPLAT_NEAREST) {
        const T fx = Mth<T>::floor_((x + O.hw) * O.pix_x);
        const T fy = Mth<T>::floor_((y + O.hw) * O.pix_y);
        const bool in = valid && fx >= T(0) && fx < T(O.nx) && fy >= T(0) && fy < T(O.ny);
        const size_t e = in ? img_base + (size_t)((int)fy * O.nx + (int)fx) : 0;
        deposit<T>(acc, in, e, S[0], S[1], S[2]);
        return;
    }
    const T fx = (x + O.hw) * O.pix_x - T(0.5);
    const T fy = (y + O.hw) * O.pix_y - T(0.5);
    const T x0 = Mth<T>::floor_(fx), y0 = Mth<T>::floor_(fy);
    const T ax = fx - x0, ay = fy - y0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int dx = q & 1, dy = q >> 1;
        const T ix = x0 + T(dx), iy = y0 + T(dy);
        const bool in = valid && ix >= T(0) && ix < T(O.nx) && iy >= T(0) && iy < T(O.ny);
        const T w = (dx ? ax : T(1) - ax) * (dy ? ay : T(1) - ay);
        const size_t e = in ? img_base + (size_t)((int)iy * O.nx + (int)ix) : 0;
        deposit<T>(acc, in, e, w * S[0], w * S[1], w * S[2]);
    }
}

template <class T>
__device__ __forceinline__ void splat(const TraceP<T> &P, bool valid, int img, T x, T y, const T S[3])
{
    splat(P.obs, P.acc, 0, valid, img, x, y, S);
}

}  // namespace qmcrt

// qmcrt_tail.cu -- qmcrt_tail_map: for one observer direction k, an upper bound per grid
// cell on the optical depth still ahead of a peel-off walk (Sec. 3.6: every peel-off of a
// trace runs along k to the edge of the grid).  Beyond the dense parts of a medium most of
// such a walk crosses cells whose depth cannot matter (the tenuous atmosphere of a disk,
// empty corners of the box); the map lets the walk stop there, leaving out at most the
// caller's tolerance.
//
// Blocks of TAIL_BLOCK^3 cells hold the largest value of their cells (K_b).  Slabs of
// blocks are taken across the axis a of largest |k_a| / h_a.  Within one slab the walk
// crosses at most TAIL_BLOCK cells along a, so along another axis b it moves by at most
// TAIL_BLOCK (h_a |k_b|) / (h_b |k_a|) <= TAIL_BLOCK cells, one more where its starting
// point lies just below a face and one more for the rounding of near-simultaneous
// crossings: from any cell of a block it stays within nlat_b blocks along b (3 for a moving
// axis, fewer for a slow one, 1 where k_b = 0), and it enters the next slab within them.
// A ray from block C therefore gathers at most
//   B(C) = (TAIL_BLOCK h_a / |k_a|) max K_b(lateral blocks of C's slab)
//          + max B(the same lateral blocks of the next slab),
// summed from the slab k leaves through, with every operation rounded up.
#include <algorithm>
#include <cmath>

#include "qmcrt.h"
#include "qmcrt_internal.h"

namespace qmcrt {

namespace {

struct TailGeom {
    int nb[3];       // blocks per axis
    int a, b, c;     // slab axis and the two lateral axes
    int sa, sb, sc;  // the direction's signs along them (0: no component)
    int lb, lc;      // lateral blocks a ray from one block can reach along b, c (offsets 0 .. l-1)
    long long ta, tb, tc;  // block-index steps along a, b, c
    int na, nbb, nbc;      // blocks along a, b, c
    float path;      // longest path through one slab, rounded up
};

__device__ __forceinline__ long long block_index(const int nb[3], int x, int y, int z)
{
    return ((long long)z * nb[1] + y) * nb[0] + x;
}

// K_b: the largest value of each block's cells (the padded grid holds +0 for empty cells
// and -0 in the padding; neither raises the maximum).
__global__ void __launch_bounds__(256) k_tail_block_max(const float *__restrict__ K, int nx, int ny, int nz, int pad,
                                                        TailGeom g, float *__restrict__ Kb)
{
    const long long px = nx + 2 * pad, py = ny + 2 * pad;
    const long long blocks = (long long)g.nb[0] * g.nb[1] * g.nb[2];
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < blocks;
         q += (long long)gridDim.x * blockDim.x) {
        const int bx = (int)(q % g.nb[0]), by = (int)((q / g.nb[0]) % g.nb[1]),
                  bz = (int)(q / ((long long)g.nb[0] * g.nb[1]));
        float m = 0.0f;
        for (int z = bz * TAIL_BLOCK; z < min(nz, (bz + 1) * TAIL_BLOCK); ++z)
            for (int y = by * TAIL_BLOCK; y < min(ny, (by + 1) * TAIL_BLOCK); ++y)
                for (int x = bx * TAIL_BLOCK; x < min(nx, (bx + 1) * TAIL_BLOCK); ++x) {
                    const float v = __ldg(K + ((z + pad) * py + (y + pad)) * px + (x + pad));
                    if (v > m) m = v;
                }
        Kb[q] = m;
    }
}

// The slab recurrence, one block of threads: slab after slab against the direction, every
// block of a slab in parallel.
__global__ void __launch_bounds__(1024) k_tail_slabs(const float *__restrict__ Kb, TailGeom g, float *__restrict__ Bb)
{
    const int na = g.na, nbb = g.nbb, nbc = g.nbc;
    const int per_slab = nbb * nbc;
    for (int step = 0; step < na; ++step) {
        const int j = g.sa > 0 ? na - 1 - step : step;  // the exit side first
        const int jn = j + g.sa;                          // the slab a ray from slab j enters next
        for (int t = threadIdx.x; t < per_slab; t += blockDim.x) {
            const int ib = t % nbb, ic = t / nbb;
            float kmax = 0.0f, nmax = 0.0f;
            for (int ob = 0; ob < g.lb; ++ob) {
                const int qb = ib + g.sb * ob;
                if (qb < 0 || qb >= nbb) continue;
                for (int oc = 0; oc < g.lc; ++oc) {
                    const int qc = ic + g.sc * oc;
                    if (qc < 0 || qc >= nbc) continue;
                    const long long lat = qb * g.tb + qc * g.tc;
                    kmax = fmaxf(kmax, Kb[j * g.ta + lat]);
                    if (jn >= 0 && jn < na) nmax = fmaxf(nmax, Bb[jn * g.ta + lat]);
                }
            }
            Bb[j * g.ta + ib * g.tb + ic * g.tc] = __fadd_ru(__fmul_ru(kmax, g.path), nmax);
        }
        __syncthreads();
    }
}

// Codes of the padded grid's cells: c = (biased exponent of B, at least 1) + 24, so that
// B < 2^(c - 150); 0 for B = 0 and for the padding; 255 above 2^104 or not finite.
__global__ void __launch_bounds__(256) k_tail_expand(const float *__restrict__ Bb, int nx, int ny, int nz, int pad,
                                                     TailGeom g, uint8_t *__restrict__ map)
{
    const long long px = nx + 2 * pad, py = ny + 2 * pad, pz = nz + 2 * pad;
    const long long cells = px * py * pz;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < cells;
         e += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(e % px) - pad, y = (int)((e / px) % py) - pad, z = (int)(e / (px * py)) - pad;
        uint8_t code = 0;
        if (x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz) {
            const float B = Bb[block_index(g.nb, x / TAIL_BLOCK, y / TAIL_BLOCK, z / TAIL_BLOCK)];
            if (!(B <= 3.0e38f)) {
                code = 255;
            } else if (B > 0.0f) {
                const int E = (int)((__float_as_uint(B) >> 23) & 0xffu);
                const int c = max(E, 1) + 24;
                code = (uint8_t)(c > 254 ? 255 : c);
            }
        }
        map[e] = code;
    }
}

int blocks_of(int n) { return (n + TAIL_BLOCK - 1) / TAIL_BLOCK; }

uint64_t aligned(uint64_t bytes) { return (bytes + 255) & ~255ull; }

}  // namespace

uint64_t tail_workspace_bytes(int nx, int ny, int nz)
{
    const uint64_t blocks = (uint64_t)blocks_of(nx) * blocks_of(ny) * blocks_of(nz);
    return 2 * aligned(blocks * sizeof(float));
}

cudaError_t launch_tail_map(const float *k_padded, int nx, int ny, int nz, int pad, const double lo[3],
                            const double hi[3], const double dir[3], uint8_t *map, void *ws, cudaStream_t s)
{
    TailGeom g;
    const int n[3] = {nx, ny, nz};
    double h[3], speed[3];
    for (int q = 0; q < 3; ++q) {
        g.nb[q] = blocks_of(n[q]);
        h[q] = (hi[q] - lo[q]) / n[q];
        speed[q] = std::fabs(dir[q]) / h[q];  // cells crossed per unit path
    }
    g.a = 0;
    for (int q = 1; q < 3; ++q)
        if (speed[q] > speed[g.a]) g.a = q;
    g.b = g.a == 0 ? 1 : 0;
    g.c = g.a == 2 ? 1 : 2;
    auto sgn = [](double v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); };
    const long long step[3] = {1, g.nb[0], (long long)g.nb[0] * g.nb[1]};
    g.na = g.nb[g.a];
    g.nbb = g.nb[g.b];
    g.nbc = g.nb[g.c];
    g.ta = step[g.a];
    g.tb = step[g.b];
    g.tc = step[g.c];
    g.sa = sgn(dir[g.a]);
    g.sb = sgn(dir[g.b]);
    g.sc = sgn(dir[g.c]);
    auto lateral = [&](int q) {
        if (dir[q] == 0.0) return 1;
        const double r = speed[q] / speed[g.a] * (1.0 + 1e-9);  // <= 1 by the choice of a
        const int reach = (TAIL_BLOCK - 1) + (int)std::floor(TAIL_BLOCK * r) + 2;  // farthest cell offset
        return 1 + reach / TAIL_BLOCK;
    };
    g.lb = lateral(g.b);
    g.lc = lateral(g.c);
    const double path = TAIL_BLOCK * h[g.a] / std::fabs(dir[g.a]) * (1.0 + 1e-6);
    g.path = std::nextafter((float)path, 3.0e38f);
    float *Kb = (float *)ws;
    const uint64_t blocks = (uint64_t)g.nb[0] * g.nb[1] * g.nb[2];
    float *Bb = (float *)((char *)ws + aligned(blocks * sizeof(float)));
    const unsigned bgrid = (unsigned)std::min<uint64_t>((blocks + 255) / 256, 152ull * 16);
    k_tail_block_max<<<bgrid, 256, 0, s>>>(k_padded, nx, ny, nz, pad, g, Kb);
    k_tail_slabs<<<1, 1024, 0, s>>>(Kb, g, Bb);
    const uint64_t cells = (uint64_t)(nx + 2 * pad) * (ny + 2 * pad) * (nz + 2 * pad);
    const unsigned egrid = (unsigned)std::min<uint64_t>((cells + 255) / 256, 152ull * 32);
    k_tail_expand<<<egrid, 256, 0, s>>>(Bb, nx, ny, nz, pad, g, map);
    return cudaGetLastError();
}

}  // namespace qmcrt

// mg.cu -- geometric multigrid V-cycle used as the preconditioner of CG for the pressure Poisson
// equation (Eq. poisson).  The paper solves it with BiCGStab or red-black SOR; red-black Gauss-Seidel
// is the smoother here.
//
// Level 0 is the fine grid: the conductance of a link is 1 when its face is uncut and inside the
// domain (or across a periodic seam), 0 otherwise, and an outflow face adds 2 to the diagonal (ghost
// -p).  A position of level l >= 1 is a block of 2x2x2 positions of level l - 1, and its unknowns are
// the connected parts of that block: unknowns of level l - 1 inside the block joined by their links
// inside the block.  So an aggregate never spans a wall -- a block cut in two by a thin plate gives
// two coarse unknowns, and a sealed pocket (the inside of a closed part of the soup) never merges
// with its surroundings on any level.  (Aggregating whole blocks instead joins the two sides of every
// wall on the coarse levels; on a dirty multi-part soup that costs several times the iterations.)
// With piecewise-constant prolongation P and restriction R = P^T the Galerkin coarse operator R A P
// is again a weighted graph Laplacian plus the outflow terms: the conductance between two coarse
// unknowns is the sum of the fine conductances between their aggregates.  Links join only
// face-neighbouring positions, so the parity of a position two-colours every level.  The V-cycle
// (pre-smoothing red then black, post-smoothing black then red, the coarse correction scaled by
// omega < 2, symmetric sweeps on the coarsest level) is a symmetric operator, as CG requires.
//
// Equations are solved in the unscaled form  sum_links g (x_N - x_P) - d x_P = dx^2 r.
#include <cooperative_groups.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <mutex>
#include <type_traits>

#include "scan.cuh"
#include "solver.cuh"

namespace cg = cooperative_groups;

namespace {

#define MG_TAIL_CTAS 8          // portable cluster size
#define MG_TAIL_MAX (1LL << 13) // levels with at most this many unknowns run in the one-launch tail
#define MG_COARSE_TARGET 1024   // coarsening stops at this many unknowns (or one position)
#define MG_MAXCH 64             // unknowns of a block whose internal links are followed (more: singletons)
#define MG_MAXE 256             // internal links followed per block
#define MG_MAXL 64              // distinct neighbours of a coarse unknown (more: the level is dropped)
#define MG_L1L 24               // level 1: a 2x2x2 block has at most 24 links leaving it

struct MGTail {
    MGLev lev[IBM_MG_MAXLEV];
    int first, nlev, sweeps, coarse_sweeps;
    double omega;
};

__device__ __forceinline__ unsigned flags_at(const Dom& D, long long P) { return D.flags ? (unsigned)D.flags[P] : 0u; }


// Conductances and Dirichlet term of a fine (level 0) cell, links in the order x-, x+, y-, y+, z-, z+.
__device__ __forceinline__ void fine_links(const Dom& D, long long P, const int x[3], unsigned fl, float g[6],
                                           long long off[6], float& d) {
    d = 0.f;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        const int a = b >> 1, s = (b & 1) ? 1 : -1;
        long long o = 0;
        const bool in = nb_offset(D, a, s, x[a], o);
        off[b] = o;
        g[b] = (!(fl & (1u << b)) && in) ? 1.f : 0.f;
        if (!in && D.bc[b] == IBM_BC_OUTFLOW) d += 2.f;
    }
}


// Cell coordinates from a linear index (grids hold fewer than 2^31 cells: 32-bit division).
__device__ __forceinline__ void coords3(long long c, int nx, int ny, int x[3]) {
    const unsigned u = (unsigned)c, unx = (unsigned)nx, uny = (unsigned)ny;
    const unsigned r = u / unx;
    x[0] = (int)(u - r * unx);
    const unsigned z = r / uny;
    x[1] = (int)(r - z * uny);
    x[2] = (int)z;
}


__device__ __forceinline__ long long pos_index(const MGLev& L, const int X[3]) {
    return X[0] + (long long)L.px * (X[1] + (long long)L.py * X[2]);
}

// ---- fine-grid smoothing ----------------------------------------------------------------------

// Gauss-Seidel value of a fine cell:  z_P = (sum_links g z_N - scale r_P) / dg, with the interior
// fast path (six uncut links, dg = 6).  Returns false for an isolated cell (dg = 0).
template <class T>
__device__ __forceinline__ T gs_value(const Dom& D, const T* __restrict__ r, const T* z, T scale, long long P, int i,
                                      int j, int k, bool zero) {
    const unsigned fl = flags_at(D, P);
    if (fl == 0u && i > 0 && i < D.nx - 1 && j > 0 && j < D.ny - 1 && k > 0 && k < D.nz - 1) {
        const T s = zero ? (T)0
                         : ((z[P - 1] + z[P + 1]) + (z[P - D.sy] + z[P + D.sy])) + (z[P - D.sz] + z[P + D.sz]);
        return (s - scale * r[P]) * (T)(1.0 / 6.0);
    }
    const int x[3] = {i, j, k};
    float g[6], d;
    long long off[6];
    fine_links(D, P, x, fl, g, off, d);
    const float dg = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + d;
    if (dg == 0.f) return (T)0;
    T s = 0;
    if (!zero) {
#pragma unroll
        for (int b = 0; b < 6; ++b)
            if (g[b] != 0.f) s += z[P + off[b]];
    }
    return (s - scale * r[P]) / (T)dg;
}

// One red-black Gauss-Seidel pass of colour `col` on level 0 for  A^ z = scale * r.  Each thread takes
// IBM_KU pairs of planes of one (i, j) column and updates the cell of colour `col` in each pair.
// With `zero` the iterate is taken as 0 (first pass of a V-cycle) and the other cell of each pair is
// cleared.
template <class T>
__global__ void __launch_bounds__(256) k_mg_smooth0(Dom D, const T* __restrict__ r, T* __restrict__ z, T scale,
                                                    int col, int zero, const SolveScal* sc) {
    if (sc->done) return;
    const int i = blockIdx.x * IBM_TX + threadIdx.x, j = blockIdx.y * IBM_TY + threadIdx.y;
    if (i >= D.nx || j >= D.ny) return;
    const int kb = blockIdx.z * (2 * IBM_KU);
    const int par = (col + i + j) & 1;
#pragma unroll
    for (int u = 0; u < IBM_KU; ++u) {
        const int k = kb + 2 * u + par;
        const long long P = i + (long long)D.sy * j + D.sz * k;
        if (k < D.nz) z[P] = gs_value<T>(D, r, z, scale, P, i, j, k, zero != 0);
        if (zero) {
            const int k2 = kb + 2 * u + (par ^ 1);
            if (k2 < D.nz) z[i + (long long)D.sy * j + D.sz * k2] = (T)0;
        }
    }
}

// Last pass of the V-cycle on level 0 (colour 0) fused with rho = (r, z) over both colours.
template <class T>
__global__ void __launch_bounds__(256) k_mg_final0(Dom D, const T* __restrict__ r, T* __restrict__ z, T scale,
                                                   SolveScal* sc, double* partials, unsigned* counter) {
    if (sc->done) return;
    const int i = blockIdx.x * IBM_TX + threadIdx.x, j = blockIdx.y * IBM_TY + threadIdx.y;
    const bool active = i < D.nx && j < D.ny;
    const int kb = blockIdx.z * (2 * IBM_KU);
    const int par = (i + j) & 1;                 // plane offset of the colour-0 cell in each pair
    T part = 0;
    if (active) {
#pragma unroll
        for (int u = 0; u < IBM_KU; ++u) {
            const int k = kb + 2 * u + par, k2 = kb + 2 * u + (par ^ 1);
            if (k < D.nz) {
                const long long P = i + (long long)D.sy * j + D.sz * k;
                const T zv = gs_value<T>(D, r, z, scale, P, i, j, k, false);
                z[P] = zv;
                part += r[P] * zv;
            }
            if (k2 < D.nz) {
                const long long P2 = i + (long long)D.sy * j + D.sz * k2;
                part += r[P2] * z[P2];
            }
        }
    }
    decltype(part) acc[1] = {part};
    grid_reduce<1>(acc, partials, counter, [&](double* t) {
        sc->rz_old = sc->rz;
        sc->rz = t[0];
    });
}

// ---- parts of a block -----------------------------------------------------------------------------

// Flags of the 2x2x2 fine cells below level-1 position X (cell m = di + 2 dj + 4 dk); bit m of the
// result says that cell m lies inside the domain.  Out-of-domain cells get flags 0.
__device__ __forceinline__ unsigned block_flags(const Dom& D, const int X[3], unsigned (&fl)[8], long long (&P)[8]) {
    unsigned in = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int x = 2 * X[0] + (m & 1), y = 2 * X[1] + ((m >> 1) & 1), z = 2 * X[2] + (m >> 2);
        const bool ok = x < D.nx && y < D.ny && z < D.nz;
        P[m] = ok ? x + (long long)D.sy * y + D.sz * z : 0;
        fl[m] = ok ? flags_at(D, P[m]) : 0u;
        in |= (ok ? 1u : 0u) << m;
    }
    return in;
}

// Connected parts of a fine block: two in-domain cells of the block are joined when the face between
// them is uncut, or when their axis is periodic with only two cells (the seam joins them too).
// part[m] = the part of cell m, parts numbered in the order of their lowest cell; returns the count.
__device__ __forceinline__ int fine_parts(const Dom& D, const unsigned (&fl)[8], unsigned in, int (&part)[8]) {
    const unsigned cut = ((fl[0] | fl[2] | fl[4] | fl[6]) & 2u) | ((fl[0] | fl[1] | fl[4] | fl[5]) & 8u) |
                         ((fl[0] | fl[1] | fl[2] | fl[3]) & 32u);
    if (in == 0xffu && cut == 0u) {
#pragma unroll
        for (int m = 0; m < 8; ++m) part[m] = 0;
        return 1;
    }
    const bool seam[3] = {D.bc[0] == IBM_BC_PERIODIC && D.nx == 2, D.bc[2] == IBM_BC_PERIODIC && D.ny == 2,
                          D.bc[4] == IBM_BC_PERIODIC && D.nz == 2};
    int lab[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) lab[m] = m;
    // minimum-label propagation; a path through the block has at most 7 links
    for (int it = 0; it < 8; ++it) {
        bool changed = false;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                if (m & (1 << a)) continue;
                const int h = m | (1 << a);
                if (!((in >> m) & 1u) || !((in >> h) & 1u)) continue;
                if ((fl[m] & (2u << (2 * a))) && !seam[a]) continue;
                const int lo = lab[m] < lab[h] ? lab[m] : lab[h];
                if (lab[m] != lo || lab[h] != lo) {
                    lab[m] = lo;
                    lab[h] = lo;
                    changed = true;
                }
            }
        if (!changed) break;
    }
    unsigned roots = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m)
        if (((in >> m) & 1u) && lab[m] == m) roots |= 1u << m;
#pragma unroll
    for (int m = 0; m < 8; ++m) part[m] = __popc(roots & ((1u << lab[m]) - 1u));
    return __popc(roots);
}

// ---- fused fine-grid passes: all four red-black half-sweeps of a smoothing phase in one pass ------
//
// A block owns an (x, y) tile of FT_TX x FT_TY cells and marches along z over a chunk of planes.  It
// keeps, for the tile plus a 4-cell halo, a ring of FT_NS planes of r, flags and z in shared memory;
// the planes arrive by TMA (one elected thread issues cp.async.bulk.tensor loads one plane ahead; an
// mbarrier per ring slot carries the byte count).  Step t takes plane t; the half-sweeps run at planes
// t, t-1, t-2, t-3 (each needs its neighbours after the previous half-sweep, one plane and one halo
// cell further out), so that after step t plane t-3 (pre-smoothing) or t-4 (post-smoothing) is final.
// The halo shrinks by one cell per half-sweep, so the tile's own cells see exactly the values the
// four separate passes compute.  Pre-smoothing starts from z = 0 (only r and the flags are read) and
// ends with the residual and its restriction to level 1; post-smoothing reads z and ends with the
// (r, z) product of the CG iteration.  Neighbouring chunks recompute each other's edge planes but
// only write their own.

#define FT_TX 48                    // tile along x (a multiple of 16: the flags box starts 16 cells left)
#ifndef FT_TY
#define FT_TY 16                    // tile along y (even: level-1 blocks are 2 x 2 x 2)
#endif
#ifndef FT_LA
#define FT_LA 2                     // planes loaded ahead of the one a step consumes
#endif
#define FT_H 4                      // halo
#define FT_RX (FT_TX + 2 * FT_H)    // r / z box along x (56 floats = 224 bytes)
#define FT_RY (FT_TY + 2 * FT_H)    // box along y
#define FT_FX (FT_TX + 32)          // flags box along x (80 bytes), starting 16 cells left of the tile
#define FT_FOFF 12                  // flags column of r/z column 0
#define FT_NS (6 + FT_LA)           // ring slots: planes t-5 .. t+FT_LA
#define FT_QX (FT_RX / 4)           // 4-cell quads per ring row
#define FT_NQ (FT_QX * FT_RY)       // quads of the ring plane
#define FT_NT (((FT_NQ + 31) / 32) * 32)   // threads: one quad each
#define FT_RBYTES (FT_RX * FT_RY * 4)
#define FT_FBYTES (FT_FX * FT_RY)
#define FT_FPAD (((FT_FBYTES + 127) / 128) * 128)
#define FT_SLOT (2 * FT_RBYTES + FT_FPAD)             // r | z | flags
#define FT_SMEM (FT_NS * FT_SLOT + 2 * FT_TX * FT_TY * 4 + 8 * FT_NS + 128)   // + alignment slack

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity, for at most about a second (clock cycles); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > 2000000000LL) return false;
    return true;
}
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

struct FTSmem {
    unsigned char* base;
    __device__ float* r(int s) const { return reinterpret_cast<float*>(base + s * FT_SLOT); }
    __device__ float* z(int s) const { return reinterpret_cast<float*>(base + s * FT_SLOT + FT_RBYTES); }
    __device__ const uint8_t* f(int s) const { return base + s * FT_SLOT + 2 * FT_RBYTES; }
    __device__ float* res(int parity) const { return reinterpret_cast<float*>(base + FT_NS * FT_SLOT) + parity * FT_TX * FT_TY; }
    __device__ uint64_t* bar(int s) const {
        return reinterpret_cast<uint64_t*>(base + FT_NS * FT_SLOT + 2 * FT_TX * FT_TY * 4) + s;
    }
};

struct FTPos {
    int x0, y0, gx0, gy0;   // tile origin; global coordinates of ring column / row 0
    int tlo;                // first plane loaded (ring slot 0, use 0)
};

__device__ __forceinline__ int ft_slot(const FTPos& P, int t) { return (t - P.tlo) % FT_NS; }
__device__ __forceinline__ unsigned ft_parity(const FTPos& P, int t) { return (unsigned)(((t - P.tlo) / FT_NS) & 1); }

// Issues the TMA loads of plane t (r and flags, and z when `withz`) into its slot, or, for a plane
// outside the domain, just completes the slot's phase.  One thread.
__device__ __forceinline__ void ft_issue(const Dom& D, const FTSmem& S, const FTPos& P, int t, bool withz,
                                         const CUtensorMap* tr, const CUtensorMap* tz, const CUtensorMap* tf) {
    const int s = ft_slot(P, t);
    uint64_t* b = S.bar(s);
    if (t < 0 || t >= D.nz) {
        mbar_arrive(b);
        return;
    }
    mbar_expect_tx(b, (withz ? 2 : 1) * FT_RBYTES + FT_FBYTES);
    tma_load3(S.r(s), tr, P.gx0, P.gy0, t, b);
    if (withz) tma_load3(S.z(s), tz, P.gx0, P.gy0, t, b);
    tma_load3((void*)S.f(s), tf, P.gx0 - FT_FOFF, P.gy0, t, b);
}

// Per-thread cells: thread q < FT_NQ owns the quad of 4 consecutive ring cells (ry, 4 qx .. 4 qx + 3),
// fixed for the whole march; the quads line up with the tile (its x-range starts at ring column 4).
// Cell masks (bit m for cell m): in the domain; interior (its in-plane neighbours are in the domain,
// which the plain form of the update needs); within distance e of the tile (the half-sweeps of halo
// e update those), for e = 0 .. 3.
struct FTQuad {
    int c;          // ring index of cell 0
    int f;          // flags-ring index of cell 0 (a multiple of 4)
    int gx, gy;     // global coordinates of cell 0
    int par;        // (gx + gy) & 1
    int tile;       // index of cell 0 in the tile (tile quads), -1 otherwise
    unsigned dom, inter, halo;   // halo: 4 bits per e
};

__device__ __forceinline__ FTQuad ft_quad(const Dom& D, const FTPos& P, int q) {
    FTQuad a;
    a.c = a.f = a.gx = a.gy = a.par = 0;
    a.tile = -1;
    a.dom = a.inter = a.halo = 0u;
    if (q >= FT_NQ) return a;
    const int ry = q / FT_QX, rx = 4 * (q % FT_QX);
    a.c = ry * FT_RX + rx;
    a.f = ry * FT_FX + rx + FT_FOFF;
    a.gx = P.gx0 + rx;
    a.gy = P.gy0 + ry;
    a.par = (a.gx + a.gy) & 1;
    const int dy = max(max(FT_H - ry, ry - (FT_H + FT_TY - 1)), 0);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int x = rx + m, gx = a.gx + m;
        const int dx = max(max(FT_H - x, x - (FT_H + FT_TX - 1)), 0);
        const bool in = gx >= 0 && gx < D.nx && a.gy >= 0 && a.gy < D.ny;
        const bool inter = gx > 0 && gx < D.nx - 1 && a.gy > 0 && a.gy < D.ny - 1;
        const int d = max(dx, dy);
        a.dom |= (in ? 1u : 0u) << m;
        a.inter |= (inter ? 1u : 0u) << m;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (in && d <= e) a.halo |= 1u << (4 * e + m);
    }
    if (dy == 0 && rx >= FT_H && rx < FT_H + FT_TX) a.tile = (ry - FT_H) * FT_TX + (rx - FT_H);
    return a;
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float f4e(const float4& v, int m) { return m == 0 ? v.x : (m == 1 ? v.y : (m == 2 ? v.z : v.w)); }

// Gauss-Seidel value of a ring cell in the generic case (a cut link or a domain face next to it):
// (sum of z over the open links - sr) / dg, dg = open links + the outflow terms.
__device__ __forceinline__ float ft_gs_generic(const Dom& D, int c, int gx, int gy, int t, unsigned fl, float sr,
                                               const float* zm, const float* zc, const float* zp) {
    const int g[3] = {gx, gy, t}, n[3] = {D.nx, D.ny, D.nz};
    float s = 0.f, dg = 0.f;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        const int a = b >> 1, sd = (b & 1) ? 1 : -1;
        const bool in = g[a] + sd >= 0 && g[a] + sd < n[a];
        if (in && !(fl & (1u << b))) {
            dg += 1.f;
            s += a == 0 ? zc[c + sd] : (a == 1 ? zc[c + sd * FT_RX] : (sd < 0 ? zm[c] : zp[c]));
        } else if (!in && D.bc[b] == IBM_BC_OUTFLOW) {
            dg += 2.f;
        }
    }
    return dg == 0.f ? 0.f : (s - sr) / dg;
}

// A z at a ring cell in the generic case, unscaled form  sum_open (z_N - z_P) - d z_P.
__device__ __forceinline__ float ft_az_generic(const Dom& D, int c, int gx, int gy, int t, unsigned fl,
                                               const float* zm, const float* zc, const float* zp) {
    const float zP = zc[c];
    const int g[3] = {gx, gy, t}, n[3] = {D.nx, D.ny, D.nz};
    float s = 0.f;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        const int a = b >> 1, sd = (b & 1) ? 1 : -1;
        const bool in = g[a] + sd >= 0 && g[a] + sd < n[a];
        if (in && !(fl & (1u << b)))
            s += (a == 0 ? zc[c + sd] : (a == 1 ? zc[c + sd * FT_RX] : (sd < 0 ? zm[c] : zp[c]))) - zP;
        else if (!in && D.bc[b] == IBM_BC_OUTFLOW)
            s += -zP - zP;
    }
    return s;
}

// The ring planes of one step: slot of plane t - k for k = 0 .. 5 (one modulo per step).
struct FTRing {
    int sl[6];
    __device__ __forceinline__ FTRing(const FTPos& P, int t) {
        sl[0] = (t - P.tlo) % FT_NS;
#pragma unroll
        for (int k = 1; k < 6; ++k) sl[k] = sl[k - 1] == 0 ? FT_NS - 1 : sl[k - 1] - 1;
    }
};

// One half-sweep of colour `col` on plane t = step - k (ring slot R.sl[k]) over the thread's cells
// within `e` of the tile.  The k-th half-sweep of a pass runs only on planes t >= tlo + k: below that
// its inputs (the previous half-sweep on plane t - 1) were never formed in this block, and nothing it
// would produce is needed.  The quad's two cells of colour col are d and d + 2; a cell with no cut
// link whose neighbours lie in the domain takes the six-neighbour sum from 16-byte loads.
__device__ __forceinline__ void ft_half_sweep(const Dom& D, const FTSmem& S, const FTPos& P, const FTQuad& Q,
                                              const FTRing& R, int k, int t, int col, int e, float scale, int kind) {
    if (t < P.tlo + kind || t < 0 || t >= D.nz) return;     // the same for the whole block
    const int d = (col + Q.par + t) & 1;
    const unsigned act = (Q.halo >> (4 * e)) & (5u << d);
    float* zc = S.z(R.sl[k]);
    const float* zm = S.z(R.sl[k + 1]);           // planes outside the domain are never read (links closed)
    const float* zp = S.z(k > 0 ? R.sl[k - 1] : R.sl[k]);
    const float* rc = S.r(R.sl[k]);
    const unsigned fl4 = *reinterpret_cast<const unsigned*>(S.f(R.sl[k]) + Q.f);
    const bool tint = t > 0 && t < D.nz - 1;
    const unsigned fa = (fl4 >> (8 * d)) & 0xffu, fb = (fl4 >> (8 * (d + 2))) & 0xffu;
    const bool onA = (act >> d) & 1u, onB = (act >> (d + 2)) & 1u;
    const bool plainA = fa == 0u && tint && ((Q.inter >> d) & 1u);
    const bool plainB = fb == 0u && tint && ((Q.inter >> (d + 2)) & 1u);
    // a warp without a generic cell skips the generic form altogether
    const bool generic = __any_sync(0xffffffffu, (onA && !plainA) || (onB && !plainB));
    if (!act) return;
    const int c = Q.c;
    const float4 z4 = lds4(zc + c), r4 = lds4(rc + c);
    const float4 ym = lds4(zc + c - FT_RX), yp = lds4(zc + c + FT_RX);
    const float4 zl = lds4(zm + c), zu = lds4(zp + c);
    const bool odd = d != 0;
    // cells A = d and B = d + 2 and their x-neighbours (the cell left of the quad and the one right of
    // it lie in the same ring row: an active quad is never in the ring's first or last column)
    const float left = zc[c - 1], right = zc[c + 4];
    const float xa_l = odd ? z4.x : left, xa_r = odd ? z4.z : z4.y;
    const float xb_l = xa_r, xb_r = odd ? right : z4.w;
    const float sa = ((xa_l + xa_r) + ((odd ? ym.y : ym.x) + (odd ? yp.y : yp.x))) + ((odd ? zl.y : zl.x) + (odd ? zu.y : zu.x));
    const float sb = ((xb_l + xb_r) + ((odd ? ym.w : ym.z) + (odd ? yp.w : yp.z))) + ((odd ? zl.w : zl.z) + (odd ? zu.w : zu.z));
    const float ra = odd ? r4.y : r4.x, rb = odd ? r4.w : r4.z;
    float va = (sa - scale * ra) * (1.f / 6.f), vb = (sb - scale * rb) * (1.f / 6.f);
    if (generic) {
        if (onA && !plainA) va = ft_gs_generic(D, c + d, Q.gx + d, Q.gy, t, fa, scale * ra, zm, zc, zp);
        if (onB && !plainB) vb = ft_gs_generic(D, c + d + 2, Q.gx + d + 2, Q.gy, t, fb, scale * rb, zm, zc, zp);
    }
    if (onA) zc[c + d] = va;
    if (onB) zc[c + d + 2] = vb;
}

// Pre-smoothing (from z = 0, colours 0, 1, 0, 1) + restriction of  scale r - A z  to the parts of the
// level-1 blocks.  Writes z on its chunk's planes [k0, k1) and b_1.
__global__ void __launch_bounds__(FT_NT, 2) k_mg_pre_fused(Dom D, float* __restrict__ z, float scale, MGLev C1,
                                                          int kchunk, SolveScal* sc,
                                                          const __grid_constant__ CUtensorMap tmr,
                                                          const __grid_constant__ CUtensorMap tmf) {
    if (sc->done) return;
    extern __shared__ __align__(128) unsigned char ft_smem[];
    __shared__ int abort_flag;
    FTSmem S{reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(ft_smem) + 127) & ~(uintptr_t)127)};
    FTPos P;
    P.x0 = blockIdx.x * FT_TX;
    P.y0 = blockIdx.y * FT_TY;
    P.gx0 = P.x0 - FT_H;
    P.gy0 = P.y0 - FT_H;
    const int k0 = blockIdx.z * kchunk, k1 = min(D.nz, k0 + kchunk);
    P.tlo = k0 - 4;
    const int thi = k1 + 3;
    float* __restrict__ b1 = (float*)C1.b;
    const FTQuad Q = ft_quad(D, P, threadIdx.x);
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < FT_NS; ++s) mbar_init(S.bar(s), 1);
        fence_barrier_init();
    }
    __syncthreads();
    int issued = P.tlo - 1;
    if (threadIdx.x == 0)
        for (int u = P.tlo; u < P.tlo + FT_LA && u <= thi; ++u) {
            ft_issue(D, S, P, u, false, &tmr, nullptr, &tmf);
            issued = u;
        }
    for (int t = P.tlo; t <= thi; ++t) {
        if (threadIdx.x == 0) {
            if (t + FT_LA <= thi) {
                ft_issue(D, S, P, t + FT_LA, false, &tmr, nullptr, &tmf);
                issued = t + FT_LA;
            }
            if (!mbar_wait(S.bar(ft_slot(P, t)), ft_parity(P, t))) abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        const FTRing R(P, t);
        // h1 on plane t: z = -scale r / dg on colour 0, 0 on colour 1 (z = 0 before the first pass)
        if (t >= 0 && t < D.nz) {
            const int s = R.sl[0];
            const float4 r4 = lds4(S.r(s) + Q.c);
            const unsigned fl4 = *reinterpret_cast<const unsigned*>(S.f(s) + Q.f);
            const bool tint = t > 0 && t < D.nz - 1;
            unsigned on = 0u, gen = 0u;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const bool o = ((Q.dom >> m) & 1u) && !((Q.par + m + t) & 1);
                const bool plain = ((fl4 >> (8 * m)) & 0xffu) == 0u && tint && ((Q.inter >> m) & 1u);
                on |= (o ? 1u : 0u) << m;
                gen |= (o && !plain ? 1u : 0u) << m;
            }
            float v[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] = ((on >> m) & 1u) ? (0.f - scale * f4e(r4, m)) * (1.f / 6.f) : 0.f;
            if (__any_sync(0xffffffffu, gen != 0u)) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (!((gen >> m) & 1u)) continue;
                    const unsigned fl = (fl4 >> (8 * m)) & 0xffu;
                    const int g[3] = {Q.gx + m, Q.gy, t}, n[3] = {D.nx, D.ny, D.nz};
                    float dg = 0.f;
#pragma unroll
                    for (int b = 0; b < 6; ++b) {
                        const int a = b >> 1, sd = (b & 1) ? 1 : -1;
                        const bool in = g[a] + sd >= 0 && g[a] + sd < n[a];
                        if (in && !(fl & (1u << b))) dg += 1.f;
                        else if (!in && D.bc[b] == IBM_BC_OUTFLOW) dg += 2.f;
                    }
                    v[m] = dg == 0.f ? 0.f : (0.f - scale * f4e(r4, m)) / dg;
                }
            }
            if (threadIdx.x < FT_NQ)
                *reinterpret_cast<float4*>(S.z(s) + Q.c) = make_float4(v[0], v[1], v[2], v[3]);
        }
        __syncthreads();
        ft_half_sweep(D, S, P, Q, R, 1, t - 1, 1, 3, scale, 1);
        __syncthreads();
        ft_half_sweep(D, S, P, Q, R, 2, t - 2, 0, 2, scale, 2);
        __syncthreads();
        ft_half_sweep(D, S, P, Q, R, 3, t - 3, 1, 1, scale, 3);
        __syncthreads();
        // plane t-3 is final: store the tile; residual of plane t-4 (its neighbours are final)
        const int tw = t - 3, tr = t - 4;
        if (tw >= k0 && tw < k1 && Q.tile >= 0 && Q.dom == 0xfu)
            *reinterpret_cast<float4*>(z + Q.gx + (long long)D.sy * Q.gy + D.sz * tw) = lds4(S.z(R.sl[3]) + Q.c);
        if (tr >= k0 && tr < k1) {
            {
                const int s = R.sl[4];
                const float* zc = S.z(s);
                const float* zm = S.z(R.sl[5]);
                const float* zp = S.z(R.sl[3]);
                const int c = Q.c;
                const unsigned fl4 = *reinterpret_cast<const unsigned*>(S.f(s) + Q.f);
                const bool tint = tr > 0 && tr < D.nz - 1;
                const bool tq = Q.tile >= 0 && Q.dom != 0u;
                unsigned gen = 0u;
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (tq && !(((fl4 >> (8 * m)) & 0xffu) == 0u && tint && ((Q.inter >> m) & 1u))) gen |= 1u << m;
                // a warp without a generic cell skips the generic form altogether
                const bool generic = __any_sync(0xffffffffu, gen != 0u);
                if (Q.tile >= 0) {
                    float v[4] = {0.f, 0.f, 0.f, 0.f};
                    if (Q.dom) {
                        const float4 z4 = lds4(zc + c), r4 = lds4(S.r(s) + c);
                        const float4 ym = lds4(zc + c - FT_RX), yp = lds4(zc + c + FT_RX);
                        const float4 zl = lds4(zm + c), zu = lds4(zp + c);
                        const float left = zc[c - 1], right = zc[c + 4];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const float xm = m == 0 ? left : f4e(z4, m - 1);
                            const float xp = m == 3 ? right : f4e(z4, m + 1);
                            float az = ((xm + xp) + (f4e(ym, m) + f4e(yp, m))) + (f4e(zl, m) + f4e(zu, m)) - 6.f * f4e(z4, m);
                            if (generic && ((gen >> m) & 1u))
                                az = ft_az_generic(D, c + m, Q.gx + m, Q.gy, tr, (fl4 >> (8 * m)) & 0xffu, zm, zc, zp);
                            v[m] = scale * f4e(r4, m) - az;
                        }
                    }
                    *reinterpret_cast<float4*>(S.res(tr & 1) + Q.tile) = make_float4(v[0], v[1], v[2], v[3]);
                }
            }
            if ((tr & 1) || tr == D.nz - 1) {
                __syncthreads();
                // restriction: the level-1 blocks of planes (tr & ~1, tr | 1)
                const int ke = tr & ~1;
                const int Z = ke >> 1;
                const bool both = ke + 1 < D.nz;
                // tr odd: the pair is (tr - 1, tr) in slots 5, 4; tr even (the last plane of an odd count): tr alone
                const uint8_t* fe = S.f((tr & 1) ? R.sl[5] : R.sl[4]);
                const uint8_t* fo = both ? S.f(R.sl[4]) : fe;
                const float* re = S.res(0);
                const float* ro = S.res(1);
                for (int q = threadIdx.x; q < (FT_TX / 2) * (FT_TY / 2); q += FT_NT) {
                    const int bx = q % (FT_TX / 2), by = q / (FT_TX / 2);
                    const int X = (P.x0 >> 1) + bx, Y = (P.y0 >> 1) + by;
                    if (X >= C1.px || Y >= C1.py) continue;
                    const bool yok = 2 * Y + 1 < D.ny;           // x: nx is even, so both columns exist
                    unsigned fl[8];
                    float rv[8];
                    unsigned in = 0;
                    const int fi = (FT_H + 2 * by) * FT_FX + FT_H + 2 * bx + FT_FOFF;
                    const int ri = (2 * by) * FT_TX + 2 * bx;
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const int di = m & 1, dj = (m >> 1) & 1, dk = m >> 2;
                        const bool ok = (dj == 0 || yok) && (dk == 0 || both);
                        fl[m] = ok ? (unsigned)(dk ? fo : fe)[fi + dj * FT_FX + di] : 0u;
                        rv[m] = ok ? (dk ? ro : re)[ri + dj * FT_TX + di] : 0.f;
                        in |= (ok ? 1u : 0u) << m;
                    }
                    int part[8];
                    const int np = fine_parts(D, fl, in, part);
                    const int o = C1.off[X + (long long)C1.px * (Y + (long long)C1.py * Z)];
                    if (np == 1) {
                        b1[o] = ((rv[0] + rv[1]) + (rv[2] + rv[3])) + ((rv[4] + rv[5]) + (rv[6] + rv[7]));
                        continue;
                    }
                    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int m = 0; m < 8; ++m)
#pragma unroll
                        for (int s2 = 0; s2 < 8; ++s2) acc[s2] += part[m] == s2 ? rv[m] : 0.f;
#pragma unroll
                    for (int s2 = 0; s2 < 8; ++s2)
                        if (s2 < np) b1[o + s2] = acc[s2];
                }
            }
        }
        fence_proxy_async();
        __syncthreads();
    }
    if (abort_flag && threadIdx.x == 0) {
        // let the loads already issued land before the block's shared memory goes away
        for (int u = issued; u > issued - FT_NS && u >= P.tlo; --u) mbar_wait(S.bar(ft_slot(P, u)), ft_parity(P, u));
        atomicExch(&sc->dev_error, 1);
    }
}

// Post-smoothing (colours 1, 0, 1, 0) of the iterate the coarse correction left (read through the
// `tmz` map from an array this pass does not write), into z; then (r, z) over the grid:
// rz_old = rz, rz = (r, z).
__global__ void __launch_bounds__(FT_NT, 2) k_mg_post_fused(Dom D, float* __restrict__ z, float scale, int kchunk,
                                                           SolveScal* sc, double* partials, unsigned* counter,
                                                           const __grid_constant__ CUtensorMap tmr,
                                                           const __grid_constant__ CUtensorMap tmz,
                                                           const __grid_constant__ CUtensorMap tmf) {
    if (sc->done) return;
    extern __shared__ __align__(128) unsigned char ft_smem[];
    __shared__ int abort_flag;
    FTSmem S{reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(ft_smem) + 127) & ~(uintptr_t)127)};
    FTPos P;
    P.x0 = blockIdx.x * FT_TX;
    P.y0 = blockIdx.y * FT_TY;
    P.gx0 = P.x0 - FT_H;
    P.gy0 = P.y0 - FT_H;
    const int k0 = blockIdx.z * kchunk, k1 = min(D.nz, k0 + kchunk);
    P.tlo = k0 - 4;
    const int thi = k1 + 3;
    const FTQuad Q = ft_quad(D, P, threadIdx.x);
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < FT_NS; ++s) mbar_init(S.bar(s), 1);
        fence_barrier_init();
    }
    __syncthreads();
    int issued = P.tlo - 1;
    if (threadIdx.x == 0)
        for (int u = P.tlo; u < P.tlo + FT_LA && u <= thi; ++u) {
            ft_issue(D, S, P, u, true, &tmr, &tmz, &tmf);
            issued = u;
        }
    float part = 0.f;
    for (int t = P.tlo; t <= thi; ++t) {
        if (threadIdx.x == 0) {
            if (t + FT_LA <= thi) {
                ft_issue(D, S, P, t + FT_LA, true, &tmr, &tmz, &tmf);
                issued = t + FT_LA;
            }
            if (!mbar_wait(S.bar(ft_slot(P, t)), ft_parity(P, t))) abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        const FTRing R(P, t);
        ft_half_sweep(D, S, P, Q, R, 1, t - 1, 1, 3, scale, 1);
        __syncthreads();
        ft_half_sweep(D, S, P, Q, R, 2, t - 2, 0, 2, scale, 2);
        __syncthreads();
        ft_half_sweep(D, S, P, Q, R, 3, t - 3, 1, 1, scale, 3);
        __syncthreads();
        // last half-sweep on plane t-4 (colour 0, the tile only); each thread then stores its quad and
        // adds r z of its four cells to the product
        const int tf = t - 4;
        // every lane takes part (the half-sweep votes across the warp); with halo 0 only the tile's
        // cells in the domain change
        if (tf >= k0 && tf < k1) ft_half_sweep(D, S, P, Q, R, 4, tf, 0, 0, scale, 4);
        if (tf >= k0 && tf < k1 && Q.tile >= 0 && Q.dom == 0xfu) {
            const int s = R.sl[4];
            const float4 z4 = lds4(S.z(s) + Q.c), r4 = lds4(S.r(s) + Q.c);
            *reinterpret_cast<float4*>(z + Q.gx + (long long)D.sy * Q.gy + D.sz * tf) = z4;
            part += (r4.x * z4.x + r4.y * z4.y) + (r4.z * z4.z + r4.w * z4.w);
        }
        fence_proxy_async();
        __syncthreads();
    }
    if (abort_flag) {
        if (threadIdx.x == 0) {
            for (int u = issued; u > issued - FT_NS && u >= P.tlo; --u) mbar_wait(S.bar(ft_slot(P, u)), ft_parity(P, u));
            atomicExch(&sc->dev_error, 1);
        }
        part = 0.f;
    }
    decltype(part) acc[1] = {part};
    grid_reduce<1>(acc, partials, counter, [&](double* tt) {
        sc->rz_old = sc->rz;
        sc->rz = tt[0];
    });
}

// ---- set-up -------------------------------------------------------------------------------------

// Level 1: parts of every block (cnt) and the part of every fine cell (sub0).
__global__ void k_parts1(Dom D, MGLev L, uint8_t* __restrict__ sub0) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < L.P; q += (long long)gridDim.x * blockDim.x) {
        int X[3];
        coords3(q, L.px, L.py, X);
        unsigned fl[8];
        long long P[8];
        const unsigned in = block_flags(D, X, fl, P);
        int part[8];
        L.cnt[q] = fine_parts(D, fl, in, part);
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if ((in >> m) & 1u) sub0[P[m]] = (uint8_t)part[m];
    }
}

// Adds conductance g towards unknown v to a small table of distinct neighbours; false when full.
template <int CAP>
__device__ __forceinline__ bool table_add(int (&nb)[CAP], float (&gv)[CAP], int& n, int v, float g) {
    for (int e = 0; e < n; ++e)
        if (nb[e] == v) {
            gv[e] += g;
            return true;
        }
    if (n == CAP) return false;
    nb[n] = v;
    gv[n] = g;
    ++n;
    return true;
}

// Writes a row sorted by neighbour index (insertion sort; rows are short).
template <int CAP>
__device__ __forceinline__ float write_row(const MGLev& L, long long u, int (&nb)[CAP], float (&gv)[CAP], int n) {
    for (int e = 1; e < n; ++e) {
        const int v = nb[e];
        const float w = gv[e];
        int f = e - 1;
        while (f >= 0 && nb[f] > v) {
            nb[f + 1] = nb[f];
            gv[f + 1] = gv[f];
            --f;
        }
        nb[f + 1] = v;
        gv[f + 1] = w;
    }
    const long long k0 = L.rp[u];
    float gs = 0.f;
    for (int e = 0; e < n; ++e) {
        L.col[k0 + e] = nb[e];
        L.g[k0 + e] = gv[e];
        gs += gv[e];
    }
    return gs;
}

// Level 1 links.  Count pass (fill = 0): rp[u] = distinct neighbours, d, pos.  Fill pass: the sorted
// row, invdg.  A fine link leaving the block joins the part of its cell to the part of the cell across.
__global__ void k_links1(Dom D, MGLev L, const uint8_t* __restrict__ sub0, int fill, int* ovf) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < L.P; q += (long long)gridDim.x * blockDim.x) {
        int X[3];
        coords3(q, L.px, L.py, X);
        unsigned fl[8];
        long long P[8];
        const unsigned in = block_flags(D, X, fl, P);
        const int np = L.cnt[q];
        const int n3[3] = {D.nx, D.ny, D.nz};
        for (int s = 0; s < np; ++s) {
            const long long u = L.off[q] + s;
            int nb[MG_L1L];
            float gv[MG_L1L];
            int n = 0;
            float dsum = 0.f;
            for (int m = 0; m < 8; ++m) {
                if (!((in >> m) & 1u) || sub0[P[m]] != s) continue;
                const int x[3] = {2 * X[0] + (m & 1), 2 * X[1] + ((m >> 1) & 1), 2 * X[2] + (m >> 2)};
                for (int b = 0; b < 6; ++b) {
                    if (fl[m] & (1u << b)) continue;
                    const int a = b >> 1, sd = (b & 1) ? 1 : -1;
                    long long o;
                    if (!nb_offset(D, a, sd, x[a], o)) {
                        if (D.bc[b] == IBM_BC_OUTFLOW) dsum += 2.f;
                        continue;
                    }
                    int y[3] = {x[0], x[1], x[2]};
                    y[a] += sd;
                    if (y[a] < 0) y[a] = n3[a] - 1;
                    if (y[a] >= n3[a]) y[a] = 0;
                    const int Y[3] = {y[0] >> 1, y[1] >> 1, y[2] >> 1};
                    if (Y[0] == X[0] && Y[1] == X[1] && Y[2] == X[2]) continue;      // inside the block
                    const int v = L.off[pos_index(L, Y)] + sub0[P[m] + o];
                    if (!table_add<MG_L1L>(nb, gv, n, v, 1.f)) *ovf = 1;
                }
            }
            if (!fill) {
                L.rp[u] = n;
                L.d[u] = dsum;
                L.pos[u] = (int32_t)q;
            } else {
                const float gs = write_row<MG_L1L>(L, u, nb, gv, n);
                L.invdg[u] = gs + dsum > 0.f ? 1.f / (gs + dsum) : 0.f;
            }
        }
    }
}

// Children of coarse position Y: the unknowns of the (up to) 8 positions of level F below it, in
// position order.  Returns how many there are; the first MG_MAXCH go into list.
__device__ __forceinline__ int block_children(const MGLev& F, const int Y[3], int (&list)[MG_MAXCH]) {
    int n = 0;
    for (int m = 0; m < 8; ++m) {
        const int X[3] = {2 * Y[0] + (m & 1), 2 * Y[1] + ((m >> 1) & 1), 2 * Y[2] + (m >> 2)};
        if (X[0] >= F.px || X[1] >= F.py || X[2] >= F.pz) continue;
        const long long q = pos_index(F, X);
        const int o = F.off[q], c = F.cnt[q];
        for (int k = 0; k < c; ++k, ++n)
            if (n < MG_MAXCH) list[n] = o + k;
    }
    return n;
}

// Level l + 1 from level l (= F): parts of each block of 8 positions.  F.parent[u] receives the part
// of u within its block (made global by k_parent_next).  Children beyond MG_MAXCH, and internal links
// beyond MG_MAXE, are not followed: such children stay parts of their own (a finer partition is as
// valid an aggregation).
__global__ void k_parts_next(MGLev F, MGLev C) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < C.P; q += (long long)gridDim.x * blockDim.x) {
        int Y[3];
        coords3(q, C.px, C.py, Y);
        int list[MG_MAXCH];
        const int ntot = block_children(F, Y, list);
        const int n = ntot < MG_MAXCH ? ntot : MG_MAXCH;
        uint8_t ea[MG_MAXE], eb[MG_MAXE];
        int ne = 0;
        for (int k = 0; k < n; ++k) {
            const int u = list[k];
            for (int e = F.rp[u]; e < F.rp[u + 1]; ++e) {
                const int w = F.col[e];
                if (w < u) continue;                       // each internal link once
                int Xw[3];
                coords3(F.pos[w], F.px, F.py, Xw);
                if ((Xw[0] >> 1) != Y[0] || (Xw[1] >> 1) != Y[1] || (Xw[2] >> 1) != Y[2]) continue;
                int kw = -1;
                for (int t = 0; t < n; ++t)
                    if (list[t] == w) {
                        kw = t;
                        break;
                    }
                if (kw < 0 || ne == MG_MAXE) continue;
                ea[ne] = (uint8_t)k;
                eb[ne] = (uint8_t)kw;
                ++ne;
            }
        }
        uint8_t lab[MG_MAXCH];
        for (int k = 0; k < n; ++k) lab[k] = (uint8_t)k;
        for (int it = 0; it < n; ++it) {
            bool changed = false;
            for (int e = 0; e < ne; ++e) {
                const uint8_t lo = lab[ea[e]] < lab[eb[e]] ? lab[ea[e]] : lab[eb[e]];
                if (lab[ea[e]] != lo || lab[eb[e]] != lo) {
                    lab[ea[e]] = lo;
                    lab[eb[e]] = lo;
                    changed = true;
                }
            }
            if (!changed) break;
        }
        // part numbers: roots in list order, then the children that were not followed
        int nroot = 0;
        uint8_t rank[MG_MAXCH];
        for (int k = 0; k < n; ++k)
            if (lab[k] == k) rank[k] = (uint8_t)nroot++;
        for (int k = 0; k < n; ++k) F.parent[list[k]] = rank[lab[k]];
        if (ntot > n) {
            int extra = 0;
            for (int m = 0; m < 8; ++m) {
                const int X[3] = {2 * Y[0] + (m & 1), 2 * Y[1] + ((m >> 1) & 1), 2 * Y[2] + (m >> 2)};
                if (X[0] >= F.px || X[1] >= F.py || X[2] >= F.pz) continue;
                const long long qx = pos_index(F, X);
                for (int k = 0; k < F.cnt[qx]; ++k, ++extra)
                    if (extra >= MG_MAXCH) F.parent[F.off[qx] + k] = nroot + (extra - MG_MAXCH);
            }
        }
        C.cnt[q] = nroot + (ntot - n);
    }
}

__global__ void k_parent_next(MGLev F, MGLev C) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < F.M; u += (long long)gridDim.x * blockDim.x) {
        int X[3];
        coords3(F.pos[u], F.px, F.py, X);
        const int Y[3] = {X[0] >> 1, X[1] >> 1, X[2] >> 1};
        F.parent[u] = C.off[pos_index(C, Y)] + F.parent[u];
    }
}

// Level l + 1 links (Galerkin sums) and children lists.  Count pass: rp[v] = distinct neighbours,
// cp[v] = children, d, pos.  Fill pass: sorted rows, invdg, children.
__global__ void k_links_next(MGLev F, MGLev C, int fill, int* ovf) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < C.P; q += (long long)gridDim.x * blockDim.x) {
        int Y[3];
        coords3(q, C.px, C.py, Y);
        const int np = C.cnt[q];
        for (int s = 0; s < np; ++s) {
            const int v = C.off[q] + s;
            int nb[MG_MAXL];
            float gv[MG_MAXL];
            int n = 0, nch = 0;
            float dsum = 0.f;
            for (int m = 0; m < 8; ++m) {
                const int X[3] = {2 * Y[0] + (m & 1), 2 * Y[1] + ((m >> 1) & 1), 2 * Y[2] + (m >> 2)};
                if (X[0] >= F.px || X[1] >= F.py || X[2] >= F.pz) continue;
                const long long qx = pos_index(F, X);
                for (int u = F.off[qx]; u < F.off[qx] + F.cnt[qx]; ++u) {
                    if (F.parent[u] != v) continue;
                    if (fill) C.ch[C.cp[v] + nch] = u;
                    ++nch;
                    dsum += F.d[u];
                    for (int e = F.rp[u]; e < F.rp[u + 1]; ++e) {
                        const int pw = F.parent[F.col[e]];
                        if (pw == v) continue;
                        if (!table_add<MG_MAXL>(nb, gv, n, pw, F.g[e])) *ovf = 1;
                    }
                }
            }
            if (!fill) {
                C.rp[v] = n;
                C.cp[v] = nch;
                C.d[v] = dsum;
                C.pos[v] = (int32_t)q;
            } else {
                const float gs = write_row<MG_MAXL>(C, v, nb, gv, n);
                C.invdg[v] = gs + dsum > 0.f ? 1.f / (gs + dsum) : 0.f;
            }
        }
    }
}

// Colour-major numbering of the unknowns: positions of colour c contribute cnt[q] unknowns each, in
// position order, after all unknowns of colour 0 when c = 1.
struct PosCount {
    const int32_t* cnt;
    int px, py, colour;
    __device__ long long operator()(long long i) const {
        int x[3];
        coords3(i, px, py, x);
        return ((x[0] + x[1] + x[2]) & 1) == colour ? cnt[i] : 0;
    }
};
struct PosEmit {
    int32_t* off;
    int px, py, colour;
    const long long* base;
    __device__ void operator()(long long i, long long o, long long) const {
        int x[3];
        coords3(i, px, py, x);
        if (((x[0] + x[1] + x[2]) & 1) == colour) off[i] = (int32_t)(o + (base ? *base : 0));
    }
};
// In-place exclusive scan of a count array (rows, children).
struct ArrCount {
    const int32_t* a;
    __device__ long long operator()(long long i) const { return a[i]; }
};
struct ArrEmit {
    int32_t* a;
    __device__ void operator()(long long i, long long o, long long) const { a[i] = (int32_t)o; }
};

// ---- the V-cycle on the coarse levels -----------------------------------------------------------

// One red-black pass of colour `col` over the unknowns t0, t0 + nt, ... of that colour.  With `zero`
// the iterate is taken as 0: colour `col` gets -b / dg and the other colour is cleared.
template <class T>
__device__ __forceinline__ void gsmooth(const MGLev& L, int col, bool zero, long long t0, long long nt) {
    const T* __restrict__ b = (const T*)L.b;
    T* x = (T*)L.x;
    if (zero) {
        for (long long u = t0; u < L.M; u += nt) {
            const bool mine = (u < L.M0) == (col == 0);
            x[u] = mine ? -b[u] * (T)L.invdg[u] : (T)0;
        }
        return;
    }
    const long long lo = col ? L.M0 : 0, hi = col ? L.M : L.M0;
    for (long long u = lo + t0; u < hi; u += nt) {
        T s = 0;
        for (int e = L.rp[u]; e < L.rp[u + 1]; ++e) s += (T)L.g[e] * x[L.col[e]];
        x[u] = (s - b[u]) * (T)L.invdg[u];
    }
}

// b_C[v] = sum over the children u of v of the level-F residual  b_u - (sum g (x_w - x_u) - d_u x_u).
template <class T>
__device__ __forceinline__ void grestrict(const MGLev& F, const MGLev& C, long long t0, long long nt) {
    const T* __restrict__ bf = (const T*)F.b;
    const T* __restrict__ xf = (const T*)F.x;
    T* __restrict__ bc = (T*)C.b;
    for (long long v = t0; v < C.M; v += nt) {
        T acc = 0;
        for (int k = C.cp[v]; k < C.cp[v + 1]; ++k) {
            const int u = C.ch[k];
            const T xu = xf[u];
            T ax = -(T)F.d[u] * xu;
            for (int e = F.rp[u]; e < F.rp[u + 1]; ++e) ax += (T)F.g[e] * (xf[F.col[e]] - xu);
            acc += bf[u] - ax;
        }
        bc[v] = acc;
    }
}

// x_F[u] += omega x_C[parent of u].
template <class T>
__device__ __forceinline__ void gprolong(const MGLev& F, const MGLev& C, T omega, long long t0, long long nt) {
    T* __restrict__ xf = (T*)F.x;
    const T* __restrict__ xc = (const T*)C.x;
    for (long long u = t0; u < F.M; u += nt) xf[u] = xf[u] + omega * xc[F.parent[u]];
}

// Coarsest level, one block: x = 0, then `sweeps` red-black passes and as many black-red (a
// symmetric operator).  The iterate stays in global memory; __syncthreads orders the passes.
template <class T>
__device__ __forceinline__ void gcoarsest(const MGLev& L, int sweeps) {
    T* x = (T*)L.x;
    for (long long u = threadIdx.x; u < L.M; u += blockDim.x) x[u] = (T)0;
    __syncthreads();
    for (int pass = 0; pass < 4 * sweeps; ++pass) {
        const int half = pass / (2 * sweeps);
        gsmooth<T>(L, (pass & 1) ^ half, false, threadIdx.x, blockDim.x);
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_gsmooth(MGLev L, int col, int zero, const SolveScal* sc) {
    if (sc->done) return;
    gsmooth<T>(L, col, zero != 0, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

template <class T>
__global__ void __launch_bounds__(256) k_grestrict(MGLev F, MGLev C, const SolveScal* sc) {
    if (sc->done) return;
    grestrict<T>(F, C, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

template <class T>
__global__ void __launch_bounds__(256) k_gprolong(MGLev F, MGLev C, T omega, const SolveScal* sc) {
    if (sc->done) return;
    gprolong<T>(F, C, omega, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

template <class T>
__global__ void __launch_bounds__(1024) k_gcoarsest(MGLev L, int sweeps, const SolveScal* sc) {
    if (sc->done) return;
    gcoarsest<T>(L, sweeps);
}

// The small levels first .. nlev-1 of a V-cycle in one launch: one cluster of MG_TAIL_CTAS blocks of
// 1024 threads walks the descent (smoothing, restriction), the coarsest solve (block 0) and the
// ascent (prolongation, smoothing), with a cluster barrier (hardware, release/acquire at cluster
// scope) between dependent passes.  These levels are small and stay in L2; as separate kernels each
// pass would cost a launch for a few microseconds of work.
template <class T>
__global__ void __launch_bounds__(1024) k_mg_tail(MGTail M, const SolveScal* sc) {
    if (sc->done) return;                       // the flag is uniform: set by an earlier kernel
    cg::cluster_group cl = cg::this_cluster();
    const long long t0 = (long long)cl.block_rank() * blockDim.x + threadIdx.x;
    const long long nt = (long long)cl.num_blocks() * blockDim.x;
    auto bar = [&]() {
        __threadfence();
        cl.sync();
    };
    const int last = M.nlev - 1;
    for (int l = M.first; l < last; ++l) {
        for (int q = 0; q < M.sweeps; ++q) {
            gsmooth<T>(M.lev[l], 0, q == 0, t0, nt);
            bar();
            gsmooth<T>(M.lev[l], 1, false, t0, nt);
            bar();
        }
        grestrict<T>(M.lev[l], M.lev[l + 1], t0, nt);
        bar();
    }
    if (cl.block_rank() == 0) gcoarsest<T>(M.lev[last], M.coarse_sweeps);
    bar();
    for (int l = last - 1; l >= M.first; --l) {
        gprolong<T>(M.lev[l], M.lev[l + 1], (T)M.omega, t0, nt);
        bar();
        for (int q = 0; q < M.sweeps; ++q) {
            gsmooth<T>(M.lev[l], 1, false, t0, nt);
            bar();
            gsmooth<T>(M.lev[l], 0, false, t0, nt);
            bar();
        }
    }
}

// ---- transfer between the fine grid and level 1 -------------------------------------------------

// b_1 of each part of a level-1 block = the sum of the fine residuals  scale r - (A z)  of its cells.
template <class T>
__global__ void __launch_bounds__(256) k_mg_restrict0(Dom D, const T* __restrict__ r, const T* __restrict__ z, T scale,
                                                      MGLev C, const SolveScal* sc) {
    if (sc->done) return;
    T* __restrict__ bc = (T*)C.b;
    auto zv = [&](long long c) { return z[c]; };
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < C.P; q += (long long)gridDim.x * blockDim.x) {
        int X[3];
        coords3(q, C.px, C.py, X);
        unsigned fl[8];
        long long P[8];
        const unsigned in = block_flags(D, X, fl, P);
        int part[8];
        const int np = fine_parts(D, fl, in, part);
        T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            if (!((in >> m) & 1u)) continue;
            const int x0 = 2 * X[0] + (m & 1), x1 = 2 * X[1] + ((m >> 1) & 1), x2 = 2 * X[2] + (m >> 2);
            const T res = scale * r[P[m]] - link_sum7<T>(D, P[m], x0, x1, x2, fl[m], z[P[m]], zv);
#pragma unroll
            for (int s = 0; s < 8; ++s) acc[s] += part[m] == s ? res : (T)0;
        }
        const int o = C.off[q];
#pragma unroll
        for (int s = 0; s < 8; ++s)
            if (s < np) bc[o + s] = acc[s];
    }
}

// z += omega x_1(part of the cell).
template <class T>
__global__ void __launch_bounds__(256) k_mg_prolong0(Dom D, T* __restrict__ z, MGLev C, T omega, const SolveScal* sc) {
    if (sc->done) return;
    const T* __restrict__ xc = (const T*)C.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < C.P; q += (long long)gridDim.x * blockDim.x) {
        int X[3];
        coords3(q, C.px, C.py, X);
        unsigned fl[8];
        long long P[8];
        const unsigned in = block_flags(D, X, fl, P);
        int part[8];
        const int np = fine_parts(D, fl, in, part);
        const int o = C.off[q];
        T v[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) v[s] = s < np ? xc[o + s] : (T)0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            if (!((in >> m) & 1u)) continue;
            T w = v[0];
#pragma unroll
            for (int s = 1; s < 8; ++s) w = part[m] == s ? v[s] : w;
            z[P[m]] = z[P[m]] + omega * w;
        }
    }
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ unsigned flags4(const Dom& D, long long P) {
    return D.flags ? *reinterpret_cast<const unsigned*>(D.flags + P) : 0u;
}

// FP32 restriction with nx a multiple of 4: one thread per pair of level-1 positions (2 xp, 2 xp + 1)
// at (Y, Z), i.e. the 4 fine cells [4 xp, 4 xp + 4) of each of the (up to) 4 fine rows below them,
// with 16-byte loads.
__global__ void __launch_bounds__(256) k_mg_restrict0_x4(Dom D, const float* __restrict__ r,
                                                         const float* __restrict__ z, float scale, MGLev C,
                                                         const SolveScal* sc) {
    if (sc->done) return;
    float* __restrict__ bc = (float*)C.b;
    const int px = D.nx / 4;
    const long long npairs = (long long)px * C.py * C.pz;
    auto zv = [&](long long c) { return z[c]; };
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < npairs;
         t += (long long)gridDim.x * blockDim.x) {
        const unsigned tu = (unsigned)t, rq = tu / (unsigned)px;
        const int xp = (int)(tu - rq * (unsigned)px), Y = (int)(rq % (unsigned)C.py), Z = (int)(rq / (unsigned)C.py);
        const int i0 = 4 * xp;
        float res[2][2][4];
        unsigned f4[2][2];
        unsigned rows = 0;
#pragma unroll
        for (int dk = 0; dk < 2; ++dk)
#pragma unroll
            for (int dj = 0; dj < 2; ++dj) {
                const int j = 2 * Y + dj, k = 2 * Z + dk;
                f4[dk][dj] = 0u;
#pragma unroll
                for (int m = 0; m < 4; ++m) res[dk][dj][m] = 0.f;
                if (j >= D.ny || k >= D.nz) continue;
                rows |= 1u << (2 * dk + dj);
                const long long P = i0 + (long long)D.sy * j + D.sz * k;
                const unsigned fl4 = flags4(D, P);
                f4[dk][dj] = fl4;
                const float4 r4 = ld4(r + P), z4 = ld4(z + P);
                const float zc[4] = {z4.x, z4.y, z4.z, z4.w}, rr[4] = {r4.x, r4.y, r4.z, r4.w};
                if (fl4 == 0u && i0 > 0 && i0 + 4 < D.nx && j > 0 && j < D.ny - 1 && k > 0 && k < D.nz - 1) {
                    const float4 ym = ld4(z + P - D.sy), yp = ld4(z + P + D.sy);
                    const float4 zm = ld4(z + P - D.sz), zp = ld4(z + P + D.sz);
                    const float xl = z[P - 1], xr = z[P + 4];
                    const float a[4] = {ym.x + yp.x + zm.x + zp.x, ym.y + yp.y + zm.y + zp.y,
                                        ym.z + yp.z + zm.z + zp.z, ym.w + yp.w + zm.w + zp.w};
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const float xm = m == 0 ? xl : zc[m - 1];
                        const float xq = m == 3 ? xr : zc[m + 1];
                        res[dk][dj][m] = scale * rr[m] - ((xm + xq) + a[m] - 6.f * zc[m]);
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const unsigned fl = (fl4 >> (8 * m)) & 0xffu;
                        res[dk][dj][m] = scale * rr[m] - link_sum7<float>(D, P + m, i0 + m, j, k, fl, zc[m], zv);
                    }
                }
            }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned fl[8];
            unsigned in = 0;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int di = m & 1, dj = (m >> 1) & 1, dk = m >> 2;
                fl[m] = (f4[dk][dj] >> (8 * (2 * h + di))) & 0xffu;
                in |= ((rows >> (2 * dk + dj)) & 1u) << m;
            }
            int part[8];
            const int np = fine_parts(D, fl, in, part);
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float v = res[m >> 2][(m >> 1) & 1][2 * h + (m & 1)];
#pragma unroll
                for (int s = 0; s < 8; ++s) acc[s] += part[m] == s ? v : 0.f;
            }
            const int o = C.off[(2 * xp + h) + (long long)C.px * (Y + (long long)C.py * Z)];
#pragma unroll
            for (int s = 0; s < 8; ++s)
                if (s < np) bc[o + s] = acc[s];
        }
    }
}

// FP32 prolongation with nx a multiple of 4, same layout as k_mg_restrict0_x4.
__global__ void __launch_bounds__(256) k_mg_prolong0_x4(Dom D, float* __restrict__ z, MGLev C, float omega,
                                                        const SolveScal* sc) {
    if (sc->done) return;
    const float* __restrict__ xc = (const float*)C.x;
    const int px = D.nx / 4;
    const long long npairs = (long long)px * C.py * C.pz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < npairs;
         t += (long long)gridDim.x * blockDim.x) {
        const unsigned tu = (unsigned)t, rq = tu / (unsigned)px;
        const int xp = (int)(tu - rq * (unsigned)px), Y = (int)(rq % (unsigned)C.py), Z = (int)(rq / (unsigned)C.py);
        const int i0 = 4 * xp;
        unsigned f4[2][2];
        unsigned rows = 0;
#pragma unroll
        for (int dk = 0; dk < 2; ++dk)
#pragma unroll
            for (int dj = 0; dj < 2; ++dj) {
                const int j = 2 * Y + dj, k = 2 * Z + dk;
                const bool ok = j < D.ny && k < D.nz;
                f4[dk][dj] = ok ? flags4(D, i0 + (long long)D.sy * j + D.sz * k) : 0u;
                rows |= (ok ? 1u : 0u) << (2 * dk + dj);
            }
        float w[2][8];     // [position][cell]: the coarse value each fine cell receives
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned fl[8];
            unsigned in = 0;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int di = m & 1, dj = (m >> 1) & 1, dk = m >> 2;
                fl[m] = (f4[dk][dj] >> (8 * (2 * h + di))) & 0xffu;
                in |= ((rows >> (2 * dk + dj)) & 1u) << m;
            }
            int part[8];
            const int np = fine_parts(D, fl, in, part);
            const int o = C.off[(2 * xp + h) + (long long)C.px * (Y + (long long)C.py * Z)];
            float v[8];
#pragma unroll
            for (int s = 0; s < 8; ++s) v[s] = s < np ? xc[o + s] : 0.f;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                float a = v[0];
#pragma unroll
                for (int s = 1; s < 8; ++s) a = part[m] == s ? v[s] : a;
                w[h][m] = a;
            }
        }
#pragma unroll
        for (int dk = 0; dk < 2; ++dk)
#pragma unroll
            for (int dj = 0; dj < 2; ++dj) {
                if (!((rows >> (2 * dk + dj)) & 1u)) continue;
                const long long P = i0 + (long long)D.sy * (2 * Y + dj) + D.sz * (2 * Z + dk);
                float4 z4 = ld4(z + P);
                const int m0 = 2 * dj + 4 * dk;
                z4.x += omega * w[0][m0];
                z4.y += omega * w[0][m0 + 1];
                z4.z += omega * w[1][m0];
                z4.w += omega * w[1][m0 + 1];
                st4(z + P, z4);
            }
    }
}

unsigned lin_blocks(long long n) {
    long long b = (n + 255) / 256;
    long long cap = 8LL * IBM_NSM;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

// ---- tensor maps of the fused passes -------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// 3-D map of an nx x ny x nz array of `esize`-byte elements, box (boxx, FT_RY, 1): one plane of a
// tile plus its halo per load.  Elements outside the array read as zero.
int make_plane_map(CUtensorMap* out, const Dom& D, const void* ptr, CUtensorMapDataType dt, int esize, int boxx) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn) return ibm_fail(IBM_E_CUDA, "multigrid: cuTensorMapEncodeTiled is not available");
    alignas(64) CUtensorMap m;
    cuuint64_t dims[3] = {(cuuint64_t)D.nx, (cuuint64_t)D.ny, (cuuint64_t)D.nz};
    cuuint64_t strides[2] = {(cuuint64_t)D.nx * esize, (cuuint64_t)D.nx * D.ny * esize};
    cuuint32_t box[3] = {(cuuint32_t)boxx, (cuuint32_t)FT_RY, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(&m, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return ibm_fail(IBM_E_CUDA, "multigrid: cuTensorMapEncodeTiled failed (%d)", (int)r);
    memcpy(out, &m, sizeof(m));
    return IBM_OK;
}

// Whether the fused passes apply, and their launch shape: tiles of FT_TX x FT_TY and the z-chunk that
// minimises waves x (chunk + 8 planes of pipeline) with two resident blocks per SM.
void fused_plan(const LesCtx& c, MG& mg, int sb) {
    const Dom& D = c.D;
    bool per = false;
    for (int f = 0; f < 6; ++f) per = per || D.bc[f] == IBM_BC_PERIODIC;
    mg.fused = mg.allow_fused && sb == 4 && mg.sweeps == 2 && mg.nlev > 1 && D.flags != nullptr && !per && D.nx % 16 == 0 &&
               D.nx >= 16 && D.ny >= 2 && D.nz >= 2 && encode_tiled() != nullptr;
    if (!mg.fused) return;
    const long long tx = (D.nx + FT_TX - 1) / FT_TX, ty = (D.ny + FT_TY - 1) / FT_TY;
    const long long slots = 2LL * IBM_NSM;
    long long best = -1;
    int best_k = D.nz + (D.nz & 1);
    for (int ch = 1; ch <= 64; ++ch) {
        int k = (D.nz + ch - 1) / ch;
        k += k & 1;
        if (k < 8 && ch > 1) break;
        const long long nchunk = (D.nz + k - 1) / k;
        const long long waves = (tx * ty * nchunk + slots - 1) / slots;
        const long long cost = waves * (k + 8);
        if (best < 0 || cost < best) {
            best = cost;
            best_k = k;
        }
    }
    mg.fz_chunk = best_k;
    mg.fgrid = dim3((unsigned)tx, (unsigned)ty, (unsigned)((D.nz + best_k - 1) / best_k));
    mg.tm_r_ptr = nullptr;
}

// ---- host side of the set-up --------------------------------------------------------------------

struct SetupTmp {
    long long* tiles = nullptr;     // scan tiles + 4 totals
    long long nt = 0;
    int* ovf = nullptr;
    uint8_t* sub0 = nullptr;
    ~SetupTmp() {
        cudaFree(tiles);
        cudaFree(ovf);
        cudaFree(sub0);
    }
};

void free_level(MGLev& L) {
    cudaFree(L.off); cudaFree(L.cnt); cudaFree(L.pos); cudaFree(L.rp); cudaFree(L.col); cudaFree(L.g);
    cudaFree(L.d); cudaFree(L.invdg); cudaFree(L.parent); cudaFree(L.cp); cudaFree(L.ch); cudaFree(L.b);
    cudaFree(L.x);
    const int px = L.px, py = L.py, pz = L.pz;
    const long long P = L.P;
    memset(&L, 0, sizeof(L));
    L.px = px; L.py = py; L.pz = pz; L.P = P;
}

#define MG_ALLOC(ptr, n)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = cudaMalloc((void**)&(ptr), ((n) > 0 ? (size_t)(n) : 1) * sizeof(*(ptr))); \
        if (e_ != cudaSuccess) return ibm_cuda_check(e_, "multigrid set-up: " #ptr);              \
    } while (0)
#define MG_ALLOCB(ptr, bytes)                                                                    \
    do {                                                                                         \
        cudaError_t e_ = cudaMalloc((void**)&(ptr), (size_t)(bytes) > 0 ? (size_t)(bytes) : 16); \
        if (e_ != cudaSuccess) return ibm_cuda_check(e_, "multigrid set-up: " #ptr);              \
    } while (0)

long long read_ll(const long long* d) {
    long long h = 0;
    cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    return h;
}

// Colour-major offsets of the positions' unknowns; sets L.M0 and L.M.
int number_unknowns(MGLev& L, SetupTmp& t) {
    long long* tot = t.tiles + t.nt;
    IBM_CUDA(scan_emit(L.P, PosCount{L.cnt, L.px, L.py, 0}, PosEmit{L.off, L.px, L.py, 0, nullptr}, t.tiles, tot, 0));
    IBM_CUDA(scan_emit(L.P, PosCount{L.cnt, L.px, L.py, 1}, PosEmit{L.off, L.px, L.py, 1, tot}, t.tiles, tot + 1, 0));
    IBM_CUDA(cudaDeviceSynchronize());
    L.M0 = read_ll(tot);
    L.M = L.M0 + read_ll(tot + 1);
    if (L.M >= (1LL << 31)) return ibm_fail(IBM_E_INVALID, "multigrid set-up: too many unknowns");
    return IBM_OK;
}

// Exclusive scan of a[0..n) in place; a[n] = total.  Returns the total in *total.
int scan_in_place(int32_t* a, long long n, SetupTmp& t, long long* total) {
    long long* tot = t.tiles + t.nt + 2;
    IBM_CUDA(scan_emit(n, ArrCount{a}, ArrEmit{a}, t.tiles, tot, 0));
    IBM_CUDA(cudaDeviceSynchronize());
    *total = read_ll(tot);
    if (*total >= (1LL << 31)) return ibm_fail(IBM_E_INVALID, "multigrid set-up: too many links");
    const int32_t h = (int32_t)*total;
    IBM_CUDA(cudaMemcpy(a + n, &h, sizeof(h), cudaMemcpyHostToDevice));
    return IBM_OK;
}

int build_level1(const LesCtx& c, MGLev& L, int sb, SetupTmp& t) {
    const Dom& D = c.D;
    L.px = (D.nx + 1) / 2;
    L.py = (D.ny + 1) / 2;
    L.pz = (D.nz + 1) / 2;
    L.P = (long long)L.px * L.py * L.pz;
    MG_ALLOC(L.off, L.P);
    MG_ALLOC(L.cnt, L.P);
    k_parts1<<<lin_blocks(L.P), 256>>>(D, L, t.sub0);
    IBM_LAUNCHED("k_parts1");
    int rc = number_unknowns(L, t);
    if (rc) return rc;
    MG_ALLOC(L.pos, L.M);
    MG_ALLOC(L.rp, L.M + 1);
    MG_ALLOC(L.d, L.M);
    MG_ALLOC(L.invdg, L.M);
    MG_ALLOC(L.parent, L.M);
    MG_ALLOCB(L.b, L.M * sb);
    MG_ALLOCB(L.x, L.M * sb);
    IBM_CUDA(cudaMemset(t.ovf, 0, sizeof(int)));
    k_links1<<<lin_blocks(L.P), 256>>>(D, L, t.sub0, 0, t.ovf);
    IBM_LAUNCHED("k_links1");
    if ((rc = scan_in_place(L.rp, L.M, t, &L.nnz))) return rc;
    MG_ALLOC(L.col, L.nnz);
    MG_ALLOC(L.g, L.nnz);
    k_links1<<<lin_blocks(L.P), 256>>>(D, L, t.sub0, 1, t.ovf);
    IBM_LAUNCHED("k_links1");
    IBM_CUDA(cudaDeviceSynchronize());
    int h = 0;
    IBM_CUDA(cudaMemcpy(&h, t.ovf, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) return ibm_fail(IBM_E_INVALID, "multigrid set-up: a level-1 block has too many links");
    return IBM_OK;
}

// Level C from level F; returns 1 (and leaves C empty) when the level would not shrink enough or
// a row would not fit, 0 when built, < 0 on error (negated status).
int build_next(MGLev& F, MGLev& C, int sb, SetupTmp& t) {
    C.px = (F.px + 1) / 2;
    C.py = (F.py + 1) / 2;
    C.pz = (F.pz + 1) / 2;
    C.P = (long long)C.px * C.py * C.pz;
    MG_ALLOC(C.off, C.P);
    MG_ALLOC(C.cnt, C.P);
    k_parts_next<<<lin_blocks(C.P), 256>>>(F, C);
    IBM_LAUNCHED("k_parts_next");
    int rc = number_unknowns(C, t);
    if (rc) return -rc;
    if (C.M > (F.M * 4) / 5) {
        free_level(C);
        return 1;
    }
    k_parent_next<<<lin_blocks(F.M), 256>>>(F, C);
    IBM_LAUNCHED("k_parent_next");
    MG_ALLOC(C.pos, C.M);
    MG_ALLOC(C.rp, C.M + 1);
    MG_ALLOC(C.cp, C.M + 1);
    MG_ALLOC(C.ch, F.M);
    MG_ALLOC(C.d, C.M);
    MG_ALLOC(C.invdg, C.M);
    MG_ALLOC(C.parent, C.M);
    MG_ALLOCB(C.b, C.M * sb);
    MG_ALLOCB(C.x, C.M * sb);
    IBM_CUDA(cudaMemset(t.ovf, 0, sizeof(int)));
    k_links_next<<<lin_blocks(C.P), 256>>>(F, C, 0, t.ovf);
    IBM_LAUNCHED("k_links_next");
    IBM_CUDA(cudaDeviceSynchronize());
    int h = 0;
    IBM_CUDA(cudaMemcpy(&h, t.ovf, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        free_level(C);
        return 1;
    }
    long long nch = 0;
    if ((rc = scan_in_place(C.rp, C.M, t, &C.nnz))) return -rc;
    if ((rc = scan_in_place(C.cp, C.M, t, &nch))) return -rc;
    if (nch != F.M) return -ibm_fail(IBM_E_INVALID, "multigrid set-up: children do not cover the level");
    MG_ALLOC(C.col, C.nnz);
    MG_ALLOC(C.g, C.nnz);
    k_links_next<<<lin_blocks(C.P), 256>>>(F, C, 1, t.ovf);
    IBM_LAUNCHED("k_links_next");
    IBM_CUDA(cudaDeviceSynchronize());
    return 0;
}

}  // namespace

// Coarse levels of a V-cycle (level 1 holds the restricted residual; on return level 1 holds the
// coarse correction): descent, coarsest solve and ascent, as separate kernels on the large levels
// and one cluster launch for the small ones.
template <class T>
static int coarse_levels(const LesCtx& c, const MG& mg, SolveScal* sc, cudaStream_t s, int& launches) {
    const T om = (T)mg.omega;
    const int SC = mg.sweeps > 0 ? 1 : 0;
    int tf = mg.nlev;
    for (int l = 1; l + 1 < mg.nlev; ++l)
        if (mg.lev[l].M <= MG_TAIL_MAX) { tf = l; break; }
    const int top = tf < mg.nlev ? tf : mg.nlev - 1;
    for (int l = 1; l < top; ++l) {
        const MGLev& L = mg.lev[l];
        for (int q = 0; q < SC; ++q) {
            k_gsmooth<T><<<lin_blocks(q == 0 ? L.M : L.M0), 256, 0, s>>>(L, 0, q == 0, sc);
            k_gsmooth<T><<<lin_blocks(L.M - L.M0), 256, 0, s>>>(L, 1, 0, sc);
            launches += 2;
        }
        k_grestrict<T><<<lin_blocks(mg.lev[l + 1].M), 256, 0, s>>>(L, mg.lev[l + 1], sc);
        ++launches;
    }
    if (tf < mg.nlev) {
        MGTail M;
        for (int l = 0; l < IBM_MG_MAXLEV; ++l) M.lev[l] = mg.lev[l];
        M.first = tf;
        M.nlev = mg.nlev;
        M.sweeps = SC;
        M.coarse_sweeps = mg.coarse_sweeps;
        M.omega = mg.omega;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(MG_TAIL_CTAS);
        cfg.blockDim = dim3(1024);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = MG_TAIL_CTAS;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        IBM_CUDA(cudaLaunchKernelEx(&cfg, k_mg_tail<T>, M, (const SolveScal*)sc));
        ++launches;
    } else {
        k_gcoarsest<T><<<1, 1024, 0, s>>>(mg.lev[mg.nlev - 1], mg.coarse_sweeps, sc);
        ++launches;
    }
    for (int l = top - 1; l >= 1; --l) {
        const MGLev& L = mg.lev[l];
        k_gprolong<T><<<lin_blocks(L.M), 256, 0, s>>>(L, mg.lev[l + 1], om, sc);
        ++launches;
        for (int q = 0; q < SC; ++q) {
            k_gsmooth<T><<<lin_blocks(L.M - L.M0), 256, 0, s>>>(L, 1, 0, sc);
            k_gsmooth<T><<<lin_blocks(L.M0), 256, 0, s>>>(L, 0, 0, sc);
            launches += 2;
        }
    }
    return IBM_OK;
}

// V-cycle with the fused fine-grid passes: pre-smoothing + restriction, the coarse levels,
// prolongation, post-smoothing + (r, z).
static int vcycle_fused(const LesCtx& c, MG& mg, const float* r, float* z, SolveScal* sc, cudaStream_t s) {
    if (mg.tm_r_ptr != r) {
        int rc = make_plane_map(&mg.tm_r, c.D, r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, FT_RX);
        if (rc) return rc;
        mg.tm_r_ptr = r;
    }
    alignas(64) CUtensorMap tr, tz, tf;
    memcpy(&tr, &mg.tm_r, sizeof(tr));
    memcpy(&tz, &mg.tm_z2, sizeof(tz));
    memcpy(&tf, &mg.tm_f, sizeof(tf));
    float* z2 = (float*)mg.z2;
    const float scale = (float)(c.D.dx * c.D.dx);
    const MGLev& L1 = mg.lev[1];
    int launches = 0;
    prof_begin(c.prof, PS_MG_FINE, s);
    k_mg_pre_fused<<<mg.fgrid, FT_NT, FT_SMEM, s>>>(c.D, z2, scale, L1, mg.fz_chunk, sc, tr, tf);
    prof_end(c.prof, PS_MG_FINE, s);
    ++launches;
    prof_begin(c.prof, PS_MG_COARSE, s);
    int rc = coarse_levels<float>(c, mg, sc, s, launches);
    if (rc) return rc;
    prof_end(c.prof, PS_MG_COARSE, s);
    prof_begin(c.prof, PS_MG_TRANSFER, s);
    k_mg_prolong0_x4<<<lin_blocks((c.D.nx / 4) * (long long)L1.py * L1.pz), 256, 0, s>>>(c.D, z2, L1, (float)mg.omega, sc);
    prof_end(c.prof, PS_MG_TRANSFER, s);
    ++launches;
    prof_begin(c.prof, PS_MG_FINE, s);
    k_mg_post_fused<<<mg.fgrid, FT_NT, FT_SMEM, s>>>(c.D, z, scale, mg.fz_chunk, sc, c.partials, c.counter, tr, tz, tf);
    prof_end(c.prof, PS_MG_FINE, s);
    ++launches;
    IBM_LAUNCHED("mg_vcycle (fused)");
    IBM_COUNT(c, launches);
    return IBM_OK;
}

void mg_free(MG& mg) {
    for (int l = 1; l < IBM_MG_MAXLEV; ++l) free_level(mg.lev[l]);
    cudaFree(mg.z2);
    mg.z2 = nullptr;
    mg.nlev = 1;
}

int mg_setup(const LesCtx& c, MG& mg, int sb) {
    for (int l = 0; l < IBM_MG_MAXLEV; ++l) memset(&mg.lev[l], 0, sizeof(MGLev));
    mg.fused = 0;
    MGLev& L0 = mg.lev[0];
    L0.px = c.D.nx;
    L0.py = c.D.ny;
    L0.pz = c.D.nz;
    L0.P = L0.M = c.D.N;
    mg.nlev = 1;
    if (c.D.N <= MG_COARSE_TARGET) return IBM_OK;      // fine smoothing alone
    SetupTmp t;
    t.nt = scan_tiles(c.D.N);
    MG_ALLOC(t.tiles, t.nt + 4);
    MG_ALLOC(t.ovf, 1);
    MG_ALLOC(t.sub0, c.D.N);
    int rc = build_level1(c, mg.lev[1], sb, t);
    if (rc) return rc;
    mg.nlev = 2;
    for (int l = 1; l + 1 < IBM_MG_MAXLEV; ++l) {
        MGLev& F = mg.lev[l];
        if (F.M <= MG_COARSE_TARGET || F.P == 1) break;
        const int r2 = build_next(F, mg.lev[l + 1], sb, t);
        if (r2 < 0) return -r2;
        if (r2 > 0) break;
        mg.nlev = l + 2;
    }
    fused_plan(c, mg, sb);
    if (mg.fused) {
        IBM_CUDA(cudaFuncSetAttribute(k_mg_pre_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, FT_SMEM));
        IBM_CUDA(cudaFuncSetAttribute(k_mg_post_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, FT_SMEM));
        if ((rc = make_plane_map(&mg.tm_f, c.D, c.D.flags, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, FT_FX))) return rc;
        MG_ALLOCB(mg.z2, c.D.N * 4);
        if ((rc = make_plane_map(&mg.tm_z2, c.D, mg.z2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, FT_RX))) return rc;
    }
    return IBM_OK;
}

// z = V-cycle(r); the last kernel stores rz_old = rz, rz = (r, z).
template <class T>
int mg_vcycle(const LesCtx& c, const MG& mg, const T* r, T* z, SolveScal* sc, cudaStream_t s) {
    const T scale = (T)(c.D.dx * c.D.dx);
    const T om = (T)mg.omega;
    const int S = mg.sweeps;
    // one sweep before and after on the coarse levels: measured faster overall on the dirty sphere than
    // S there too (a few more outer iterations, much less coarse-level work)
    const int SC = S > 0 ? 1 : 0;
    const CellGrid& g = c.cg;
    int launches = 0;
    bool vec = false;
    if constexpr (std::is_same<T, float>::value) vec = x4_ok(c);
    if constexpr (std::is_same<T, float>::value) {
        if (mg.fused) return vcycle_fused(c, const_cast<MG&>(mg), r, z, sc, s);
    }
    auto fine = [&](int col, int zero) {
        prof_begin(c.prof, PS_MG_FINE, s);
        if constexpr (std::is_same<T, float>::value) {
            if (vec) launch_mg_smooth0_x4(c, r, z, scale, col, zero, 0, sc, s);
            else k_mg_smooth0<T><<<c.cgrid, g.block, 0, s>>>(c.D, r, z, scale, col, zero, sc);
        } else {
            k_mg_smooth0<T><<<c.cgrid, g.block, 0, s>>>(c.D, r, z, scale, col, zero, sc);
        }
        prof_end(c.prof, PS_MG_FINE, s);
        ++launches;
    };
    for (int q = 0; q < S; ++q) {
        fine(0, q == 0);
        fine(1, 0);
    }
    if (mg.nlev > 1) {
        const MGLev& L1 = mg.lev[1];
        prof_begin(c.prof, PS_MG_TRANSFER, s);
        if constexpr (std::is_same<T, float>::value) {
            if (vec) k_mg_restrict0_x4<<<lin_blocks((c.D.nx / 4) * (long long)L1.py * L1.pz), 256, 0, s>>>(c.D, r, z, scale, L1, sc);
            else k_mg_restrict0<T><<<lin_blocks(L1.P), 256, 0, s>>>(c.D, r, z, scale, L1, sc);
        } else {
            k_mg_restrict0<T><<<lin_blocks(L1.P), 256, 0, s>>>(c.D, r, z, scale, L1, sc);
        }
        prof_end(c.prof, PS_MG_TRANSFER, s);
        ++launches;
        prof_begin(c.prof, PS_MG_COARSE, s);
        // levels >= tf (if any) run in one cluster launch; separate kernels above them
        int tf = mg.nlev;
        for (int l = 1; l + 1 < mg.nlev; ++l)
            if (mg.lev[l].M <= MG_TAIL_MAX) { tf = l; break; }
        const int top = tf < mg.nlev ? tf : mg.nlev - 1;
        for (int l = 1; l < top; ++l) {
            const MGLev& L = mg.lev[l];
            for (int q = 0; q < SC; ++q) {
                k_gsmooth<T><<<lin_blocks(q == 0 ? L.M : L.M0), 256, 0, s>>>(L, 0, q == 0, sc);
                k_gsmooth<T><<<lin_blocks(L.M - L.M0), 256, 0, s>>>(L, 1, 0, sc);
                launches += 2;
            }
            k_grestrict<T><<<lin_blocks(mg.lev[l + 1].M), 256, 0, s>>>(L, mg.lev[l + 1], sc);
            ++launches;
        }
        if (tf < mg.nlev) {
            MGTail M;
            for (int l = 0; l < IBM_MG_MAXLEV; ++l) M.lev[l] = mg.lev[l];
            M.first = tf;
            M.nlev = mg.nlev;
            M.sweeps = SC;
            M.coarse_sweeps = mg.coarse_sweeps;
            M.omega = mg.omega;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(MG_TAIL_CTAS);
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = 0;
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = MG_TAIL_CTAS;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            IBM_CUDA(cudaLaunchKernelEx(&cfg, k_mg_tail<T>, M, (const SolveScal*)sc));
            ++launches;
        } else {
            k_gcoarsest<T><<<1, 1024, 0, s>>>(mg.lev[mg.nlev - 1], mg.coarse_sweeps, sc);
            ++launches;
        }
        for (int l = top - 1; l >= 1; --l) {
            const MGLev& L = mg.lev[l];
            k_gprolong<T><<<lin_blocks(L.M), 256, 0, s>>>(L, mg.lev[l + 1], om, sc);
            ++launches;
            for (int q = 0; q < SC; ++q) {
                k_gsmooth<T><<<lin_blocks(L.M - L.M0), 256, 0, s>>>(L, 1, 0, sc);
                k_gsmooth<T><<<lin_blocks(L.M0), 256, 0, s>>>(L, 0, 0, sc);
                launches += 2;
            }
        }
        prof_end(c.prof, PS_MG_COARSE, s);
        prof_begin(c.prof, PS_MG_TRANSFER, s);
        if constexpr (std::is_same<T, float>::value) {
            if (vec) k_mg_prolong0_x4<<<lin_blocks((c.D.nx / 4) * (long long)L1.py * L1.pz), 256, 0, s>>>(c.D, z, L1, om, sc);
            else k_mg_prolong0<T><<<lin_blocks(L1.P), 256, 0, s>>>(c.D, z, L1, om, sc);
        } else {
            k_mg_prolong0<T><<<lin_blocks(L1.P), 256, 0, s>>>(c.D, z, L1, om, sc);
        }
        prof_end(c.prof, PS_MG_TRANSFER, s);
        ++launches;
    }
    for (int q = 0; q < S; ++q) {
        fine(1, 0);
        if (q + 1 < S) fine(0, 0);
    }
    prof_begin(c.prof, PS_MG_FINE, s);
    if constexpr (std::is_same<T, float>::value) {
        if (vec) launch_mg_smooth0_x4(c, r, z, scale, 0, 0, 1, sc, s);
        else k_mg_final0<T><<<c.cgrid, g.block, 0, s>>>(c.D, r, z, scale, sc, c.partials, c.counter);
    } else {
        k_mg_final0<T><<<c.cgrid, g.block, 0, s>>>(c.D, r, z, scale, sc, c.partials, c.counter);
    }
    prof_end(c.prof, PS_MG_FINE, s);
    ++launches;
    IBM_LAUNCHED("mg_vcycle");
    IBM_COUNT(c, launches);
    return IBM_OK;
}

template int mg_vcycle<float>(const LesCtx&, const MG&, const float*, float*, SolveScal*, cudaStream_t);
template int mg_vcycle<double>(const LesCtx&, const MG&, const double*, double*, SolveScal*, cudaStream_t);

// mg.cu -- geometric multigrid V-cycle used as the preconditioner of CG for the pressure Poisson
// equation (Eq. poisson).  The paper solves it with BiCGStab or red-black SOR; red-black Gauss-Seidel
// is the smoother here.
//
// Level 0 is the fine grid: the conductance of a link is 1 when its face is uncut and inside the
// domain (or across a periodic seam), 0 otherwise, and an outflow face adds 2 to the diagonal (ghost
// -p).  A coarse cell aggregates the 2x2x2 fine cells below it; with piecewise-constant prolongation
// P and restriction R = P^T the Galerkin coarse operator R A P is again a 7-point operator whose link
// conductance is the sum of the fine conductances crossing the coarse face, so walls seen by the fine
// grid weaken the coarse links in proportion.  The V-cycle (pre-smoothing red then black,
// post-smoothing black then red, the coarse correction scaled by omega < 2, symmetric sweeps on the
// coarsest grid) is a symmetric operator, as CG requires.
//
// Equations are solved in the unscaled form  sum_links g (x_N - x_P) - d x_P = dx^2 r.
#include <cooperative_groups.h>
#include <type_traits>

#include "solver.cuh"

namespace cg = cooperative_groups;

namespace {

#define MG_TAIL_CTAS 8          // portable cluster size
#define MG_TAIL_MAX_CELLS (1LL << 13)

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

// Neighbour offset on a coarse level (periodic axes wrap).
__device__ __forceinline__ bool lev_off(const MGLev& L, int a, int s, int xa, long long& off) {
    const int n = a == 0 ? L.nx : (a == 1 ? L.ny : L.nz);
    const long long st = a == 0 ? 1 : (a == 1 ? L.sy : L.sz);
    const int y = xa + s;
    if (y >= 0 && y < n) { off = s * st; return true; }
    if (!L.per[a]) return false;
    off = -(long long)s * (n - 1) * st;
    return true;
}

// Coarse cell links: g of the -a link is the +a link of the lower neighbour.
__device__ __forceinline__ void coarse_links(const MGLev& L, long long P, const int x[3], float g[6], long long off[6]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        long long om = 0, op = 0;
        const bool inm = lev_off(L, a, -1, x[a], om);
        const bool inp = lev_off(L, a, +1, x[a], op);
        off[2 * a] = om;
        off[2 * a + 1] = op;
        g[2 * a] = inm ? L.g[a][P + om] : 0.f;
        g[2 * a + 1] = inp ? L.g[a][P] : 0.f;
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

// ---- set-up -------------------------------------------------------------------------------------

// Level 1 from the fine grid: conductances of the coarse +a links and the Dirichlet term.
__global__ void k_mg_build1(Dom D, MGLev C) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < C.N; q += (long long)gridDim.x * blockDim.x) {
        int X[3];
        coords3(q, C.nx, C.ny, X);
        const int n[3] = {D.nx, D.ny, D.nz};
        float ga[3] = {0.f, 0.f, 0.f}, dsum = 0.f;
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    const int x[3] = {2 * X[0] + di, 2 * X[1] + dj, 2 * X[2] + dk};
                    if (x[0] >= n[0] || x[1] >= n[1] || x[2] >= n[2]) continue;
                    const long long P = x[0] + (long long)D.sy * x[1] + D.sz * x[2];
                    float g[6], d;
                    long long off[6];
                    fine_links(D, P, x, flags_at(D, P), g, off, d);
                    dsum += d;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if ((x[a] & 1) || x[a] + 1 == n[a]) ga[a] += g[2 * a + 1];   // crosses the coarse +a face
                }
        C.g[0][q] = ga[0];
        C.g[1][q] = ga[1];
        C.g[2][q] = ga[2];
        C.d[q] = dsum;
    }
}

// Level l + 1 from level l.
__global__ void k_mg_build_next(MGLev F, MGLev C) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < C.N; q += (long long)gridDim.x * blockDim.x) {
        int X[3];
        coords3(q, C.nx, C.ny, X);
        const int n[3] = {F.nx, F.ny, F.nz};
        float ga[3] = {0.f, 0.f, 0.f}, dsum = 0.f;
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    const int x[3] = {2 * X[0] + di, 2 * X[1] + dj, 2 * X[2] + dk};
                    if (x[0] >= n[0] || x[1] >= n[1] || x[2] >= n[2]) continue;
                    const long long P = x[0] + F.sy * x[1] + F.sz * x[2];
                    dsum += F.d[P];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if ((x[a] & 1) || x[a] + 1 == n[a]) ga[a] += F.g[a][P];
                }
        C.g[0][q] = ga[0];
        C.g[1][q] = ga[1];
        C.g[2][q] = ga[2];
        C.d[q] = dsum;
    }
}

__global__ void k_mg_invdiag(MGLev L) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < L.N; q += (long long)gridDim.x * blockDim.x) {
        int x[3];
        coords3(q, L.nx, L.ny, x);
        float g[6];
        long long off[6];
        coarse_links(L, q, x, g, off);
        const float dg = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + L.d[q];
        L.invdg[q] = dg > 0.f ? 1.f / dg : 0.f;
    }
}

// ---- smoothing, transfer ------------------------------------------------------------------------

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

// One red-black pass of colour `col` on a coarse level.  Work item t covers the t-th cell of that
// colour (row-major over the half-rows), t = t0, t0 + nt, ...; with `zero` the iterate is taken as 0
// and the cell of the other colour next to it is cleared.
template <class T>
__device__ __forceinline__ void smooth_level(const MGLev& L, int col, bool zero, long long t0, long long nt) {
    const T* __restrict__ b = (const T*)L.b;
    T* __restrict__ x = (T*)L.x;
    const int hx = (L.nx + 1) >> 1;
    const long long n = (long long)hx * L.ny * L.nz;
    for (long long t = t0; t < n; t += nt) {
        int c[3];
        coords3(t, hx, L.ny, c);
        const int par = (col + c[1] + c[2]) & 1;
        const int x0 = 2 * c[0] + par, x1 = 2 * c[0] + (par ^ 1);
        const long long row = L.sy * c[1] + L.sz * c[2];
        if (zero && x1 < L.nx) x[row + x1] = (T)0;
        if (x0 >= L.nx) continue;
        c[0] = x0;
        const long long q = row + x0;
        const float inv = L.invdg[q];
        if (inv == 0.f) { x[q] = (T)0; continue; }
        T s = 0;
        if (!zero) {
            float g[6];
            long long off[6];
            coarse_links(L, q, c, g, off);
#pragma unroll
            for (int e = 0; e < 6; ++e)
                if (g[e] != 0.f) s += (T)g[e] * x[q + off[e]];
        }
        x[q] = (s - b[q]) * (T)inv;
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_mg_smoothc(MGLev L, int col, int zero, const SolveScal* sc) {
    if (sc->done) return;
    smooth_level<T>(L, col, zero != 0, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                    (long long)gridDim.x * blockDim.x);
}

// Residual of level 0 restricted to level 1: each coarse cell sums the residuals of its children.
template <class T>
__global__ void k_mg_restrict0(Dom D, const T* __restrict__ r, const T* __restrict__ z, T scale, MGLev C,
                               const SolveScal* sc) {
    if (sc->done) return;
    T* __restrict__ bc = (T*)C.b;
    const int n[3] = {D.nx, D.ny, D.nz};
    auto zv = [&](long long c) { return z[c]; };
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < C.N; q += (long long)gridDim.x * blockDim.x) {
        int X[3];
        coords3(q, C.nx, C.ny, X);
        T acc = 0;
#pragma unroll
        for (int dk = 0; dk < 2; ++dk)
#pragma unroll
            for (int dj = 0; dj < 2; ++dj)
#pragma unroll
                for (int di = 0; di < 2; ++di) {
                    const int x0 = 2 * X[0] + di, x1 = 2 * X[1] + dj, x2 = 2 * X[2] + dk;
                    if (x0 >= n[0] || x1 >= n[1] || x2 >= n[2]) continue;
                    const long long P = x0 + (long long)D.sy * x1 + D.sz * x2;
                    const T az = link_sum7<T>(D, P, x0, x1, x2, flags_at(D, P), z[P], zv);
                    acc += scale * r[P] - az;
                }
        bc[q] = acc;
    }
}

// Residual of coarse level F restricted to level C (sum over the children).
template <class T>
__device__ __forceinline__ void restrict_level(const MGLev& F, const MGLev& C, long long t0, long long nt) {
    const T* __restrict__ bf = (const T*)F.b;
    const T* __restrict__ xf = (const T*)F.x;
    T* __restrict__ bc = (T*)C.b;
    const int n[3] = {F.nx, F.ny, F.nz};
    for (long long q = t0; q < C.N; q += nt) {
        int X[3];
        coords3(q, C.nx, C.ny, X);
        T acc = 0;
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    const int x[3] = {2 * X[0] + di, 2 * X[1] + dj, 2 * X[2] + dk};
                    if (x[0] >= n[0] || x[1] >= n[1] || x[2] >= n[2]) continue;
                    const long long P = x[0] + F.sy * x[1] + F.sz * x[2];
                    float g[6];
                    long long off[6];
                    coarse_links(F, P, x, g, off);
                    const T xP = xf[P];
                    T ax = -(T)F.d[P] * xP;
#pragma unroll
                    for (int e = 0; e < 6; ++e)
                        if (g[e] != 0.f) ax += (T)g[e] * (xf[P + off[e]] - xP);
                    acc += bf[P] - ax;
                }
        bc[q] = acc;
    }
}

template <class T>
__global__ void k_mg_restrictc(MGLev F, MGLev C, const SolveScal* sc) {
    if (sc->done) return;
    restrict_level<T>(F, C, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// Coarse correction: x_fine += omega * x_coarse(parent), level 0 or a coarse level.
template <class T>
__device__ __forceinline__ void prolong_level(long long N, int nx, int ny, T* __restrict__ xf, const MGLev& C, T omega,
                                              long long t0, long long nt) {
    const T* __restrict__ xc = (const T*)C.x;
    for (long long q = t0; q < N; q += nt) {
        int x[3];
        coords3(q, nx, ny, x);
        const long long parent = (x[0] >> 1) + C.sy * (x[1] >> 1) + C.sz * (x[2] >> 1);
        xf[q] = xf[q] + omega * xc[parent];
    }
}

template <class T>
__global__ void k_mg_prolong(long long N, int nx, int ny, T* __restrict__ xf, const MGLev C, T omega,
                             const SolveScal* sc) {
    if (sc->done) return;
    prolong_level<T>(N, nx, ny, xf, C, omega, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                     (long long)gridDim.x * blockDim.x);
}

// Coarsest level (at most 1024 cells, one block of 1024 threads, one cell per thread): `sweeps`
// red-black passes then as many black-red (a symmetric operator).  Each thread keeps its links and
// right-hand side in registers; the iterate lives in shared memory.
template <class T>
__device__ __forceinline__ void coarsest_solve(const MGLev& L, int sweeps, T* xs) {
    const long long q = threadIdx.x;
    const bool act = q < L.N;
    int col = 0;
    float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, inv = 0.f;
    int nb[6] = {0, 0, 0, 0, 0, 0};
    T bq = 0;
    if (act) {
        int c[3];
        coords3(q, L.nx, L.ny, c);
        col = (c[0] + c[1] + c[2]) & 1;
        long long off[6];
        coarse_links(L, q, c, g, off);
#pragma unroll
        for (int e = 0; e < 6; ++e) nb[e] = (int)(q + off[e]);
        inv = L.invdg[q];
        bq = ((const T*)L.b)[q];
    }
    xs[threadIdx.x] = (T)0;
    __syncthreads();
    for (int pass = 0; pass < 4 * sweeps; ++pass) {
        const int half = pass / (2 * sweeps);                 // 0: red-black order, 1: black-red
        const int want = ((pass & 1) ^ half);
        if (act && col == want && inv != 0.f) {
            T s = 0;
#pragma unroll
            for (int e = 0; e < 6; ++e)
                if (g[e] != 0.f) s += (T)g[e] * xs[nb[e]];
            xs[threadIdx.x] = (s - bq) * (T)inv;
        }
        __syncthreads();
    }
    if (act) ((T*)L.x)[q] = xs[threadIdx.x];
}

template <class T>
__global__ void __launch_bounds__(1024) k_mg_coarsest(MGLev L, int sweeps, const SolveScal* sc) {
    if (sc->done) return;
    __shared__ T xs[1024];
    coarsest_solve<T>(L, sweeps, xs);
}

// The small levels first .. nlev-1 of a V-cycle in one launch: one cluster of MG_TAIL_CTAS blocks of
// 1024 threads walks the descent (smoothing, restriction), the coarsest solve (block 0) and the
// ascent (prolongation, smoothing), with a cluster barrier (hardware, release/acquire at cluster
// scope) between dependent passes.  These levels are a few MB at most and stay in L2; as separate
// kernels each pass would cost a launch for a few microseconds of work.
template <class T>
__global__ void __launch_bounds__(1024) k_mg_tail(MGTail M, const SolveScal* sc) {
    if (sc->done) return;                       // the flag is uniform: set by an earlier kernel
    __shared__ T xs[1024];
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
            smooth_level<T>(M.lev[l], 0, q == 0, t0, nt);
            bar();
            smooth_level<T>(M.lev[l], 1, false, t0, nt);
            bar();
        }
        restrict_level<T>(M.lev[l], M.lev[l + 1], t0, nt);
        bar();
    }
    if (cl.block_rank() == 0) coarsest_solve<T>(M.lev[last], M.coarse_sweeps, xs);
    bar();
    for (int l = last - 1; l >= M.first; --l) {
        const MGLev& F = M.lev[l];
        prolong_level<T>(F.N, F.nx, F.ny, (T*)F.x, M.lev[l + 1], (T)M.omega, t0, nt);
        bar();
        for (int q = 0; q < M.sweeps; ++q) {
            smooth_level<T>(F, 1, false, t0, nt);
            bar();
            smooth_level<T>(F, 0, false, t0, nt);
            bar();
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

unsigned lin_blocks(long long n) {
    long long b = (n + 255) / 256;
    long long cap = 8LL * IBM_NSM;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

int mg_levels_for(int nx, int ny, int nz, int dims[][3], int maxlev) {
    int n = 0;
    int d[3] = {nx, ny, nz};
    for (;;) {
        dims[n][0] = d[0];
        dims[n][1] = d[1];
        dims[n][2] = d[2];
        ++n;
        const long long cells = (long long)d[0] * d[1] * d[2];
        if (n == maxlev || cells <= 1024 || (d[0] == 1 && d[1] == 1 && d[2] == 1)) break;
        for (int a = 0; a < 3; ++a) d[a] = (d[a] + 1) / 2;
    }
    return n;
}

int mg_setup(const LesCtx& c, MG& mg, cudaStream_t s) {
    if (mg.nlev < 2) return IBM_OK;
    k_mg_build1<<<lin_blocks(mg.lev[1].N), 256, 0, s>>>(c.D, mg.lev[1]);
    for (int l = 1; l + 1 < mg.nlev; ++l)
        k_mg_build_next<<<lin_blocks(mg.lev[l + 1].N), 256, 0, s>>>(mg.lev[l], mg.lev[l + 1]);
    for (int l = 1; l < mg.nlev; ++l) k_mg_invdiag<<<lin_blocks(mg.lev[l].N), 256, 0, s>>>(mg.lev[l]);
    IBM_LAUNCHED("mg_setup");
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
        prof_begin(c.prof, PS_MG_TRANSFER, s);
        if constexpr (std::is_same<T, float>::value) {
            if (vec) launch_mg_restrict0_x4(c, r, z, scale, mg.lev[1], sc, s);
            else k_mg_restrict0<T><<<lin_blocks(mg.lev[1].N), 256, 0, s>>>(c.D, r, z, scale, mg.lev[1], sc);
        } else {
            k_mg_restrict0<T><<<lin_blocks(mg.lev[1].N), 256, 0, s>>>(c.D, r, z, scale, mg.lev[1], sc);
        }
        prof_end(c.prof, PS_MG_TRANSFER, s);
        ++launches;
        prof_begin(c.prof, PS_MG_COARSE, s);
        // levels >= tf (if any) run in one cluster launch; separate kernels above them
        int tf = mg.nlev;
        for (int l = 1; l + 1 < mg.nlev; ++l)
            if (mg.lev[l].N <= MG_TAIL_MAX_CELLS) { tf = l; break; }
        const int top = tf < mg.nlev ? tf : mg.nlev - 1;
        for (int l = 1; l < top; ++l) {
            const MGLev& L = mg.lev[l];
            for (int q = 0; q < SC; ++q) {
                k_mg_smoothc<T><<<lin_blocks((L.N + 1) / 2), 256, 0, s>>>(L, 0, q == 0, sc);
                k_mg_smoothc<T><<<lin_blocks((L.N + 1) / 2), 256, 0, s>>>(L, 1, 0, sc);
                launches += 2;
            }
            k_mg_restrictc<T><<<lin_blocks(mg.lev[l + 1].N), 256, 0, s>>>(L, mg.lev[l + 1], sc);
            ++launches;
        }
        if (tf < mg.nlev) {
            MGTail M;
            for (int l = 0; l < mg.nlev; ++l) M.lev[l] = mg.lev[l];
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
            k_mg_coarsest<T><<<1, 1024, 0, s>>>(mg.lev[mg.nlev - 1], mg.coarse_sweeps, sc);
            ++launches;
        }
        for (int l = top - 1; l >= 1; --l) {
            const MGLev& L = mg.lev[l];
            k_mg_prolong<T><<<lin_blocks(L.N), 256, 0, s>>>(L.N, L.nx, L.ny, (T*)L.x, mg.lev[l + 1], om, sc);
            ++launches;
            for (int q = 0; q < SC; ++q) {
                k_mg_smoothc<T><<<lin_blocks((L.N + 1) / 2), 256, 0, s>>>(L, 1, 0, sc);
                k_mg_smoothc<T><<<lin_blocks((L.N + 1) / 2), 256, 0, s>>>(L, 0, 0, sc);
                launches += 2;
            }
        }
        prof_end(c.prof, PS_MG_COARSE, s);
        prof_begin(c.prof, PS_MG_TRANSFER, s);
        k_mg_prolong<T><<<lin_blocks(c.D.N), 256, 0, s>>>(c.D.N, c.D.nx, c.D.ny, z, mg.lev[1], om, sc);
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

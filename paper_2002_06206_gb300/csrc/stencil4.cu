// stencil4.cu -- FP32 fine-grid stencil kernels that give each thread 4 consecutive cells along x:
// one 16-byte load per array and row instead of four 4-byte loads, and one set of index arithmetic
// per 4 cells.  They compute exactly what the per-cell kernels compute (the 7-point link sum of
// Eq. poisson with Neumann cut links and p = 0 outflow faces) and are used when nx is a multiple of 4,
// so that every row starts on a 16-byte boundary.
#include "solver.cuh"

namespace {

#define X4_TX 32     // threads along x (128 cells)
#define X4_TY 8

// Persistent launch: a fixed number of blocks walks the (x, y, z) tiles of the grid, so that a kernel
// ending in a grid reduction pays the reduction tail once per block, not once per wave of tiles.
// Tile indices are 32-bit (a grid has fewer than 2^31 cells): a 64-bit division per tile would cost
// more than the tile's arithmetic.
#define X4_TILE_LOOP_BEGIN                                                                      \
    const unsigned gx_ = (D.nx / 4 + X4_TX - 1) / X4_TX, gy_ = (D.ny + X4_TY - 1) / X4_TY;     \
    const unsigned ntiles_ = gx_ * gy_ * (unsigned)((D.nz + IBM_KU - 1) / IBM_KU);             \
    for (unsigned tile_ = blockIdx.x; tile_ < ntiles_; tile_ += gridDim.x) {                   \
        const unsigned r_ = tile_ / gx_;                                                       \
        const int bx_ = (int)(tile_ - r_ * gx_), by_ = (int)(r_ % gy_), bz_ = (int)(r_ / gy_); \
        const int i0 = 4 * (bx_ * X4_TX + threadIdx.x), j = by_ * X4_TY + threadIdx.y;         \
        const int kb = bz_ * IBM_KU;                                                           \
        const bool active = i0 < D.nx && j < D.ny;
#define X4_TILE_LOOP_END }

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float el(const float4& v, int m) { return m == 0 ? v.x : (m == 1 ? v.y : (m == 2 ? v.z : v.w)); }

// The chunk [i0, i0 + 4) of row (j, k) has no cut link and all its neighbours inside the domain.
__device__ __forceinline__ bool plain_chunk(const Dom& D, int i0, int j, int k, unsigned fl4) {
    return fl4 == 0u && i0 > 0 && i0 + 4 < D.nx && j > 0 && j < D.ny - 1 && k > 0 && k < D.nz - 1;
}

__device__ __forceinline__ unsigned flags4(const Dom& D, long long P) {
    return D.flags ? *reinterpret_cast<const unsigned*>(D.flags + P) : 0u;
}

// CG first half (see poisson.cu): p = src + beta p_old, q = A p, (p, q).
__global__ void __launch_bounds__(256, 4) k_cg_dir_spmv_x4(Dom D, const float* __restrict__ r,
                                                        const float* __restrict__ pold, float* __restrict__ pnew,
                                                        float* __restrict__ q, float idx2, SolveScal* sc,
                                                        double* partials, unsigned* counter, int pcg) {
    if (sc->done) return;
    const float beta = sc->restart ? 0.f : (float)(pcg ? sc->rz / sc->rz_old : sc->rr / sc->rr_old);
    float part = 0.f;
    auto pv = [&](long long c) { return r[c] + beta * pold[c]; };
    X4_TILE_LOOP_BEGIN
#pragma unroll
    for (int u = 0; u < IBM_KU; ++u) {
        const int k = kb + u;
        if (!active || k >= D.nz) continue;
        const long long P = i0 + (long long)D.sy * j + D.sz * k;
        const unsigned fl4 = flags4(D, P);
        const float4 r4 = ld4(r + P), o4 = ld4(pold + P);
        float pc[4] = {r4.x + beta * o4.x, r4.y + beta * o4.y, r4.z + beta * o4.z, r4.w + beta * o4.w};
        float qv[4];
        if (plain_chunk(D, i0, j, k, fl4)) {
            const float4 ym = ld4(r + P - D.sy), ymo = ld4(pold + P - D.sy);
            const float4 yp = ld4(r + P + D.sy), ypo = ld4(pold + P + D.sy);
            const float4 zm = ld4(r + P - D.sz), zmo = ld4(pold + P - D.sz);
            const float4 zp = ld4(r + P + D.sz), zpo = ld4(pold + P + D.sz);
            const float xl = pv(P - 1), xr = pv(P + 4);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float xm = m == 0 ? xl : pc[m - 1];
                const float xp = m == 3 ? xr : pc[m + 1];
                const float yy = (el(ym, m) + beta * el(ymo, m)) + (el(yp, m) + beta * el(ypo, m));
                const float zz = (el(zm, m) + beta * el(zmo, m)) + (el(zp, m) + beta * el(zpo, m));
                qv[m] = ((xm + xp) + yy + zz - 6.f * pc[m]) * idx2;
            }
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const unsigned fl = (fl4 >> (8 * m)) & 0xffu;
                qv[m] = link_sum7<float>(D, P + m, i0 + m, j, k, fl, pc[m], pv) * idx2;
            }
        }
        st4(pnew + P, make_float4(pc[0], pc[1], pc[2], pc[3]));
        st4(q + P, make_float4(qv[0], qv[1], qv[2], qv[3]));
        part += (pc[0] * qv[0] + pc[1] * qv[1]) + (pc[2] * qv[2] + pc[3] * qv[3]);
    }
    X4_TILE_LOOP_END
    decltype(part) acc[1] = {part};
    grid_reduce<1>(acc, partials, counter, [&](double* t) { sc->pq = t[0]; });
}

// Gauss-Seidel value of one fine cell in the generic case (cut links or domain faces).
__device__ __forceinline__ float gs_generic(const Dom& D, const float* r, const float* z, float scale, long long P,
                                            int i, int j, int k, unsigned fl, bool zero) {
    const int x[3] = {i, j, k};
    float s = 0.f, dg = 0.f;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        const int a = b >> 1, sd = (b & 1) ? 1 : -1;
        long long o = 0;
        const bool in = nb_offset(D, a, sd, x[a], o);
        if (!(fl & (1u << b)) && in) {
            dg += 1.f;
            if (!zero) s += z[P + o];
        } else if (!in && D.bc[b] == IBM_BC_OUTFLOW) {
            dg += 2.f;
        }
    }
    return dg == 0.f ? 0.f : (s - scale * r[P]) / dg;
}

// Gauss-Seidel update of cells C0 and C0 + 2 of a plain chunk (compile-time positions, so every
// element access is a register).
template <int C0>
__device__ __forceinline__ void gs_plain(float (&zc)[4], const float4& r4, const float* z, long long P, const Dom& D,
                                         float scale, bool zero) {
    const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
    if (zero) {
        zc[C0] = -scale * rr[C0] * (1.f / 6.f);
        zc[C0 + 2] = -scale * rr[C0 + 2] * (1.f / 6.f);
        return;
    }
    const float4 ym4 = ld4(z + P - D.sy), yp4 = ld4(z + P + D.sy);
    const float4 zm4 = ld4(z + P - D.sz), zp4 = ld4(z + P + D.sz);
    const float ym[4] = {ym4.x, ym4.y, ym4.z, ym4.w}, yp[4] = {yp4.x, yp4.y, yp4.z, yp4.w};
    const float zm[4] = {zm4.x, zm4.y, zm4.z, zm4.w}, zp[4] = {zp4.x, zp4.y, zp4.z, zp4.w};
    const float xl = C0 == 0 ? z[P - 1] : 0.f, xr = C0 == 1 ? z[P + 4] : 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int m = C0 + 2 * h;
        const float xm = m == 0 ? xl : zc[m - 1];
        const float xp = m == 3 ? xr : zc[m + 1];
        const float s = ((xm + xp) + (ym[m] + yp[m])) + (zm[m] + zp[m]);
        zc[m] = (s - scale * rr[m]) * (1.f / 6.f);
    }
}

// One red-black pass of colour `col` (see mg.cu), 4 cells per thread: the cells of the other colour
// are read and written back unchanged, which no other thread modifies during the pass.  With `fin`
// this is the last pass of the V-cycle (colour 0) and (r, z) over all cells is reduced as well.
__global__ void __launch_bounds__(256, 4) k_mg_smooth0_x4(Dom D, const float* __restrict__ r, float* z, float scale,
                                                       int col, int zero, int fin, SolveScal* sc, double* partials,
                                                       unsigned* counter) {
    if (sc->done) return;
    float part = 0.f;
    X4_TILE_LOOP_BEGIN
#pragma unroll
    for (int u = 0; u < IBM_KU; ++u) {
        const int k = kb + u;
        if (!active || k >= D.nz) continue;
        const long long P = i0 + (long long)D.sy * j + D.sz * k;
        const unsigned fl4 = flags4(D, P);
        const float4 r4 = ld4(r + P);
        float zc[4];
        const int c0 = (i0 + j + k + col) & 1;       // m with (i0 + m + j + k) % 2 == col: m = c0, c0 + 2
        if (zero) {
            zc[0] = zc[1] = zc[2] = zc[3] = 0.f;
        } else {
            const float4 z4 = ld4(z + P);
            zc[0] = z4.x; zc[1] = z4.y; zc[2] = z4.z; zc[3] = z4.w;
        }
        if (plain_chunk(D, i0, j, k, fl4)) {
            // the colour's two cells are m = c0 and c0 + 2; c0 is uniform across a warp (same j, k)
            if (c0 == 0) gs_plain<0>(zc, r4, z, P, D, scale, zero != 0);
            else gs_plain<1>(zc, r4, z, P, D, scale, zero != 0);
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = c0 + 2 * h;
                const unsigned fl = (fl4 >> (8 * m)) & 0xffu;
                const float g = gs_generic(D, r, z, scale, P + m, i0 + m, j, k, fl, zero != 0);
                if (m == 0) zc[0] = g;
                else if (m == 1) zc[1] = g;
                else if (m == 2) zc[2] = g;
                else zc[3] = g;
            }
        }
        st4(z + P, make_float4(zc[0], zc[1], zc[2], zc[3]));
        if (fin) part += (r4.x * zc[0] + r4.y * zc[1]) + (r4.z * zc[2] + r4.w * zc[3]);
    }
    X4_TILE_LOOP_END
    decltype(part) acc[1] = {part};
    if (fin)
        grid_reduce<1>(acc, partials, counter, [&](double* t) {
            sc->rz_old = sc->rz;
            sc->rz = t[0];
        });
}

}  // namespace

bool x4_ok(const LesCtx& c) { return (c.D.nx % 4) == 0; }

dim3 x4_grid(const LesCtx& c) {
    const long long tiles = (long long)((c.D.nx / 4 + X4_TX - 1) / X4_TX) * ((c.D.ny + X4_TY - 1) / X4_TY) *
                            ((c.D.nz + IBM_KU - 1) / IBM_KU);
    const long long cap = 4LL * IBM_NSM;      // resident blocks of 256 threads at <= 64 registers
    return dim3((unsigned)(tiles < cap ? tiles : cap));
}

void launch_cg_dir_spmv_x4(const LesCtx& c, const float* src, const float* pold, float* pnew, float* q, float idx2,
                           SolveScal* sc, int pcg, cudaStream_t s) {
    k_cg_dir_spmv_x4<<<x4_grid(c), dim3(X4_TX, X4_TY), 0, s>>>(c.D, src, pold, pnew, q, idx2, sc, c.partials,
                                                               c.counter, pcg);
}

void launch_mg_smooth0_x4(const LesCtx& c, const float* r, float* z, float scale, int col, int zero, int fin,
                          SolveScal* sc, cudaStream_t s) {
    k_mg_smooth0_x4<<<x4_grid(c), dim3(X4_TX, X4_TY), 0, s>>>(c.D, r, z, scale, col, zero, fin, sc, c.partials,
                                                              c.counter);
}

// les.cu -- the per-step stencil kernels of the immersed-boundary LES (Sec. 2.1-2.4): CSM eddy
// viscosity, the momentum flux with the QUICK hybrid and its two predictors (Crank-Nicolson with a
// BiCGStab momentum solve, Adams-Bashforth 2), distributed direct forcing, face velocities, Poisson
// right-hand side, velocity correction, and the Shepard surface and viscous forces.
//
// Cell kernels use a 32 x 8 thread tile over (x, y) so that consecutive threads touch consecutive
// cells (coalesced rows); the momentum flux walks z-marching tiles staged in shared memory, with the
// cells next to cut links in a separate general kernel.
#include "solver.cuh"

#ifndef IBM_FLUX_GEN_MINB
#define IBM_FLUX_GEN_MINB 4   // the general-cell flux kernels gather from global memory: occupancy pays for small spills
#endif
#ifndef IBM_FLUX_MINB
#define IBM_FLUX_MINB 3
#endif

namespace {

template <class T>
__device__ __forceinline__ void grad_at(const Dom& D, const T* __restrict__ u, long long P, const int x[3],
                                        unsigned fl, T inv2dx, T G[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T up = vel_across(D, u, b, P, x[a], fl, a, +1);
            const T um = vel_across(D, u, b, P, x[a], fl, a, -1);
            G[a][b] = (up - um) * inv2dx;
        }
}

__device__ __forceinline__ unsigned flags_at(const Dom& D, long long P) { return D.flags ? (unsigned)D.flags[P] : 0u; }

// Eq. Smagorinsky with the coherent-structure coefficient of Eq. Q / Eq. FCS.  One thread per cell.
template <class T>
__global__ void __launch_bounds__(256) k_csm(Dom D, const T* __restrict__ u, T* __restrict__ nut) {
    const int i = blockIdx.x * IBM_TX + threadIdx.x, j = blockIdx.y * IBM_TY + threadIdx.y, k = blockIdx.z;
    if (i >= D.nx || j >= D.ny) return;
    const T inv2dx = (T)0.5 * dom_idx<T>(D), delta2 = dom_dx<T>(D) * dom_dx<T>(D);
    const long long P = i + (long long)D.sy * j + D.sz * k;
    const unsigned fl = flags_at(D, P);
    const int x[3] = {i, j, k};
    T G[3][3];
    if (fl == 0u && i > 0 && i < D.nx - 1 && j > 0 && j < D.ny - 1 && k > 0 && k < D.nz - 1) {
        const long long o[3] = {1, (long long)D.sy, D.sz};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) G[a][b] = (u[b * D.N + P + o[a]] - u[b * D.N + P - o[a]]) * inv2dx;
    } else {
        grad_at(D, u, P, x, fl, inv2dx, G);
    }
    T SS = 0, WW = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T S = (T)0.5 * (G[a][b] + G[b][a]);
            const T W = (T)0.5 * (G[a][b] - G[b][a]);
            SS += S * S;
            WW += W * W;
        }
    const T Q = (T)0.5 * (WW - SS), E = (T)0.5 * (WW + SS);
    const T F = E > (T)0 ? Q / E : (T)0;
    const T aF = F < (T)0 ? -F : F;
    const T C = (T)(1.0 / 20.0) * (aF * sqrt(aF));
    nut[P] = C * delta2 * sqrt(SS);
}

// Advected value on the face of P towards side s along axis a: the central value blended with a
// fraction gam of QUICK (6 upwind + 3 downwind - far upwind)/8, the far upwind value read across the
// upwind cell's outer link.  L and R are the lower and upper cells of the face, so both cells of a face
// compute the same value.  Cut faces and domain faces keep the central value.
template <class T>
__device__ __forceinline__ T face_adv(const Dom& D, const T* __restrict__ u, int c, long long P, const int x[3],
                                      unsigned fl, int a, int s, T uP, T uN, T Uf, T gam) {
    const T central = (T)0.5 * (uP + uN);
    if (gam == (T)0) return central;
    long long off;
    if ((fl & (1u << (2 * a + (s > 0)))) || !nb_offset(D, a, s, x[a], off)) return central;
    const int n = a == 0 ? D.nx : (a == 1 ? D.ny : D.nz);
    const long long Nn = P + off;
    const long long Lc = s > 0 ? P : Nn, Rc = s > 0 ? Nn : P;
    const int xo = x[a] + s < 0 ? n - 1 : (x[a] + s >= n ? 0 : x[a] + s);
    const int xL = s > 0 ? x[a] : xo, xR = s > 0 ? xo : x[a];
    const T uL = s > 0 ? uP : uN, uR = s > 0 ? uN : uP;
    T q;
    if (Uf >= (T)0) {
        const T far = vel_across(D, u, c, Lc, xL, D.flags ? (unsigned)D.flags[Lc] : 0u, a, -1);
        q = ((T)6 * uL + (T)3 * uR - far) / (T)8;
    } else {
        const T far = vel_across(D, u, c, Rc, xR, D.flags ? (unsigned)D.flags[Rc] : 0u, a, +1);
        q = ((T)6 * uR + (T)3 * uL - far) / (T)8;
    }
    return ((T)1 - gam) * central + gam * q;
}

// L(u) of a cell per unit volume: flux-form advection with the face velocity U (central value
// blended with QUICK), diffusion with nu + nu_t, the transpose part of the SGS stress divergence.
// flux_general applies the ghost and boundary rules of vel_across on every link; the tiled fast path
// evaluates the same formulas for a cell where they reduce to direct reads (fast_cell).  With D.hom set
// the ghost values lose their wall and inflow velocities, which gives the linear part of L.

// The cell and its six neighbours (across periodic seams too) have no cut link: its flux then needs
// only neighbour values and the domain-boundary ghosts, which the tiles below hold.
__device__ __forceinline__ bool fast_cell(const Dom& D, long long P, int i, int j, int k) {
    if (!D.flags) return true;
    const uint8_t* f = D.flags;
    unsigned m = f[P];
    const int x[3] = {i, j, k};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            long long off;
            if (nb_offset(D, a, s, x[a], off)) m |= f[P + off];
        }
    return (m & 63u) == 0u;
}

// Fast cells run in z-marching tiles: a block of 32 x 8 threads owns an (x, y) tile and walks FT_KZ
// planes; u (three components) and nu_t of the planes k-2 .. k+2 over the tile plus a two-cell halo
// sit in a five-plane ring in shared memory, so every neighbour read of the flux is a shared-memory
// load at a fixed offset.  Halo positions across a periodic seam hold the wrapped cell; one cell
// beyond a non-periodic domain face they hold the boundary ghost of vel_across (a function of the
// cell across that face alone), so cells on the domain faces are fast too.  Links through a domain
// face take the boundary forms of flux_general (near-cell nu_t and cross derivative, central advected
// value).  Cells that are not fast_cell are skipped (the general kernel takes them).
//
// The flux form is conservative: the face between L and R = L + e_a gives L the term Phi and R the
// term -Phi, so the march evaluates every face once.  Each thread takes its cell's -x, -y and +z
// faces (two warps add the tile's last x column and y row); the x and y faces meet in shared memory,
// the z face stays in registers for the next plane.  A plane's sums run one step later, so a single
// barrier per plane orders both the face buffers (two of them, by plane parity) and the ring.
#define FT_X 32
#define FT_Y 8
#define FT_H 2
#define FT_SX (FT_X + 2 * FT_H)
#define FT_SY (FT_Y + 2 * FT_H)
#define FT_PL (FT_SX * FT_SY)
#define FT_NV 4
#define FT_KZ 16
#define FT_RING 6
#define FT_FXN (FT_Y * (FT_X + 1))   // x faces of a tile plane, per component
#define FT_FYN ((FT_Y + 1) * FT_X)   // y faces

// Domain-boundary ghost of component c across face (a, s) of the cell holding v (vel_across's rules).
template <class T>
__device__ __forceinline__ T bc_ghost(const Dom& D, int a, int s, int c, T v) {
    switch (D.bc[2 * a + (s > 0)]) {
        case IBM_BC_INFLOW: return (D.hom ? (T)0 : (T)2 * (T)D.u_in[c]) - v;
        case IBM_BC_OUTFLOW: return v;
        case IBM_BC_SLIP: return c == a ? -v : v;
        default: return -v;
    }
}

// Phi of the face between L = R - e_A and R, per component: the term of L's flux sum (R takes -Phi).
// S[d] is ring plane k + d - 2; R sits at in-plane ring index c0 of plane k + ZR and at global (g0, g1,
// g2), g_A = 0 .. n_A naming the face.  A face on a non-periodic domain side (R or L outside) takes the
// boundary forms of the cell inside.  Positions outside the domain give unused values (U reads 0).
template <class T, int A, int ZR>
__device__ __forceinline__ void ft_face(const Dom& D, const FaceLayout& F, const T* __restrict__ U,
                                        const T* const (&S)[5], int c0, int g0, int g1, int g2, T nu, T gam,
                                        T inv2dx, T invdx, T (&phi)[3]) {
    constexpr int EX = A == 0, EY = A == 1, EZ = A == 2;
    // variable v at R + (dx, dy, dz)
    auto V = [&](int v, int dx, int dy, int dz) -> T { return S[ZR + 2 + dz][v * FT_PL + c0 + dy * FT_SX + dx]; };
    const int g[3] = {g0, g1, g2}, n[3] = {D.nx, D.ny, D.nz};
    const bool per = D.bc[2 * A] == IBM_BC_PERIODIC;
    const bool dlo = !per && g[A] == 0, dhi = !per && g[A] == n[A];
    bool valid = g[A] >= 0 && g[A] <= n[A];
#pragma unroll
    for (int b = 0; b < 3; ++b)
        if (b != A) valid = valid && g[b] >= 0 && g[b] < n[b];
    const T Uf = valid ? U[F.index(A, g0, g1, g2)] : (T)0;
    const T nutL = V(3, -EX, -EY, -EZ), nutR = V(3, 0, 0, 0);
    const T nutf = dlo ? nutR : (dhi ? nutL : (T)0.5 * (nutL + nutR));
    const T nuf = nu + nutf;
    const bool quick = gam != (T)0 && !dlo && !dhi;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T uL = V(c, -EX, -EY, -EZ), uR = V(c, 0, 0, 0);
        const T D1 = (uR - uL) * invdx;
        T Tt = D1;
        if (c != A) {
            // d u_A / d x_c at L and at R (central)
            const int cx = c == 0, cy = c == 1, cz = c == 2;
            const T gL = (V(A, cx - EX, cy - EY, cz - EZ) - V(A, -cx - EX, -cy - EY, -cz - EZ)) * inv2dx;
            const T gR = (V(A, cx, cy, cz) - V(A, -cx, -cy, -cz)) * inv2dx;
            Tt = dlo ? gR : (dhi ? gL : (T)0.5 * (gL + gR));
        }
        T adv = (T)0.5 * (uL + uR);
        if (quick) {
            // far upwind: L - e_A for U >= 0, R + e_A otherwise
            const bool up = Uf >= (T)0;
            const T far = up ? V(c, -2 * EX, -2 * EY, -2 * EZ) : V(c, EX, EY, EZ);
            const T q = up ? ((T)6 * uL + (T)3 * uR - far) / (T)8 : ((T)6 * uR + (T)3 * uL - far) / (T)8;
            adv = ((T)1 - gam) * adv + gam * q;
        }
        phi[c] = -Uf * adv + nuf * D1 + nutf * Tt;
    }
}

template <class T, class Epi>
__device__ __forceinline__ void fast_tile_march(const Dom& D, const FaceLayout& F, const T* __restrict__ u,
                                                const T* __restrict__ U, const T* __restrict__ nut, T nu, T gam,
                                                Epi epi) {
    extern __shared__ __align__(16) unsigned char ft_raw[];
    T* sm = reinterpret_cast<T*>(ft_raw);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + FT_X * ty;
    const T inv2dx = (T)0.5 * dom_idx<T>(D), invdx = dom_idx<T>(D);
    auto slot = [](int kk) { return ((kk % FT_RING) + FT_RING) % FT_RING; };
    const int n[3] = {D.nx, D.ny, D.nz};
    const int gx = (D.nx + FT_X - 1) / FT_X, gy = (D.ny + FT_Y - 1) / FT_Y, gz = (D.nz + FT_KZ - 1) / FT_KZ;
    const long long items = (long long)gx * gy * gz;
    // the planes' values a thread stages: FT_PL <= 2 * 256 halo-tile positions per plane
    T pf[2][FT_NV];
    int x0 = 0, y0 = 0;
    // the thread's halo-tile positions (fixed) and whether the tile's halo box lies inside the domain
    // in x and y (then a plane inside the domain needs no boundary logic)
    const int ex0 = tid % FT_SX - FT_H, ey0 = tid / FT_SX - FT_H;
    const int ex1 = (tid + FT_X * FT_Y) % FT_SX - FT_H, ey1 = (tid + FT_X * FT_Y) / FT_SX - FT_H;
    bool inner = false;
    auto fetch = [&](int kk) {
        if (inner && kk >= 0 && kk < D.nz) {
            const long long base = x0 + (long long)D.sy * y0 + D.sz * kk;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int e = tid + t * (FT_X * FT_Y);
                pf[t][0] = pf[t][1] = pf[t][2] = pf[t][3] = (T)0;
                if (e >= FT_PL) continue;
                const long long c = base + (t ? ex1 : ex0) + (long long)D.sy * (t ? ey1 : ey0);
                pf[t][0] = u[c];
                pf[t][1] = u[D.N + c];
                pf[t][2] = u[2 * D.N + c];
                pf[t][3] = nut[c];
            }
            return;
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int e = tid + t * (FT_X * FT_Y);
            pf[t][0] = pf[t][1] = pf[t][2] = pf[t][3] = (T)0;
            if (e >= FT_PL) continue;
            int g[3] = {x0 + e % FT_SX - FT_H, y0 + e / FT_SX - FT_H, kk};
            int out = 0, oa = 0, os = 0, depth = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (g[a] >= 0 && g[a] < n[a]) continue;
                if (D.bc[2 * a] == IBM_BC_PERIODIC) {
                    g[a] = ((g[a] % n[a]) + n[a]) % n[a];
                    continue;
                }
                ++out;
                oa = a;
                os = g[a] < 0 ? -1 : 1;
                depth = g[a] < 0 ? -g[a] : g[a] - n[a] + 1;
                g[a] = g[a] < 0 ? 0 : n[a] - 1;
            }
            // corners and second ghost layers are never read by a fast cell
            if (out > 1 || depth > 1 || g[0] < 0 || g[0] >= n[0] || g[1] < 0 || g[1] >= n[1] || g[2] < 0 ||
                g[2] >= n[2])
                continue;
            const long long c = g[0] + (long long)D.sy * g[1] + D.sz * g[2];
            T v0 = u[c], v1 = u[D.N + c], v2 = u[2 * D.N + c];
            if (out) {
                v0 = bc_ghost(D, oa, os, 0, v0);
                v1 = bc_ghost(D, oa, os, 1, v1);
                v2 = bc_ghost(D, oa, os, 2, v2);
            }
            pf[t][0] = v0;
            pf[t][1] = v1;
            pf[t][2] = v2;
            pf[t][3] = nut[c];
        }
    };
    auto commit = [&](int kk) {
        T* dst = sm + slot(kk) * (FT_NV * FT_PL);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int e = tid + t * (FT_X * FT_Y);
            if (e >= FT_PL) continue;
#pragma unroll
            for (int v = 0; v < FT_NV; ++v) dst[v * FT_PL + e] = pf[t][v];
        }
    };
    const int cidx = (ty + FT_H) * FT_SX + (tx + FT_H);
    T* const fxs = sm + FT_RING * FT_NV * FT_PL;     // [parity][component][FT_Y][FT_X + 1]
    T* const fys = fxs + 2 * 3 * FT_FXN;               // [parity][component][FT_Y + 1][FT_X]
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        x0 = (int)(item % gx) * FT_X;
        y0 = (int)((item / gx) % gy) * FT_Y;
        inner = x0 >= FT_H && x0 + FT_X + FT_H <= D.nx && y0 >= FT_H && y0 + FT_Y + FT_H <= D.ny;
        const int z0 = (int)(item / ((long long)gx * gy)) * FT_KZ;
        const int z1 = z0 + FT_KZ < D.nz ? z0 + FT_KZ : D.nz;
        for (int kk = z0 - 2; kk <= z0 + 2; ++kk) {
            fetch(kk);
            commit(kk);
        }
        if (z0 + 3 <= z1 + 1) fetch(z0 + 3);
        __syncthreads();
        const int i = x0 + tx, j = y0 + ty;
        const bool inxy = i < D.nx && j < D.ny;
        // the cell of the plane whose sums are pending: fast, index, u; its -z and +z faces
        bool pf_fast = false;
        long long pP = 0;
        T pu[3] = {0, 0, 0}, zlo[3] = {0, 0, 0}, zhi[3] = {0, 0, 0};
        int s0 = slot(z0 - 2);          // ring slot of plane k - 2, advanced with k (no division per cell)
        for (int k = z0; k <= z1; ++k, s0 = s0 + 1 == FT_RING ? 0 : s0 + 1) {
            // plane k + 3, fetched into registers during the previous step, goes into the ring slot that
            // plane k - 3 left (the previous barrier ended every read of it); then plane k + 4 is fetched,
            // so each load has a whole step and a barrier to land.  The barrier at the end of the step
            // publishes plane k + 3.
            if (k < z1 && k + 3 <= z1 + 1) {
                T* dst = sm + (s0 == 0 ? FT_RING - 1 : s0 - 1) * (FT_NV * FT_PL);   // slot of k - 3 = s0 - 1
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int e = tid + t * (FT_X * FT_Y);
                    if (e >= FT_PL) continue;
#pragma unroll
                    for (int v = 0; v < FT_NV; ++v) dst[v * FT_PL + e] = pf[t][v];
                }
                if (k + 4 <= z1 + 1) fetch(k + 4);
            }
            if (k > z0) {
                // sums of plane k - 1, whose faces the previous step wrote
                if (pf_fast) {
                    const int pb = (k - 1) & 1;
                    const T* fx = fxs + pb * 3 * FT_FXN + ty * (FT_X + 1) + tx;
                    const T* fy = fys + pb * 3 * FT_FYN + ty * FT_X + tx;
                    T h[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        h[c] = ((fx[c * FT_FXN + 1] - fx[c * FT_FXN]) + (fy[c * FT_FYN + FT_X] - fy[c * FT_FYN]) +
                                (zhi[c] - zlo[c])) * invdx;
                    epi(pP, h, pu);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) zlo[c] = zhi[c];
            }
            if (k == z1) break;
            const T* S[5];
#pragma unroll
            for (int d = 0; d < 5; ++d) {
                const int sd = s0 + d;
                S[d] = sm + (sd >= FT_RING ? sd - FT_RING : sd) * (FT_NV * FT_PL);
            }
            const long long P = i + (long long)D.sy * j + D.sz * k;
            pf_fast = inxy && (D.fast ? D.fast[P] != 0 : fast_cell(D, P, i, j, k));
            pP = P;
#pragma unroll
            for (int c = 0; c < 3; ++c) pu[c] = S[2][c * FT_PL + cidx];
            if (k == z0) ft_face<T, 2, 0>(D, F, U, S, cidx, i, j, k, nu, gam, inv2dx, invdx, zlo);
            ft_face<T, 2, 1>(D, F, U, S, cidx, i, j, k + 1, nu, gam, inv2dx, invdx, zhi);
            const int b = k & 1;
            T* fx = fxs + b * 3 * FT_FXN;
            T* fy = fys + b * 3 * FT_FYN;
            T ph[3];
            ft_face<T, 0, 0>(D, F, U, S, cidx, i, j, k, nu, gam, inv2dx, invdx, ph);
#pragma unroll
            for (int c = 0; c < 3; ++c) fx[c * FT_FXN + ty * (FT_X + 1) + tx] = ph[c];
            ft_face<T, 1, 0>(D, F, U, S, cidx, i, j, k, nu, gam, inv2dx, invdx, ph);
#pragma unroll
            for (int c = 0; c < 3; ++c) fy[c * FT_FYN + ty * FT_X + tx] = ph[c];
            if (ty == 0) {
                // the +y faces of the tile's last row
                ft_face<T, 1, 0>(D, F, U, S, (FT_Y + FT_H) * FT_SX + tx + FT_H, i, y0 + FT_Y, k, nu, gam, inv2dx,
                                 invdx, ph);
#pragma unroll
                for (int c = 0; c < 3; ++c) fy[c * FT_FYN + FT_Y * FT_X + tx] = ph[c];
            } else if (ty == 1 && tx < FT_Y) {
                // the +x faces of the tile's last column (row tx)
                ft_face<T, 0, 0>(D, F, U, S, (tx + FT_H) * FT_SX + FT_X + FT_H, x0 + FT_X, y0 + tx, k, nu, gam,
                                 inv2dx, invdx, ph);
#pragma unroll
                for (int c = 0; c < 3; ++c) fx[c * FT_FXN + tx * (FT_X + 1) + FT_X] = ph[c];
            }
            __syncthreads();
        }
    }
}

template <class T>
size_t fast_tile_smem() { return (size_t)(FT_RING * FT_NV * FT_PL + 2 * 3 * (FT_FXN + FT_FYN)) * sizeof(T); }

template <class T>
__device__ __forceinline__ void flux_general(const Dom& D, const FaceLayout& F, const T* __restrict__ u,
                                             const T* __restrict__ U, const T* __restrict__ nut, long long P, int i,
                                             int j, int k, T nu, T gam, T (&h)[3]) {
    const T inv2dx = (T)0.5 * dom_idx<T>(D), invdx = dom_idx<T>(D);
    const int n[3] = {D.nx, D.ny, D.nz};
    const unsigned fl = flags_at(D, P);
    const int x[3] = {i, j, k};
    const T nutP = nut[P];
    h[0] = h[1] = h[2] = (T)0;
        T GP[3][3];
        grad_at(D, u, P, x, fl, inv2dx, GP);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int s = -1; s <= 1; s += 2) {
                const int fx0 = x[0] + (a == 0 && s > 0), fx1 = x[1] + (a == 1 && s > 0), fx2 = x[2] + (a == 2 && s > 0);
                const T Uf = U[F.index(a, fx0, fx1, fx2)];
                const int bit = 2 * a + (s > 0);
                long long off = 0;
                const bool interior = !(fl & (1u << bit)) && nb_offset(D, a, s, x[a], off);
                T nutf = nutP;
                T GN[3] = {0, 0, 0};
                if (interior) {
                    const long long Nn = P + off;
                    nutf = (T)0.5 * (nutP + nut[Nn]);
                    int xn[3] = {x[0], x[1], x[2]};
                    xn[a] += s;
                    if (xn[a] < 0) xn[a] += n[a];
                    if (xn[a] >= n[a]) xn[a] -= n[a];
                    const unsigned fln = flags_at(D, Nn);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (q == a) continue;
                        GN[q] = (vel_across(D, u, a, Nn, xn[q], fln, q, +1) - vel_across(D, u, a, Nn, xn[q], fln, q, -1)) * inv2dx;
                    }
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T uP = u[c * D.N + P];
                    const T uN = vel_across(D, u, c, P, x[a], fl, a, s);
                    const T D1 = (uN - uP) * invdx;
                    T Tt;
                    if (c == a) Tt = D1;
                    else if (interior) Tt = (T)s * (T)0.5 * (GP[c][a] + GN[c]);
                    else Tt = (T)s * GP[c][a];
                    const T conv = -(T)s * Uf * face_adv(D, u, c, P, x, fl, a, s, uP, uN, Uf, gam);
                    h[c] += conv + (nu + nutf) * D1 + nutf * Tt;
                }
            }
    #pragma unroll
    for (int c = 0; c < 3; ++c) h[c] *= invdx;
}

// (grids hold fewer than 2^31 cells: 32-bit division)
__device__ __forceinline__ void cell_coords(const Dom& D, long long P, int& i, int& j, int& k) {
    const unsigned u = (unsigned)P, sy = (unsigned)D.sy, sz = (unsigned)D.sz;
    const unsigned kk = u / sz, r = u - kk * sz, jj = r / sy;
    k = (int)kk;
    j = (int)jj;
    i = (int)(r - jj * sy);
}

// Calls body(P, i, j, k) for the entries of the list of the cells that are not fast_cell, strided
// over a capped grid.
template <class Body>
__device__ __forceinline__ void for_general_cells(const Dom& D, const int32_t* __restrict__ list, long long nlist,
                                                  Body body) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nlist; q += (long long)gridDim.x * blockDim.x) {
        const long long P = list[q];
        int i, j, k;
        cell_coords(D, P, i, j, k);
        body(P, i, j, k);
    }
}

// Runs epi(P, h, u_P) over the kernel's cells: z-marching shared-memory tiles of fast cells, or the
// general list.
template <bool GENERAL, class T, class Epi>
__device__ __forceinline__ void flux_cells(const Dom& D, const FaceLayout& F, const T* __restrict__ u,
                                           const T* __restrict__ U, const T* __restrict__ nut, T nu, T gam,
                                           const int32_t* __restrict__ list, long long nlist, Epi epi) {
    if constexpr (GENERAL) {
        for_general_cells(D, list, nlist, [&](long long P, int i, int j, int k) {
            T h[3];
            flux_general(D, F, u, U, nut, P, i, j, k, nu, gam, h);
            const T uc[3] = {u[P], u[D.N + P], u[2 * D.N + P]};
            epi(P, h, uc);
        });
    } else {
        fast_tile_march<T>(D, F, u, U, nut, nu, gam, epi);
    }
}

// Momentum predictor, Adams-Bashforth 2 in time (Euler on the first step).  One thread per cell.
// Resident blocks of 256 threads per SM the fast FP32 flux kernels are compiled for (register cap).
template <class T, bool GENERAL>
struct FluxOcc {
    static constexpr int value = sizeof(T) == 4 ? (GENERAL ? IBM_FLUX_GEN_MINB : IBM_FLUX_MINB) : 1;
};

template <bool GENERAL, class T>
__global__ void __launch_bounds__(256, (FluxOcc<T, GENERAL>::value)) k_predict(Dom D, FaceLayout F, const T* __restrict__ u, const T* __restrict__ U,
                                                 const T* __restrict__ nut, const T* Hprev, T* H,
                                                 T* __restrict__ ustar, T nu, T dt, int first, T gam,
                                                 const int32_t* __restrict__ list, long long nlist) {
    flux_cells<GENERAL, T>(D, F, u, U, nut, nu, gam, list, nlist, [&](long long P, const T (&h)[3], const T (&uc)[3]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long oc = c * D.N + P;
            const T hc = h[c];
            const T hp = first ? (T)0 : Hprev[oc];
            H[oc] = hc;
            ustar[oc] = first ? uc[c] + dt * hc : uc[c] + dt * ((T)1.5 * hc - (T)0.5 * hp);
        }
    });
}

// Distributed direct forcing (Eq. forcing_term, Eq. discrete_forcing_term), gathered per Omega_inc
// cell over its own link records: the velocity at the wall point X is interpolated between the cell
// and the cell behind the wall, the force (u_IB - u_X)/dt is spread to the cell with the ghost branch
// (dx - d)/(dx + d) of Eq. distribution_function (the cell is a ghost of the stencil across the wall;
// weight 1 at d = 0 puts it on u_IB), and a cell whose weights add up to more than 1 takes their
// normalised sum.  All reads use the unforced u*, so the result does not depend on thread order.
template <class T>
__global__ void __launch_bounds__(256) k_forcing_gather(Dom D, const int32_t* __restrict__ inc, long long n_inc,
                                                        const T* __restrict__ us, double* __restrict__ delta, T dt,
                                                        int deadend_on, double vol, double* partials,
                                                        unsigned* counter, double* fscal) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n_inc; q += (long long)gridDim.x * blockDim.x) {
        const long long X = inc[q];
        const unsigned fl = D.flags[X];
        T d3[3] = {0, 0, 0};
        T wsum = 0;
        const bool dead = deadend_on && __popc(fl & 63u) >= 5;
        if (!dead) {
            for (int bit = 0; bit < 6; ++bit) {
                if (!((fl >> bit) & 1u)) continue;
                const LinkRec& r = link_record(D, X, fl, bit);
                const long long G = r.far;
                const T d = (T)r.d, wn = (T)r.w_ghost;
                wsum += wn;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T uX = ((T)1 - d) * us[c * D.N + X] + d * us[c * D.N + G];
                    const T Fc = ((T)r.uib[c] - uX) / dt;
                    d3[c] += dt * wn * Fc;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T dc = wsum > (T)1 ? d3[c] / wsum : d3[c];
            delta[3 * q + c] = (double)dc;
            acc[c] += (double)dc * vol;
        }
    }
    grid_reduce<3>(acc, partials, counter, [&](double* tot) {
        fscal[0] = tot[0];
        fscal[1] = tot[1];
        fscal[2] = tot[2];
    });
}

template <class T>
__global__ void k_forcing_apply(Dom D, const int32_t* __restrict__ inc, long long n_inc, const double* __restrict__ delta,
                                T* __restrict__ us) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n_inc; q += (long long)gridDim.x * blockDim.x) {
        const long long X = inc[q];
#pragma unroll
        for (int c = 0; c < 3; ++c) us[c * D.N + X] = us[c * D.N + X] + (T)delta[3 * q + c];
    }
}

__device__ __forceinline__ void face_coords(const FaceLayout& F, int a, long long idx, int x[3]) {
    x[0] = (int)(idx % F.dim[a][0]);
    long long t = idx / F.dim[a][0];
    x[1] = (int)(t % F.dim[a][1]);
    x[2] = (int)(t / F.dim[a][1]);
}

__device__ __forceinline__ long long cell_of(const Dom& D, const int x[3]) {
    return x[0] + (long long)D.sy * x[1] + D.sz * x[2];
}

// Normal velocity of the wall on a cut face between cells L and R along a: the mean of u_IB.e_a over
// the face's link records (L's +a record and, when present, R's -a record), in FP64.
__device__ __forceinline__ double cut_face_velocity(const Dom& D, long long L, long long R, int a) {
    const unsigned fL = D.flags[L], fR = D.flags[R];
    double sum = link_record(D, L, fL, 2 * a + 1).uib[a];
    double n = 1.0;
    if ((fR >> (2 * a)) & 1u) {
        sum += link_record(D, R, fR, 2 * a).uib[a];
        n = 2.0;
    }
    return sum / n;
}

// Face velocity of the intermediate field on the faces of axis a: the mean of the two cell values on
// uncut interior faces, the wall's normal velocity on cut faces (zero for a stationary body), the
// boundary value on domain faces.
template <class T>
__global__ void k_faces(Dom D, FaceLayout F, int a, const T* __restrict__ us, T* __restrict__ Us) {
    const long long nf = (long long)F.dim[a][0] * F.dim[a][1] * F.dim[a][2];
    const int na = a == 0 ? D.nx : (a == 1 ? D.ny : D.nz);
    const long long st = a == 0 ? 1 : (a == 1 ? (long long)D.sy : D.sz);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nf; idx += (long long)gridDim.x * blockDim.x) {
        int x[3];
        face_coords(F, a, idx, x);
        const int f = x[a];
        T v;
        if (f > 0 && f < na) {
            const long long R = cell_of(D, x), L = R - st;
            const bool cut = D.flags && ((D.flags[L] >> (2 * a + 1)) & 1u);
            v = cut ? (T)cut_face_velocity(D, L, R, a) : (T)0.5 * (us[a * D.N + L] + us[a * D.N + R]);
        } else {
            const int s = f == 0 ? -1 : 1;
            const int bc = D.bc[2 * a + (s > 0)];
            int xi[3] = {x[0], x[1], x[2]};
            if (bc == IBM_BC_PERIODIC) {
                xi[a] = na - 1;
                const long long L = cell_of(D, xi);
                xi[a] = 0;
                const long long R = cell_of(D, xi);
                v = (T)0.5 * (us[a * D.N + L] + us[a * D.N + R]);
            } else if (bc == IBM_BC_INFLOW) {
                v = (T)D.u_in[a];
            } else if (bc == IBM_BC_OUTFLOW) {
                xi[a] = f == 0 ? 0 : na - 1;
                v = us[a * D.N + cell_of(D, xi)];
            } else {
                v = (T)0;
            }
        }
        Us[F.off[a] + idx] = v;
    }
}

// Net boundary flux: fscal[3] = outward flux of inflow faces, fscal[4] = of outflow faces,
// fscal[5] = number of outflow faces.
template <class T>
__global__ void k_boundary_flux(Dom D, FaceLayout F, const T* __restrict__ Us, double* partials, unsigned* counter,
                                double* fscal) {
    const int n[3] = {D.nx, D.ny, D.nz};
    long long plane[6], tot = 0;
    for (int p = 0; p < 6; ++p) {
        const int a = p >> 1;
        plane[p] = (long long)n[(a + 1) % 3] * n[(a + 2) % 3];
        tot += plane[p];
    }
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < tot; g += (long long)gridDim.x * blockDim.x) {
        int p = 0;
        long long r = g;
        while (r >= plane[p]) r -= plane[p++];
        const int bc = D.bc[p];
        if (bc != IBM_BC_INFLOW && bc != IBM_BC_OUTFLOW) continue;
        const int a = p >> 1, s = (p & 1) ? 1 : -1;
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        int x[3];
        x[b] = (int)(r % n[b]);
        x[c] = (int)(r / n[b]);
        x[a] = s < 0 ? 0 : n[a];
        const double v = (double)Us[F.index(a, x[0], x[1], x[2])];
        if (bc == IBM_BC_INFLOW) acc[0] += s * v;
        else { acc[1] += s * v; acc[2] += 1.0; }
    }
    grid_reduce<3>(acc, partials, counter, [&](double* t) {
        fscal[3] = t[0];
        fscal[4] = t[1];
        fscal[5] = t[2];
    });
}

template <class T>
__global__ void k_outflow_shift(Dom D, FaceLayout F, T* __restrict__ Us, const double* __restrict__ fscal) {
    const double nout = fscal[5];
    if (nout == 0.0) return;
    const double shift = (-fscal[3] - fscal[4]) / nout;
    const int n[3] = {D.nx, D.ny, D.nz};
    for (int p = 0; p < 6; ++p) {
        if (D.bc[p] != IBM_BC_OUTFLOW) continue;
        const int a = p >> 1, s = (p & 1) ? 1 : -1;
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const long long np = (long long)n[b] * n[c];
        for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < np; r += (long long)gridDim.x * blockDim.x) {
            int x[3];
            x[b] = (int)(r % n[b]);
            x[c] = (int)(r / n[b]);
            x[a] = s < 0 ? 0 : n[a];
            const long long fi = F.index(a, x[0], x[1], x[2]);
            Us[fi] = (T)((double)Us[fi] + s * shift);
        }
    }
}

// Eq. poisson right-hand side: b = div(U*) / dt, evaluated in the working precision and stored in
// FP64 (the pressure solve's FP64 residual b - A p starts from it).
template <class T>
__global__ void __launch_bounds__(256) k_rhs(Dom D, FaceLayout F, const T* __restrict__ Us, double* __restrict__ b,
                                             double inv_dxdt) {
    const int i = blockIdx.x * IBM_TX + threadIdx.x, j = blockIdx.y * IBM_TY + threadIdx.y, k = blockIdx.z;
    if (i >= D.nx || j >= D.ny) return;
    const T inv = (T)inv_dxdt;
    {
        const long long P = i + (long long)D.sy * j + D.sz * k;
        T div = 0;
        div += Us[F.index(0, i + 1, j, k)] - Us[F.index(0, i, j, k)];
        div += Us[F.index(1, i, j + 1, k)] - Us[F.index(1, i, j, k)];
        div += Us[F.index(2, i, j, k + 1)] - Us[F.index(2, i, j, k)];
        b[P] = (double)(div * inv);
    }
}

// Eq. correction on the cells: central pressure gradient through the link values.
template <class T>
__global__ void __launch_bounds__(256) k_correct_cells(Dom D, const T* __restrict__ us, const double* __restrict__ p,
                                                       T* __restrict__ u, T c) {
    // c = dt / (2 dx); the FP64 pressure difference is rounded once, then scaled
    const int i = blockIdx.x * IBM_TX + threadIdx.x, j = blockIdx.y * IBM_TY + threadIdx.y, k = blockIdx.z;
    if (i >= D.nx || j >= D.ny) return;
    {
        const long long P = i + (long long)D.sy * j + D.sz * k;
        const unsigned fl = flags_at(D, P);
        const int x[3] = {i, j, k};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double pp = p_across(D, p, P, x[a], fl, a, +1);
            const double pm = p_across(D, p, P, x[a], fl, a, -1);
            u[a * D.N + P] = us[a * D.N + P] - c * (T)(pp - pm);
        }
    }
}

// Eq. correction on the faces of axis a: compact pressure difference across the face.
template <class T>
__global__ void k_correct_faces(Dom D, FaceLayout F, int a, const T* __restrict__ Us, const double* __restrict__ p,
                                T* __restrict__ U, T dtdx) {
    const long long nf = (long long)F.dim[a][0] * F.dim[a][1] * F.dim[a][2];
    const int na = a == 0 ? D.nx : (a == 1 ? D.ny : D.nz);
    const long long st = a == 0 ? 1 : (a == 1 ? (long long)D.sy : D.sz);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nf; idx += (long long)gridDim.x * blockDim.x) {
        int x[3];
        face_coords(F, a, idx, x);
        const int f = x[a];
        const long long fi = F.off[a] + idx;
        double pl, pr;
        if (f > 0 && f < na) {
            const long long R = cell_of(D, x), L = R - st;
            if (D.flags && ((D.flags[L] >> (2 * a + 1)) & 1u)) { U[fi] = Us[fi]; continue; }
            pl = p[L];
            pr = p[R];
        } else {
            const int s = f == 0 ? -1 : 1;
            const int bc = D.bc[2 * a + (s > 0)];
            int xi[3] = {x[0], x[1], x[2]};
            if (bc == IBM_BC_PERIODIC) {
                xi[a] = na - 1;
                pl = p[cell_of(D, xi)];
                xi[a] = 0;
                pr = p[cell_of(D, xi)];
            } else if (bc == IBM_BC_OUTFLOW) {
                xi[a] = f == 0 ? 0 : na - 1;
                const double pin = p[cell_of(D, xi)];
                if (s < 0) { pl = -pin; pr = pin; } else { pl = pin; pr = -pin; }
            } else {
                U[fi] = Us[fi];
                continue;
            }
        }
        U[fi] = Us[fi] - dtdx * (T)(pr - pl);
    }
}

// Eq. force: Shepard average of p on each side of every triangle over the 2x2x2 block of cell
// centres around its centroid.
__global__ void k_forces(Dom D, const float* __restrict__ tri, long long ntri, const double* __restrict__ p,
                         double* partials, unsigned* counter, double* out) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntri; t += (long long)gridDim.x * blockDim.x) {
        double V[3][3];
        bool ok = true;
        for (int q = 0; q < 9; ++q) {
            V[q / 3][q % 3] = (double)tri[9 * t + q];
            ok = ok && isfinite(V[q / 3][q % 3]);
        }
        if (!ok) continue;
        double e1[3], e2[3], nrm[3], X[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = V[1][d] - V[0][d];
            e2[d] = V[2][d] - V[0][d];
            X[d] = (V[0][d] + V[1][d] + V[2][d]) / 3.0;
        }
        nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double len = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        if (!(len > 0.0)) continue;
        const double area = 0.5 * len * D.dx * D.dx;
        for (int d = 0; d < 3; ++d) nrm[d] /= len;
        long long base[3];
        for (int d = 0; d < 3; ++d) base[d] = (long long)floor(X[d] - 0.5);
        double sw[2] = {0.0, 0.0}, sp[2] = {0.0, 0.0};
        const long long n[3] = {D.nx, D.ny, D.nz};
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    const long long x[3] = {base[0] + di, base[1] + dj, base[2] + dk};
                    if (x[0] < 0 || x[1] < 0 || x[2] < 0 || x[0] >= n[0] || x[1] >= n[1] || x[2] >= n[2]) continue;
                    double r2 = 0.0, sd = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        const double r = ((double)x[d] + 0.5) - X[d];
                        r2 += r * r;
                        sd += nrm[d] * r;
                    }
                    if (sd == 0.0) continue;
                    if (r2 < 1e-24) r2 = 1e-24;
                    const double w = 1.0 / r2;
                    const int side = sd > 0.0 ? 0 : 1;
                    sw[side] += w;
                    sp[side] += w * p[x[0] + (long long)D.sy * x[1] + D.sz * x[2]];
                }
        if (sw[0] == 0.0 || sw[1] == 0.0) continue;
        const double pf = sp[0] / sw[0], pb = sp[1] / sw[1];
        for (int d = 0; d < 3; ++d) acc[d] += area * (pb - pf) * nrm[d];
        acc[3] += 1.0;
    }
    grid_reduce<4>(acc, partials, counter, [&](double* t) {
        for (int q = 0; q < 4; ++q) out[q] = t[q];
    });
}

// Viscous force on the body: the molecular diffusive flux nu (u_P - u_G) dx through every cut link,
// u_G the Eq. q_axis ghost value the momentum equation uses there.  One thread per link record.
template <class T>
__global__ void k_viscous_force(Dom D, const T* __restrict__ u, double nu, double* partials, unsigned* counter,
                                double* out) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long nrec = D.flags ? (long long)D.nrec : 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nrec; q += (long long)gridDim.x * blockDim.x) {
        const LinkRec& R = D.rec[q];
        const long long P = R.cell;
        const int a = R.axis, sd = R.side;
        const int xa = a == 0 ? (int)(P % D.nx) : (a == 1 ? (int)((P / D.nx) % D.ny) : (int)(P / D.sz));
        const unsigned fl = D.flags[P];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double uG = (double)vel_across(D, u, c, P, xa, fl, a, sd);
            acc[c] += nu * ((double)u[c * D.N + P] - uG) * D.dx;
        }
        acc[3] += 1.0;
    }
    grid_reduce<4>(acc, partials, counter, [&](double* t) {
        for (int q = 0; q < 4; ++q) out[q] = t[q];
    });
}

unsigned lin_blocks(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    long long cap = 16LL * IBM_NSM;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}


// ---- Crank-Nicolson predictor (Eq. crank-nicolson) -----------------------------------------------
// delta = u* - u^n solves M delta = delta - (dt/2) L_0(delta) = dt L(u^n) over the stacked three
// components; BiCGStab from delta = 0, scalars on the device (the same recurrences as the pressure
// BiCGStab).  Cell kernels loop over a capped grid; per-thread sums run in the working precision and
// the block and grid sums in FP64.

// The fast kernel of a pair leaves its sums in sc->part; the general kernel, launched after it, adds
// its own and finishes (so the totals are formed in a fixed order).
template <class T, bool GENERAL>
__global__ void __launch_bounds__(256, (FluxOcc<T, GENERAL>::value)) k_cn_begin(Dom D, FaceLayout F, const T* __restrict__ u, const T* __restrict__ U,
                                                  const T* __restrict__ nut, T* __restrict__ H, T* __restrict__ r,
                                                  T* __restrict__ rh, T* __restrict__ x, T nu, T gam, T dt, double tol2,
                                                  int maxit, int keepx, SolveScal* sc, double* partials, unsigned* counter,
                                                  const int32_t* __restrict__ list, long long nlist) {
    T a0 = 0;
    flux_cells<GENERAL, T>(D, F, u, U, nut, nu, gam, list, nlist, [&](long long P, const T (&h)[3], const T (&uc)[3]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long q = c * D.N + P;
            const T b = dt * h[c];
            H[q] = h[c];
            r[q] = b;
            rh[q] = b;
            if (!keepx) x[q] = (T)0;
            a0 += b * b;
        }
    });
    T acc[1] = {a0};
    grid_reduce<1>(acc, partials, counter, [&](double* t) {
        if (!GENERAL) {
            sc->part[0] = t[0];
            return;
        }
        const double bb = t[0] + sc->part[0];
        sc->bb = bb;
        sc->rr = bb;
        sc->rho = bb;
        sc->rho_old = 1.0;
        sc->alpha = 1.0;
        sc->omega = 1.0;
        sc->target2 = tol2 * bb;
        sc->iters = 0;
        sc->maxit = maxit;
        sc->restart = 1;
        sc->nonfinite = isfinite(bb) ? 0 : 1;
        sc->done = (bb == 0.0 || !isfinite(bb)) ? 1 : 0;
    });
}

// p = r (first iteration) or r + beta (p - omega v)
template <class T>
__global__ void k_cn_p(long long n, const T* __restrict__ r, T* __restrict__ p, const T* __restrict__ v,
                       const SolveScal* sc) {
    if (sc->done) return;
    const bool rs = sc->restart != 0;
    const T beta = rs ? (T)0 : (T)((sc->rho / sc->rho_old) * (sc->alpha / sc->omega));
    const T om = rs ? (T)0 : (T)sc->omega;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        p[q] = rs ? r[q] : r[q] + beta * (p[q] - om * v[q]);
}

// y = M xin = xin - (dt/2) L_0(xin).  mode 0: (w, y) -> alpha = rho / (r_hat, v).  mode 1 (xin = s):
// (y, s), (y, y) -> omega.  mode 2 (warm start, xin = the previous increment): r = b - M xin with b
// read from and r written to r2, r_hat = r in y, (r, r) -> rr = rho.
template <class T, bool GENERAL>
__global__ void __launch_bounds__(256, (FluxOcc<T, GENERAL>::value)) k_cn_apply(Dom D, FaceLayout F, const T* __restrict__ xin,
                                                  const T* __restrict__ U, const T* __restrict__ nut,
                                                  T* __restrict__ y, const T* __restrict__ w, T* r2, T nu, T gam,
                                                  T hdt, int mode, SolveScal* sc, double* partials,
                                                  unsigned* counter, const int32_t* __restrict__ list, long long nlist) {
    if (sc->done) return;
    T a0 = 0, a1 = 0;
    flux_cells<GENERAL, T>(D, F, xin, U, nut, nu, gam, list, nlist, [&](long long P, const T (&h)[3], const T (&uc)[3]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long q = c * D.N + P;
            const T xv = uc[c];
            const T yv = xv - hdt * h[c];
            if (mode == 2) {
                const T rn = r2[q] - yv;
                r2[q] = rn;
                y[q] = rn;
                a0 += rn * rn;
                continue;
            }
            y[q] = yv;
            if (mode == 0) {
                a0 += w[q] * yv;
            } else {
                a0 += yv * xv;
                a1 += yv * yv;
            }
        }
    });
    T acc[2] = {a0, a1};
    grid_reduce<2>(acc, partials, counter, [&](double* t) {
        if (!GENERAL) {
            sc->part[0] = t[0];
            sc->part[1] = t[1];
            return;
        }
        const double t0 = t[0] + sc->part[0], t1 = t[1] + sc->part[1];
        if (mode == 2) {
            sc->rr = t0;
            sc->rho = t0;
            if (!isfinite(t0)) sc->nonfinite = 1;
            if (!isfinite(t0) || t0 <= sc->target2) sc->done = 1;
            return;
        }
        if (mode == 0) {
            sc->rv = t0;
            sc->alpha = t0 != 0.0 ? sc->rho / t0 : 0.0;
            if (t0 == 0.0 || !isfinite(t0)) {
                if (!isfinite(t0)) sc->nonfinite = 1;
                sc->done = 1;                                        // breakdown
            }
        } else {
            sc->ts = t0;
            sc->tt = t1;
            sc->omega = t1 > 0.0 ? t0 / t1 : 0.0;
        }
    });
}

// s = r - alpha v
template <class T>
__global__ void k_cn_s(long long n, const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ sv,
                       const SolveScal* sc) {
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        sv[q] = r[q] - alpha * v[q];
}

// x += alpha p + omega s, r = s - omega t; (r_hat, r), (r, r); convergence test.
template <class T>
__global__ void __launch_bounds__(256) k_cn_xr(long long n, const T* __restrict__ p, const T* __restrict__ sv,
                                               const T* __restrict__ tv, const T* __restrict__ rh, T* __restrict__ x,
                                               T* __restrict__ r, SolveScal* sc, double* partials, unsigned* counter) {
    if (sc->done) return;
    const T alpha = (T)sc->alpha, om = (T)sc->omega;
    T a0 = 0, a1 = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        x[q] = x[q] + alpha * p[q] + om * sv[q];
        const T rv = sv[q] - om * tv[q];
        r[q] = rv;
        a0 += rh[q] * rv;
        a1 += rv * rv;
    }
    T acc[2] = {a0, a1};
    grid_reduce<2>(acc, partials, counter, [&](double* t) {
        sc->rho_old = sc->rho;
        sc->rho = t[0];
        sc->rr_old = sc->rr;
        sc->rr = t[1];
        sc->restart = 0;
        sc->iters += 1;
        if (!isfinite(t[1])) {
            sc->nonfinite = 1;
            sc->done = 1;
        } else if (t[1] <= sc->target2 || sc->iters >= sc->maxit || sc->omega == 0.0 || t[0] == 0.0) {
            sc->done = 1;
        }
    });
}

template <class T>
__global__ void k_cn_finish(long long n, const T* __restrict__ u, const T* __restrict__ x, T* __restrict__ ustar) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        ustar[q] = u[q] + x[q];
}

// Persistent launch of the tiled flux kernels: as many blocks as fit on the GPU at once (measured
// for the heaviest of them at set-up), each walking tiles until none is left.
int g_tile_blocks[2] = {2 * IBM_NSM, 2 * IBM_NSM};   // FP32, FP64

template <class T>
dim3 tile_grid(const LesCtx& c) {
    const long long items = (long long)((c.D.nx + FT_X - 1) / FT_X) * ((c.D.ny + FT_Y - 1) / FT_Y) *
                            ((c.D.nz + FT_KZ - 1) / FT_KZ);
    const long long cap = g_tile_blocks[sizeof(T) == 8];
    return dim3((unsigned)(items < cap ? items : cap));
}

template <class T>
int predict_cn_t(const LesCtx& c, const T* u, const T* U, const T* nut, T* H, T* ustar, int* iters, cudaStream_t s) {
    CNWork& w = *c.cn;
    Dom Dh = c.D;
    Dh.hom = 1;
    const long long n3 = 3 * c.D.N;
    const unsigned nbv = lin_blocks(n3, 256);
    T *r = (T*)w.r, *rh = (T*)w.rh, *p = (T*)w.p, *v = (T*)w.v, *sv = (T*)w.sv, *tv = (T*)w.tv, *x = (T*)w.x;
    const T nu = (T)c.nu, gam = (T)c.quick, dt = (T)c.dt, hdt = (T)(0.5 * c.dt);
    const unsigned ngen = lin_blocks(c.n_general > 0 ? c.n_general : 1, 256);
    prof_begin(c.prof, PS_PREDICT, s);
    // warm start from the previous step's increment (the increment changes slowly from step to step)
    const int keepx = w.have_x;
    k_cn_begin<T, false><<<tile_grid<T>(c), dim3(FT_X, FT_Y), fast_tile_smem<T>(), s>>>(c.D, c.F, u, U, nut, H, r, rh, x, nu, gam, dt, w.tol * w.tol,
                                                        w.maxit, keepx, w.sc, c.partials, c.counter, nullptr, 0);
    k_cn_begin<T, true><<<ngen, 256, 0, s>>>(c.D, c.F, u, U, nut, H, r, rh, x, nu, gam, dt, w.tol * w.tol, w.maxit,
                                             keepx, w.sc, c.partials, c.counter, c.general, c.n_general);
    prof_end(c.prof, PS_PREDICT, s);
    IBM_LAUNCHED("k_cn_begin");
    IBM_COUNT(c, 2);
    auto apply = [&](const T* in, T* out, int mode) {
        const T* wv = mode == 2 ? nullptr : rh;
        T* r2 = mode == 2 ? r : nullptr;
        k_cn_apply<T, false><<<tile_grid<T>(c), dim3(FT_X, FT_Y), fast_tile_smem<T>(), s>>>(Dh, c.F, in, U, nut, out, wv, r2, nu, gam, hdt, mode, w.sc,
                                                            c.partials, c.counter, nullptr, 0);
        k_cn_apply<T, true><<<ngen, 256, 0, s>>>(Dh, c.F, in, U, nut, out, wv, r2, nu, gam, hdt, mode, w.sc, c.partials,
                                                 c.counter, c.general, c.n_general);
    };
    if (keepx) {
        apply(x, rh, 2);
        IBM_COUNT(c, 2);
    }
    for (;;) {
        prof_begin(c.prof, PS_MOMENTUM, s);
        for (int it = 0; it < 4; ++it) {
            k_cn_p<T><<<nbv, 256, 0, s>>>(n3, r, p, v, w.sc);
            apply(p, v, 0);
            k_cn_s<T><<<nbv, 256, 0, s>>>(n3, r, v, sv, w.sc);
            apply(sv, tv, 1);
            k_cn_xr<T><<<nbv, 256, 0, s>>>(n3, p, sv, tv, rh, x, r, w.sc, c.partials, c.counter);
        }
        prof_end(c.prof, PS_MOMENTUM, s);
        IBM_LAUNCHED("crank-nicolson bicgstab");
        IBM_COUNT(c, 28);
        IBM_CUDA(cudaMemcpyAsync(w.hsc, w.sc, sizeof(SolveScal), cudaMemcpyDeviceToHost, s));
        IBM_CUDA(cudaStreamSynchronize(s));
        if (w.hsc->done) break;
    }
    k_cn_finish<T><<<nbv, 256, 0, s>>>(n3, u, x, ustar);
    IBM_LAUNCHED("k_cn_finish");
    IBM_COUNT(c, 1);
    if (iters) *iters = w.hsc->iters;
    w.have_x = !w.hsc->nonfinite && w.hsc->rr <= w.hsc->target2;
    if (w.hsc->nonfinite) return ibm_fail(IBM_E_NONFINITE, "crank-nicolson momentum solve: non-finite residual");
    if (!(w.hsc->rr <= w.hsc->target2))
        return ibm_fail(IBM_E_NOCONV, "crank-nicolson momentum solve: relative residual %.3e after %d iterations",
                        sqrt(w.hsc->rr / (w.hsc->bb > 0 ? w.hsc->bb : 1.0)), w.hsc->iters);
    return IBM_OK;
}

}  // namespace

namespace {
// Order-preserving compaction of the general cells: one block per (y, z) row, ballots over x.
__global__ void k_list_general(Dom D, const unsigned long long* __restrict__ row_off,
                               int32_t* __restrict__ list) {
    const int j = blockIdx.x, k = blockIdx.y;
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const long long row = j + (long long)D.ny * k;
    for (int i0 = 0; i0 < D.nx; i0 += 32) {
        const int i = i0 + threadIdx.x;
        const long long P = i + (long long)D.sy * j + D.sz * k;
        const bool g = i < D.nx && !fast_cell(D, P, i, j, k);
        const unsigned m = __ballot_sync(0xffffffffu, g);
        if (g) list[row_off[row] + base + __popc(m & ((1u << threadIdx.x) - 1u))] = (int32_t)P;
        __syncwarp();
        if (threadIdx.x == 0) base += __popc(m);
        __syncwarp();
    }
}

__global__ void k_row_counts(Dom D, unsigned long long* __restrict__ rc, uint8_t* __restrict__ fast) {
    const int j = blockIdx.x, k = blockIdx.y;
    unsigned n = 0;
    for (int i = threadIdx.x; i < D.nx; i += 32) {
        const long long P = i + (long long)D.sy * j + D.sz * k;
        const bool f = fast_cell(D, P, i, j, k);
        fast[P] = f ? 1 : 0;
        n += !f;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if (threadIdx.x == 0) rc[j + (long long)D.ny * k] = n;
}

__global__ void k_row_scan(long long nrows, unsigned long long* __restrict__ rc, unsigned long long* total) {
    // one thread: rows are few (ny * nz) and this runs once per solver state
    unsigned long long acc = 0;
    for (long long r = 0; r < nrows; ++r) {
        const unsigned long long v = rc[r];
        rc[r] = acc;
        acc += v;
    }
    *total = acc;
}
}  // namespace

int flux_kernels_setup() {
    // the tiles need more than the default 48 KB of dynamic shared memory
    const int bytes = (int)fast_tile_smem<double>(), bytesf = (int)fast_tile_smem<float>();
    IBM_CUDA(cudaFuncSetAttribute(k_predict<false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    IBM_CUDA(cudaFuncSetAttribute(k_cn_begin<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    IBM_CUDA(cudaFuncSetAttribute(k_cn_apply<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    IBM_CUDA(cudaFuncSetAttribute(k_predict<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytesf));
    IBM_CUDA(cudaFuncSetAttribute(k_cn_begin<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytesf));
    IBM_CUDA(cudaFuncSetAttribute(k_cn_apply<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytesf));
    int dev = 0, nsm = IBM_NSM, bf = 0, bd = 0;
    IBM_CUDA(cudaGetDevice(&dev));
    IBM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    IBM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_cn_apply<float, false>, FT_X * FT_Y,
                                                           fast_tile_smem<float>()));
    IBM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, k_cn_apply<double, false>, FT_X * FT_Y,
                                                           fast_tile_smem<double>()));
    g_tile_blocks[0] = (bf > 0 ? bf : 1) * nsm;
    g_tile_blocks[1] = (bd > 0 ? bd : 1) * nsm;
    return IBM_OK;
}

int build_general_list(LesCtx& c, cudaStream_t s) {
    const long long nrows = (long long)c.D.ny * c.D.nz;
    unsigned long long* rc = nullptr;
    IBM_CUDA(cudaMalloc((void**)&rc, (size_t)(nrows + 1) * sizeof(unsigned long long)));
    dim3 rows((unsigned)c.D.ny, (unsigned)c.D.nz);
    cudaError_t e0 = cudaMalloc((void**)&c.fastmask, (size_t)c.D.N);
    if (e0 != cudaSuccess) {
        cudaFree(rc);
        return ibm_fail(IBM_E_NOMEM, "momentum flux: fast-cell mask (%lld bytes)", (long long)c.D.N);
    }
    k_row_counts<<<rows, 32, 0, s>>>(c.D, rc, c.fastmask);
    k_row_scan<<<1, 1, 0, s>>>(nrows, rc, rc + nrows);
    unsigned long long total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, rc + nrows, sizeof(total), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.general, (size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    if (e == cudaSuccess && total > 0) {
        k_list_general<<<rows, 32, 0, s>>>(c.D, rc, c.general);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(rc);
    if (e != cudaSuccess) return ibm_cuda_check(e, "momentum flux: general-cell list");
    c.n_general = (long long)total;
    c.D.fast = c.fastmask;
    return IBM_OK;
}

int launch_csm(const LesCtx& c, const void* u, void* nut, cudaStream_t s) {
    if (c.prec == IBM_FP64)
        k_csm<double><<<c.pgrid, c.cg.block, 0, s>>>(c.D, (const double*)u, (double*)nut);
    else
        k_csm<float><<<c.pgrid, c.cg.block, 0, s>>>(c.D, (const float*)u, (float*)nut);
    IBM_LAUNCHED("k_csm");
    IBM_COUNT(c, 1);
    return IBM_OK;
}

template <class T>
static void predict_t(const LesCtx& c, const T* u, const T* U, const T* nut, const T* Hprev, T* H, T* ustar, int first,
                      cudaStream_t s) {
    k_predict<false, T><<<tile_grid<T>(c), dim3(FT_X, FT_Y), fast_tile_smem<T>(), s>>>(c.D, c.F, u, U, nut, Hprev, H, ustar, (T)c.nu, (T)c.dt, first,
                                                       (T)c.quick, nullptr, 0);
    if (c.n_general > 0)
        k_predict<true, T><<<lin_blocks(c.n_general, 256), 256, 0, s>>>(c.D, c.F, u, U, nut, Hprev, H, ustar,
                                                                         (T)c.nu, (T)c.dt, first, (T)c.quick,
                                                                         c.general, c.n_general);
}

int launch_predict(const LesCtx& c, const void* u, const void* U, const void* nut, const void* Hprev, void* H,
                   void* ustar, int first, cudaStream_t s) {
    if (c.prec == IBM_FP64)
        predict_t<double>(c, (const double*)u, (const double*)U, (const double*)nut, (const double*)Hprev, (double*)H,
                          (double*)ustar, first, s);
    else
        predict_t<float>(c, (const float*)u, (const float*)U, (const float*)nut, (const float*)Hprev, (float*)H,
                         (float*)ustar, first, s);
    IBM_LAUNCHED("k_predict");
    IBM_COUNT(c, c.n_general > 0 ? 2 : 1);
    return IBM_OK;
}

int launch_predict_cn(const LesCtx& c, const void* u, const void* U, const void* nut, void* H, void* ustar,
                      int* iters, cudaStream_t s) {
    if (!c.cn) return ibm_fail(IBM_E_INVALID, "crank-nicolson predictor: state created without integrator = 1");
    if (c.prec == IBM_FP64)
        return predict_cn_t<double>(c, (const double*)u, (const double*)U, (const double*)nut, (double*)H,
                                    (double*)ustar, iters, s);
    return predict_cn_t<float>(c, (const float*)u, (const float*)U, (const float*)nut, (float*)H, (float*)ustar,
                               iters, s);
}

int launch_forcing(const LesCtx& c, void* ustar, cudaStream_t s) {
    if (c.n_inc == 0 || !c.D.flags) {
        IBM_CUDA(cudaMemsetAsync(c.fscal, 0, 3 * sizeof(double), s));
        return IBM_OK;
    }
    const unsigned nb = lin_blocks(c.n_inc, 256);
    const double vol = c.D.dx * c.D.dx * c.D.dx;
    if (c.prec == IBM_FP64) {
        k_forcing_gather<double><<<nb, 256, 0, s>>>(c.D, c.inc, c.n_inc, (const double*)ustar, c.fdelta, c.dt,
                                                    c.deadend_on, vol, c.partials, c.counter, c.fscal);
        k_forcing_apply<double><<<nb, 256, 0, s>>>(c.D, c.inc, c.n_inc, c.fdelta, (double*)ustar);
    } else {
        k_forcing_gather<float><<<nb, 256, 0, s>>>(c.D, c.inc, c.n_inc, (const float*)ustar, c.fdelta, (float)c.dt,
                                                   c.deadend_on, vol, c.partials, c.counter, c.fscal);
        k_forcing_apply<float><<<nb, 256, 0, s>>>(c.D, c.inc, c.n_inc, c.fdelta, (float*)ustar);
    }
    IBM_LAUNCHED("k_forcing");
    IBM_COUNT(c, 2);
    return IBM_OK;
}

template <class T>
static void faces_t(const LesCtx& c, const T* us, T* Us, cudaStream_t s) {
    for (int a = 0; a < 3; ++a) {
        const long long nf = (long long)c.F.dim[a][0] * c.F.dim[a][1] * c.F.dim[a][2];
        k_faces<T><<<lin_blocks(nf, 256), 256, 0, s>>>(c.D, c.F, a, us, Us);
    }
    k_boundary_flux<T><<<64, 256, 0, s>>>(c.D, c.F, Us, c.partials, c.counter, c.fscal);
    k_outflow_shift<T><<<64, 256, 0, s>>>(c.D, c.F, Us, c.fscal);
}

int launch_faces(const LesCtx& c, const void* ustar, void* Ustar, cudaStream_t s) {
    if (c.prec == IBM_FP64) faces_t<double>(c, (const double*)ustar, (double*)Ustar, s);
    else faces_t<float>(c, (const float*)ustar, (float*)Ustar, s);
    IBM_LAUNCHED("k_faces");
    IBM_COUNT(c, 5);
    return IBM_OK;
}

int launch_rhs(const LesCtx& c, const void* Ustar, double* b, cudaStream_t s) {
    const double inv = 1.0 / (c.D.dx * c.dt);
    if (c.prec == IBM_FP64)
        k_rhs<double><<<c.pgrid, c.cg.block, 0, s>>>(c.D, c.F, (const double*)Ustar, b, inv);
    else
        k_rhs<float><<<c.pgrid, c.cg.block, 0, s>>>(c.D, c.F, (const float*)Ustar, b, inv);
    IBM_LAUNCHED("k_rhs");
    IBM_COUNT(c, 1);
    return IBM_OK;
}

template <class T>
static void correct_t(const LesCtx& c, const T* us, const T* Us, const double* p, T* u, T* U, cudaStream_t s) {
    k_correct_cells<T><<<c.pgrid, c.cg.block, 0, s>>>(c.D, us, p, u, (T)(c.dt / (2.0 * c.D.dx)));
    for (int a = 0; a < 3; ++a) {
        const long long nf = (long long)c.F.dim[a][0] * c.F.dim[a][1] * c.F.dim[a][2];
        k_correct_faces<T><<<lin_blocks(nf, 256), 256, 0, s>>>(c.D, c.F, a, Us, p, U, (T)(c.dt / c.D.dx));
    }
}

int launch_correct(const LesCtx& c, const void* ustar, const void* Ustar, const double* p, void* u, void* U,
                   cudaStream_t s) {
    if (c.prec == IBM_FP64)
        correct_t<double>(c, (const double*)ustar, (const double*)Ustar, p, (double*)u, (double*)U, s);
    else
        correct_t<float>(c, (const float*)ustar, (const float*)Ustar, p, (float*)u, (float*)U, s);
    IBM_LAUNCHED("k_correct");
    IBM_COUNT(c, 4);
    return IBM_OK;
}

int launch_forces(const LesCtx& c, const float* tri, long long ntri, const double* p, double* d_out4, cudaStream_t s) {
    k_forces<<<lin_blocks(ntri, 128), 128, 0, s>>>(c.D, tri, ntri, p, c.partials, c.counter, d_out4);
    IBM_LAUNCHED("k_forces");
    IBM_COUNT(c, 1);
    return IBM_OK;
}

int launch_viscous_force(const LesCtx& c, const void* u, double* d_out4, cudaStream_t s) {
    const unsigned nb = lin_blocks(c.n_rec > 0 ? c.n_rec : 1, 256);
    if (c.prec == IBM_FP64)
        k_viscous_force<double><<<nb, 256, 0, s>>>(c.D, (const double*)u, c.nu, c.partials, c.counter, d_out4);
    else
        k_viscous_force<float><<<nb, 256, 0, s>>>(c.D, (const float*)u, c.nu, c.partials, c.counter, d_out4);
    IBM_LAUNCHED("k_viscous_force");
    IBM_COUNT(c, 1);
    return IBM_OK;
}

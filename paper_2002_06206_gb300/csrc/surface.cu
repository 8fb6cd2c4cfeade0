// surface.cu -- surface pressure per triangle side (Eq. force) with the thin-plate filter of
// Eq. force_filter, read as: a cell centre takes part in the Shepard average of a surface node X only
// if the open segment from X to it crosses no other triangle of the soup.
//
// The triangles are binned once per soup (ibm_surface_create) into 2x2x2-cell bins by their bounding
// boxes; a segment from a centroid to a cell of its 2x2x2 block stays inside one 1x1x1 box, so only
// the <= 8 bins over that box are searched.  This unit is compiled without FMA contraction: the
// orientation tests and the Shepard sums round every product and sum separately, in the same order
// as the plain definition, so the visibility decisions and the per-side averages are reproducible.
#include <math_constants.h>

#include "scan.cuh"

namespace {

constexpr int BIN = 2;          // bin edge in cells
constexpr int BIN_ORIGIN = -2;  // bins cover [-2, n + 2) along each axis

struct Bins {
    int nb[3];
    long long nbins;
};

__device__ __forceinline__ bool load_tri(const float* __restrict__ t, double V[3][3]) {
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        V[q / 3][q % 3] = (double)t[q];
        ok = ok && isfinite(V[q / 3][q % 3]);
    }
    return ok;
}

// Bin range [lo, hi] along axis a covered by [mn, mx]; false if outside the binned region.
__device__ __forceinline__ bool bin_range(const Bins& B, int a, double mn, double mx, int& lo, int& hi) {
    const double o = (double)BIN_ORIGIN;
    double l = floor((mn - o) / BIN), h = floor((mx - o) / BIN);
    if (h < 0.0 || l >= (double)B.nb[a]) return false;
    lo = l < 0.0 ? 0 : (int)l;
    hi = h >= (double)B.nb[a] ? B.nb[a] - 1 : (int)h;
    return true;
}

__device__ __forceinline__ bool tri_bins(const Bins& B, const double V[3][3], int lo[3], int hi[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double mn = fmin(fmin(V[0][a], V[1][a]), V[2][a]);
        const double mx = fmax(fmax(V[0][a], V[1][a]), V[2][a]);
        if (!bin_range(B, a, mn, mx, lo[a], hi[a])) return false;
    }
    return true;
}

__global__ void k_bin_count(const float* __restrict__ tri, long long ntri, Bins B, unsigned* __restrict__ cnt) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntri; t += (long long)gridDim.x * blockDim.x) {
        double V[3][3];
        int lo[3], hi[3];
        if (!load_tri(tri + 9 * t, V) || !tri_bins(B, V, lo, hi)) continue;
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i)
                    atomicAdd(&cnt[i + (long long)B.nb[0] * (j + (long long)B.nb[1] * k)], 1u);
    }
}

struct BinCount {
    const unsigned* c;
    __device__ long long operator()(long long i) const { return (long long)c[i]; }
};
struct BinOffset {
    long long* off;
    __device__ void operator()(long long i, long long o, long long) const { off[i] = o; }
};

__global__ void k_bin_fill(const float* __restrict__ tri, long long ntri, Bins B, const long long* __restrict__ off,
                           unsigned* __restrict__ cursor, int32_t* __restrict__ ent) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntri; t += (long long)gridDim.x * blockDim.x) {
        double V[3][3];
        int lo[3], hi[3];
        if (!load_tri(tri + 9 * t, V) || !tri_bins(B, V, lo, hi)) continue;
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    const long long b = i + (long long)B.nb[0] * (j + (long long)B.nb[1] * k);
                    ent[off[b] + atomicAdd(&cursor[b], 1u)] = (int32_t)t;
                }
    }
}

// orient3d(a, b, c, d) = det[b - a; c - a; d - a], each operation rounded once, in this order.
__device__ __forceinline__ double orient3(const double* a, const double* b, const double* c, const double* d) {
    const double u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
    const double v0 = c[0] - a[0], v1 = c[1] - a[1], v2 = c[2] - a[2];
    const double w0 = d[0] - a[0], w1 = d[1] - a[1], w2 = d[2] - a[2];
    const double m0 = v1 * w2 - v2 * w1;
    const double m1 = v0 * w2 - v2 * w0;
    const double m2 = v0 * w1 - v1 * w0;
    return (u0 * m0 - u1 * m1) + u2 * m2;
}

// The open segment X-Y crosses triangle V: X and Y strictly on opposite sides of its plane, the line
// through them inside the triangle or on its edges.
__device__ __forceinline__ bool crosses(const double* X, const double* Y, const double V[3][3]) {
    const double o1 = orient3(V[0], V[1], V[2], X), o2 = orient3(V[0], V[1], V[2], Y);
    if (!((o1 > 0.0 && o2 < 0.0) || (o1 < 0.0 && o2 > 0.0))) return false;
    const double e0 = orient3(X, Y, V[0], V[1]), e1 = orient3(X, Y, V[1], V[2]), e2 = orient3(X, Y, V[2], V[0]);
    return (e0 >= 0.0 && e1 >= 0.0 && e2 >= 0.0) || (e0 <= 0.0 && e1 <= 0.0 && e2 <= 0.0);
}

__device__ bool hidden(const float* __restrict__ tri, long long self, const double* X, const double* Y, const Bins& B,
                       const long long* __restrict__ off, const int32_t* __restrict__ ent) {
    double mn[3], mx[3];
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        mn[a] = fmin(X[a], Y[a]);
        mx[a] = fmax(X[a], Y[a]);
        if (!bin_range(B, a, mn[a], mx[a], lo[a], hi[a])) return false;
    }
    for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                const long long b = i + (long long)B.nb[0] * (j + (long long)B.nb[1] * k);
                for (long long e = off[b]; e < off[b + 1]; ++e) {
                    const long long o = ent[e];
                    if (o == self) continue;
                    double V[3][3];
                    if (!load_tri(tri + 9 * o, V)) continue;
                    bool apart = false;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const double tmn = fmin(fmin(V[0][a], V[1][a]), V[2][a]);
                        const double tmx = fmax(fmax(V[0][a], V[1][a]), V[2][a]);
                        apart = apart || tmx < mn[a] || tmn > mx[a];
                    }
                    if (!apart && crosses(X, Y, V)) return true;
                }
            }
    return false;
}

// One thread per triangle: Shepard averages over the 2x2x2 block of cell centres around the centroid,
// split by the side of the triangle's plane, each side on its own.
__global__ void __launch_bounds__(128) k_surface_pressure(const float* __restrict__ tri, long long ntri, int nx, int ny,
                                                          int nz, double dx, const double* __restrict__ p, int zfilter,
                                                          Bins B, const long long* __restrict__ off,
                                                          const int32_t* __restrict__ ent, double* __restrict__ pside,
                                                          double* partials, unsigned* counter, double* out) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntri; t += (long long)gridDim.x * blockDim.x) {
        pside[2 * t] = CUDART_NAN;
        pside[2 * t + 1] = CUDART_NAN;
        double V[3][3];
        if (!load_tri(tri + 9 * t, V)) continue;
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
        const double area = 0.5 * len * dx * dx;
        for (int d = 0; d < 3; ++d) nrm[d] /= len;
        long long base[3];
        for (int d = 0; d < 3; ++d) base[d] = (long long)floor(X[d] - 0.5);
        double sw[2] = {0.0, 0.0}, sp[2] = {0.0, 0.0};
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    const long long x[3] = {base[0] + di, base[1] + dj, base[2] + dk};
                    if (x[0] < 0 || x[1] < 0 || x[2] < 0 || x[0] >= nx || x[1] >= ny || x[2] >= nz) continue;
                    double Y[3], r2 = 0.0, sd = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        Y[d] = (double)x[d] + 0.5;
                        const double r = Y[d] - X[d];
                        r2 += r * r;
                        sd += nrm[d] * r;
                    }
                    if (sd == 0.0) continue;
                    if (zfilter && hidden(tri, t, X, Y, B, off, ent)) continue;
                    if (r2 < 1e-24) r2 = 1e-24;
                    const double w = 1.0 / r2;
                    const int side = sd > 0.0 ? 0 : 1;
                    sw[side] += w;
                    sp[side] += w * p[x[0] + (long long)nx * (x[1] + (long long)ny * x[2])];
                }
        for (int s = 0; s < 2; ++s) {
            if (sw[s] == 0.0) continue;
            const double ps = sp[s] / sw[s];
            pside[2 * t + s] = ps;
            for (int d = 0; d < 3; ++d) acc[d] += (s == 0 ? -1.0 : 1.0) * area * ps * nrm[d];
            acc[3] += 1.0;
        }
    }
    grid_reduce<4>(acc, partials, counter, [&](double* tot) {
        for (int q = 0; q < 4; ++q) out[q] = tot[q];
    });
}

unsigned nblocks(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 8LL * IBM_NSM;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

struct ibm_surface {
    ibm_grid grid;
    const float* tri;
    long long ntri;
    Bins B;
    long long* off;        // nbins + 1
    int32_t* ent;
    long long nent;
    double* partials;
    unsigned* counter;
    double* out4;
    double* hout;          // pinned
};

extern "C" void ibm_surface_destroy(ibm_surface* S) {
    if (!S) return;
    cudaFree(S->off);
    cudaFree(S->ent);
    cudaFree(S->partials);
    cudaFree(S->counter);
    cudaFree(S->out4);
    cudaFreeHost(S->hout);
    free(S);
}

extern "C" int ibm_surface_create(const ibm_grid* g, const float* d_tri, int64_t ntri, void* stream,
                                  ibm_surface** out) {
    if (!out) return ibm_fail(IBM_E_INVALID, "ibm_surface_create: null output");
    *out = nullptr;
    int rc = ibm_check_grid(g);
    if (rc) return rc;
    if (ntri < 0 || (ntri > 0 && !d_tri) || ntri > 0x7fffffffLL)
        return ibm_fail(IBM_E_INVALID, "ibm_surface_create: bad soup");
    cudaStream_t s = (cudaStream_t)stream;
    ibm_surface* S = (ibm_surface*)calloc(1, sizeof(ibm_surface));
    if (!S) return ibm_fail(IBM_E_NOMEM, "ibm_surface_create: host allocation");
    S->grid = *g;
    S->tri = d_tri;
    S->ntri = ntri;
    const int n[3] = {g->nx, g->ny, g->nz};
    S->B.nbins = 1;
    for (int a = 0; a < 3; ++a) {
        S->B.nb[a] = (n[a] - 2 * BIN_ORIGIN + BIN - 1) / BIN;
        S->B.nbins *= S->B.nb[a];
    }
    const long long nb = S->B.nbins;
    const long long nt = scan_tiles(nb) + 1;
    unsigned* cnt = nullptr;
    long long* tiles = nullptr;
    cudaError_t e = cudaSuccess;
#define SALLOC(p, bytes)                                                     \
    if (e == cudaSuccess) e = cudaMalloc((void**)&(p), (size_t)(bytes))
    SALLOC(S->off, (nb + 1) * sizeof(long long));
    SALLOC(cnt, nb * sizeof(unsigned));
    SALLOC(tiles, (nt + 1) * sizeof(long long));
    SALLOC(S->partials, 8LL * IBM_NSM * 4 * sizeof(double));
    SALLOC(S->counter, sizeof(unsigned));
    SALLOC(S->out4, 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&S->hout, 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, nb * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) {
        cudaFree(cnt);
        cudaFree(tiles);
        ibm_surface_destroy(S);
        return ibm_fail(IBM_E_NOMEM, "ibm_surface_create: %s", cudaGetErrorString(e));
    }
    if (ntri > 0) k_bin_count<<<nblocks(ntri, 256), 256, 0, s>>>(d_tri, ntri, S->B, cnt);
    e = cudaGetLastError();
    // offsets: exclusive scan of the counts, total in off[nb]
    if (e == cudaSuccess) e = scan_emit(nb, BinCount{cnt}, BinOffset{S->off}, tiles, S->off + nb, s);
    long long total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, S->off + nb, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        S->nent = total;
        e = cudaMalloc((void**)&S->ent, (size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, nb * sizeof(unsigned), s);
    if (e == cudaSuccess && ntri > 0) {
        k_bin_fill<<<nblocks(ntri, 256), 256, 0, s>>>(d_tri, ntri, S->B, S->off, cnt, S->ent);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(cnt);
    cudaFree(tiles);
    if (e != cudaSuccess) {
        ibm_surface_destroy(S);
        return ibm_cuda_check(e, "ibm_surface_create");
    }
    *out = S;
    return IBM_OK;
}

extern "C" int ibm_surface_pressure(ibm_surface* S, const double* d_p, int32_t zfilter, double* d_pside,
                                    double* h_out4, void* stream) {
    if (!S || !d_p || !d_pside) return ibm_fail(IBM_E_INVALID, "ibm_surface_pressure: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (S->ntri == 0) {
        if (h_out4) h_out4[0] = h_out4[1] = h_out4[2] = h_out4[3] = 0.0;
        return IBM_OK;
    }
    k_surface_pressure<<<nblocks(S->ntri, 128), 128, 0, s>>>(S->tri, S->ntri, S->grid.nx, S->grid.ny, S->grid.nz,
                                                              S->grid.dx, d_p, zfilter ? 1 : 0, S->B, S->off, S->ent,
                                                              d_pside, S->partials, S->counter, S->out4);
    IBM_CUDA(cudaGetLastError());
    if (h_out4) {
        IBM_CUDA(cudaMemcpyAsync(S->hout, S->out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
        IBM_CUDA(cudaStreamSynchronize(s));
        for (int q = 0; q < 4; ++q) h_out4[q] = S->hout[q];
    }
    return IBM_OK;
}

extern "C" int64_t ibm_surface_bin_entries(const ibm_surface* S) { return S ? S->nent : -1; }

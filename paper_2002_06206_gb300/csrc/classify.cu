// classify.cu -- per-geometry kernels: exact axis-aligned ray/triangle classification (Sec. 2.4.1)
// and the setup of the link records (Sec. 2.4.1-2.4.2).
//
// Every floating-point operation of the predicate and of the record coefficients is written with an
// explicit IEEE round-to-nearest intrinsic (no FMA contraction), so the result is reproducible bit
// for bit by any FP64 implementation that evaluates the same expressions in the same order.
#include <stdlib.h>

#include "scan.cuh"

namespace {

// Candidate lines of a triangle: its projected bounding box widened by this margin (grid units).
// The edge tolerance admits points at most eps_edge * (triangle height) outside the triangle.
constexpr double kLineMargin = 1e-4;
constexpr unsigned long long kEmpty = 0xffffffffffffffffULL;

struct Tri { double v[3][3]; };

__device__ __forceinline__ bool load_tri(const float* __restrict__ t, Tri& T) {
    bool ok = true;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double x = (double)t[3 * p + d];
            T.v[p][d] = x;
            ok = ok && isfinite(x);
        }
    return ok;
}

__device__ __forceinline__ long long clamp_line(double v, long long n) {
    if (!(v > -1.0)) return -1;
    if (v > (double)n) return n;
    return (long long)v;
}

// [lo, hi] of line indices j with j + 1/2 in [mn - margin, mx + margin], clamped to [0, n-1].
__device__ __forceinline__ void line_range(double mn, double mx, long long n, long long& lo, long long& hi) {
    double l = ceil(__dsub_rn(__dsub_rn(mn, kLineMargin), 0.5));
    double h = floor(__dsub_rn(__dadd_rn(mx, kLineMargin), 0.5));
    lo = l < 0.0 ? 0 : clamp_line(l, n);
    hi = clamp_line(h, n);
    if (hi > n - 1) hi = n - 1;
}

__device__ __forceinline__ void tri_lines(const Tri& T, int a, const long long n[3], long long& jb0,
                                          long long& jb1, long long& jc0, long long& jc1) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    line_range(fmin(fmin(T.v[0][b], T.v[1][b]), T.v[2][b]), fmax(fmax(T.v[0][b], T.v[1][b]), T.v[2][b]),
               n[b], jb0, jb1);
    line_range(fmin(fmin(T.v[0][c], T.v[1][c]), T.v[2][c]), fmax(fmax(T.v[0][c], T.v[1][c]), T.v[2][c]),
               n[c], jc0, jc1);
}

// Twice the signed area of (P, Q, q) in the (b, c) projection.
__device__ __forceinline__ double orient(double Pb, double Pc, double Qb, double Qc, double qb, double qc) {
    double l = __dmul_rn(__dsub_rn(Qb, Pb), __dsub_rn(qc, Pc));
    double r = __dmul_rn(__dsub_rn(Qc, Pc), __dsub_rn(qb, Pb));
    return __dsub_rn(l, r);
}

// The grid line through (qb, qc) parallel to axis a crosses the triangle iff its barycentric weights
// (w0, w1, w2)/W in the projection are all >= -eps_edge; W = 0 (|W| <= eps_det) is the parallel case
// that Moller-Trumbore's determinant test rejects.
__device__ __forceinline__ bool line_hit(const Tri& T, int a, double qb, double qc, double eps_edge,
                                         double eps_det, double& x_hit) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    const double* A = T.v[0];
    const double* B = T.v[1];
    const double* C = T.v[2];
    double w0 = orient(B[b], B[c], C[b], C[c], qb, qc);
    double w1 = orient(C[b], C[c], A[b], A[c], qb, qc);
    double w2 = orient(A[b], A[c], B[b], B[c], qb, qc);
    double W = __dadd_rn(__dadd_rn(w0, w1), w2);
    if (!(fabs(W) > eps_det)) return false;
    double thr = __dmul_rn(eps_edge, fabs(W));
    double s0 = W > 0 ? w0 : -w0, s1 = W > 0 ? w1 : -w1, s2 = W > 0 ? w2 : -w2;
    if (!(s0 >= -thr && s1 >= -thr && s2 >= -thr)) return false;
    double num = __dadd_rn(__dadd_rn(__dmul_rn(w0, A[a]), __dmul_rn(w1, B[a])), __dmul_rn(w2, C[a]));
    x_hit = __ddiv_rn(num, W);
    return true;
}

__global__ void k_fill_u64(unsigned long long* __restrict__ p, long long n, unsigned long long v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

struct LineCount {
    const float* tri;
    long long n[3];
    __device__ long long operator()(long long item) const {
        Tri T;
        if (!load_tri(tri + 9 * (item / 3), T)) return 0;
        long long jb0, jb1, jc0, jc1;
        tri_lines(T, (int)(item % 3), n, jb0, jb1, jc0, jc1);
        if (jb1 < jb0 || jc1 < jc0) return 0;
        return (jb1 - jb0 + 1) * (jc1 - jc0 + 1);
    }
};

struct StoreOffset {
    long long* off;
    __device__ void operator()(long long i, long long o, long long) const { off[i] = o; }
};

// One thread per (triangle, axis, line) test; the owning (triangle, axis) item is found by binary
// search in the exclusive offsets.  Hits update the per-face min/max of t through 64-bit integer
// atomics on the bit patterns of t >= 0 (their order is the order of the values), so the result
// does not depend on the order in which threads run.
__global__ void __launch_bounds__(256) k_test_lines(const float* __restrict__ tri, long long nitems,
                                                    const long long* __restrict__ off, const long long* __restrict__ total,
                                                    long long nx, long long ny, long long nz, double eps_edge,
                                                    double eps_det, unsigned long long* __restrict__ tmin,
                                                    unsigned long long* __restrict__ tmax) {
    const long long ntests = *total;
    const long long n[3] = {nx, ny, nz};
    const long long N = nx * ny * nz;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ntests;
         g += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = nitems - 1;        // last item with off[item] <= g
        while (lo < hi) {
            long long mid = (lo + hi + 1) >> 1;
            if (off[mid] <= g) lo = mid; else hi = mid - 1;
        }
        const long long item = lo;
        const int a = (int)(item % 3);
        Tri T;
        load_tri(tri + 9 * (item / 3), T);
        long long jb0, jb1, jc0, jc1;
        tri_lines(T, a, n, jb0, jb1, jc0, jc1);
        const long long l = g - off[item];
        const long long nb = jb1 - jb0 + 1;
        const long long jb = jb0 + l % nb, jc = jc0 + l / nb;
        double xh;
        if (!line_hit(T, a, (double)jb + 0.5, (double)jc + 0.5, eps_edge, eps_det, xh)) continue;
        double xm = __dsub_rn(xh, 0.5);
        double f = floor(xm);
        if (!(f >= 0.0 && f <= (double)(n[a] - 2))) continue;
        double t = __dsub_rn(xm, f);
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        long long x[3];
        x[a] = (long long)f;
        x[b] = jb;
        x[c] = jc;
        const long long fid = a * N + x[0] + nx * (x[1] + ny * x[2]);
        const unsigned long long bits = (unsigned long long)__double_as_longlong(t);
        atomicMin(&tmin[fid], bits);
        atomicMax(&tmax[fid], bits);
    }
}

// Flags bits 0-5 from the per-face hit table (bits 6-7 cleared).
__global__ void k_cut_flags(int nx, int ny, int nz, const unsigned long long* __restrict__ tmin,
                            uint8_t* __restrict__ flags) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / ((long long)nx * ny));
        const int x[3] = {i, j, k};
        const long long st[3] = {1, nx, (long long)nx * ny};
        unsigned f = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (tmin[a * N + c] != kEmpty) f |= 1u << (2 * a + 1);
            if (x[a] > 0 && tmin[a * N + c - st[a]] != kEmpty) f |= 1u << (2 * a);
        }
        flags[c] = (uint8_t)f;
    }
}

struct FaceHit {
    const unsigned long long* tmin;
    __device__ long long operator()(long long f) const { return tmin[f] != kEmpty ? 1 : 0; }
};

struct EmitCut {
    const unsigned long long* tmin;
    const unsigned long long* tmax;
    int64_t* face_id;
    double* t_lo;
    double* t_hi;
    long long cap;
    __device__ void operator()(long long f, long long o, long long c) const {
        if (c && o < cap) {
            face_id[o] = f;
            t_lo[o] = __longlong_as_double((long long)tmin[f]);
            t_hi[o] = __longlong_as_double((long long)tmax[f]);
        }
    }
};

struct Workspace {
    unsigned long long* tmin;
    unsigned long long* tmax;
    long long* item_off;
    long long* tiles;
    long long* scalars;   // [0] tests, [1] cut faces
    size_t bytes;
};

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

Workspace carve(void* base, long long N, long long ntri) {
    Workspace w;
    char* p = (char*)base;
    size_t o = 0;
    const long long nt = scan_tiles(3 * N > 3 * ntri ? 3 * N : 3 * ntri) + 1;
    w.tmin = (unsigned long long*)(p + o); o += align256(sizeof(unsigned long long) * 3 * N);
    w.tmax = (unsigned long long*)(p + o); o += align256(sizeof(unsigned long long) * 3 * N);
    w.item_off = (long long*)(p + o); o += align256(sizeof(long long) * (3 * ntri + 1));
    w.tiles = (long long*)(p + o); o += align256(sizeof(long long) * nt);
    w.scalars = (long long*)(p + o); o += align256(sizeof(long long) * 4);
    w.bytes = o;
    return w;
}

unsigned blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    long long cap = 32LL * IBM_NSM;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

extern "C" size_t ibm_classify_workspace_bytes(const ibm_grid* g, int64_t ntri) {
    if (!g || g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || ntri < 0) return 0;
    return carve(nullptr, (long long)g->nx * g->ny * g->nz, ntri).bytes;
}

int ibm_check_grid(const ibm_grid* g);

extern "C" int ibm_classify(const ibm_grid* g, const float* d_tri, int64_t ntri, const ibm_geom_params* gp,
                            uint8_t* d_flags, int64_t* d_face_id, double* d_t_lo, double* d_t_hi, int64_t cap,
                            int64_t* n_cut, int64_t* n_tests, void* d_ws, size_t ws_bytes, void* stream) {
    int rc = ibm_check_grid(g);
    if (rc) return rc;
    if (!gp || !d_flags || !n_cut || (ntri > 0 && !d_tri) || ntri < 0 || cap < 0 ||
        (cap > 0 && (!d_face_id || !d_t_lo || !d_t_hi)))
        return ibm_fail(IBM_E_INVALID, "ibm_classify: null or negative argument");
    const long long N = (long long)g->nx * g->ny * g->nz;
    Workspace w = carve(d_ws, N, ntri);
    if (!d_ws || ws_bytes < w.bytes)
        return ibm_fail(IBM_E_INVALID, "ibm_classify: workspace of %zu bytes, %zu needed", ws_bytes, w.bytes);
    cudaStream_t s = (cudaStream_t)stream;
    k_fill_u64<<<blocks_for(3 * N, 256), 256, 0, s>>>(w.tmin, 3 * N, kEmpty);
    k_fill_u64<<<blocks_for(3 * N, 256), 256, 0, s>>>(w.tmax, 3 * N, 0ULL);
    IBM_LAUNCHED("ibm_classify: fill");
    const long long nitems = 3 * ntri;
    if (nitems > 0) {
        LineCount lc{d_tri, {g->nx, g->ny, g->nz}};
        IBM_CUDA(scan_emit(nitems, lc, StoreOffset{w.item_off}, w.tiles, w.scalars + 0, s));
        k_test_lines<<<32 * IBM_NSM, 256, 0, s>>>(d_tri, nitems, w.item_off, w.scalars + 0, g->nx, g->ny, g->nz,
                                                  gp->eps_edge, gp->eps_det, w.tmin, w.tmax);
        IBM_LAUNCHED("ibm_classify: k_test_lines");
    } else {
        IBM_CUDA(cudaMemsetAsync(w.scalars, 0, sizeof(long long), s));
    }
    k_cut_flags<<<blocks_for(N, 256), 256, 0, s>>>(g->nx, g->ny, g->nz, w.tmin, d_flags);
    IBM_LAUNCHED("ibm_classify: k_cut_flags");
    // count first; the list is only written when it fits
    IBM_CUDA(scan_emit(3 * N, FaceHit{w.tmin}, EmitCut{w.tmin, w.tmax, d_face_id, d_t_lo, d_t_hi, cap},
                       w.tiles, w.scalars + 1, s));
    long long host[2];
    IBM_CUDA(cudaMemcpyAsync(host, w.scalars, sizeof(host), cudaMemcpyDeviceToHost, s));
    IBM_CUDA(cudaStreamSynchronize(s));
    *n_cut = host[1];
    if (n_tests) *n_tests = host[0];
    if (host[1] > cap)
        return ibm_fail(IBM_E_CAPACITY, "ibm_classify: %lld cut faces, capacity %lld", host[1], (long long)cap);
    return IBM_OK;
}

// ------------------------------------------------------------------------------------------------
// Setup

struct ibm_geom {
    ibm_grid grid;
    ibm_geom_params gp;
    long long N;
    long long n_cut, n_rec, n_inc;
    uint8_t* flags;        // caller-owned
    int32_t* cellrec;      // [N]
    int32_t* inc;          // [n_inc] Omega_inc cells in index order
    LinkRec* rec;          // [n_rec]
};

namespace {

__global__ void k_region_bits(int nx, int ny, int nz, uint8_t* __restrict__ flags) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const unsigned f = flags[c] & 63u;
        unsigned out = f;
        if (f) {
            out |= 64u;
        } else {
            const int x[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
            const int n[3] = {nx, ny, nz};
            const long long st[3] = {1, nx, (long long)nx * ny};
            bool adj = false;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (x[a] > 0 && (flags[c - st[a]] & 63u)) adj = true;
                if (x[a] < n[a] - 1 && (flags[c + st[a]] & 63u)) adj = true;
            }
            if (adj) out |= 128u;
        }
        flags[c] = (uint8_t)out;
    }
}

// Packed count per cell: records in the low 32 bits, one Omega_inc slot in the high bits.
struct RecCount {
    const uint8_t* flags;
    __device__ long long operator()(long long c) const {
        const unsigned f = flags[c] & 63u;
        return f ? ((1LL << 32) | (long long)__popc(f)) : 0;
    }
};

struct EmitCellrec {
    int32_t* cellrec;
    int32_t* inc;
    __device__ void operator()(long long c, long long o, long long cnt) const {
        if (cnt) {
            cellrec[c] = (int32_t)(o & 0xffffffffLL);
            inc[o >> 32] = (int32_t)c;
        } else {
            cellrec[c] = -1;
        }
    }
};

__device__ __forceinline__ long long find_face(const int64_t* __restrict__ fid, long long n, long long key) {
    long long lo = 0, hi = n - 1;
    while (lo <= hi) {
        long long mid = lo + ((hi - lo) >> 1);
        long long v = fid[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// Eq. q_axis: upper branch (Dx/d) q_IB + ((d - Dx)/d) q_P on d/Dx >= 1/2; lower branch
// 2 q_IB + ((2d - Dx)/Dx) q_O - (2d/Dx) q_P on d/Dx < 1/2 when the opposite neighbour O is usable;
// otherwise the upper branch at d = 1/2.  Eq. distribution_function weights with the near distance d.
__global__ void k_build_records(int nx, int ny, int nz, const uint8_t* __restrict__ flags,
                                const int32_t* __restrict__ inc, long long n_inc,
                                const int32_t* __restrict__ cellrec, const int64_t* __restrict__ fid,
                                const double* __restrict__ t_lo, const double* __restrict__ t_hi, long long n_cut,
                                LinkRec* __restrict__ rec, int* __restrict__ err) {
    const long long N = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n_inc; q += (long long)gridDim.x * blockDim.x) {
        const long long P = inc[q];
        const unsigned f = flags[P] & 63u;
        const int x[3] = {(int)(P % nx), (int)((P / nx) % ny), (int)(P / ((long long)nx * ny))};
        const int n[3] = {nx, ny, nz};
        const long long st[3] = {1, nx, (long long)nx * ny};
        int k = cellrec[P];
        for (int bit = 0; bit < 6; ++bit) {
            if (!((f >> bit) & 1u)) continue;
            const int a = bit >> 1, s = (bit & 1) ? 1 : -1;
            const long long lower = s > 0 ? P : P - st[a];
            const long long idx = find_face(fid, n_cut, a * N + lower);
            LinkRec r;
            if (idx < 0) {
                atomicExch(err, 1);
                r = LinkRec{};
                rec[k++] = r;
                continue;
            }
            const double d = s > 0 ? t_lo[idx] : __dsub_rn(1.0, t_hi[idx]);
            r.cell = (int32_t)P;
            r.far = (int32_t)(P + s * st[a]);
            r.axis = (int8_t)a;
            r.side = (int8_t)s;
            r.pad = 0;
            r.d = d;
            const int yo = x[a] - s;
            const bool o_ok = yo >= 0 && yo < n[a] && !((f >> (2 * a + (s > 0 ? 0 : 1))) & 1u);
            if (d >= 0.5) {
                r.branch = 0;
                r.opp = -1;
                r.c_ib = __ddiv_rn(1.0, d);
                r.c_p = __ddiv_rn(__dsub_rn(d, 1.0), d);
                r.c_o = 0.0;
            } else if (o_ok) {
                r.branch = 1;
                r.opp = (int32_t)(P - s * st[a]);
                r.c_ib = 2.0;
                r.c_o = __dsub_rn(__dmul_rn(2.0, d), 1.0);
                r.c_p = -__dmul_rn(2.0, d);
            } else {
                r.branch = 2;
                r.opp = -1;
                r.c_ib = 2.0;
                r.c_p = -1.0;
                r.c_o = 0.0;
            }
            const double den = __dadd_rn(1.0, d);
            r.w_fluid = __ddiv_rn(d, den);
            r.w_ghost = __ddiv_rn(__dsub_rn(1.0, d), den);
            r.uib[0] = r.uib[1] = r.uib[2] = 0.0;
            rec[k++] = r;
        }
    }
}

__global__ void k_export(const LinkRec* __restrict__ rec, long long n, int64_t* __restrict__ idx,
                         double* __restrict__ coef) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const LinkRec& r = rec[q];
        if (idx) {
            idx[6 * q + 0] = r.cell;
            idx[6 * q + 1] = r.far;
            idx[6 * q + 2] = r.opp;
            idx[6 * q + 3] = r.axis;
            idx[6 * q + 4] = r.side;
            idx[6 * q + 5] = r.branch;
        }
        if (coef) {
            coef[6 * q + 0] = r.d;
            coef[6 * q + 1] = r.c_ib;
            coef[6 * q + 2] = r.c_p;
            coef[6 * q + 3] = r.c_o;
            coef[6 * q + 4] = r.w_fluid;
            coef[6 * q + 5] = r.w_ghost;
        }
    }
}

__global__ void k_export_cellrec(const int32_t* __restrict__ cr, long long n, int64_t* __restrict__ out) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        out[q] = cr[q];
}

__global__ void k_set_uib(LinkRec* __restrict__ rec, long long n, const double* __restrict__ uib) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) rec[q].uib[c] = uib ? uib[3 * q + c] : 0.0;
}

}  // namespace

extern "C" void ibm_geom_destroy(ibm_geom* G) {
    if (!G) return;
    cudaFree(G->cellrec);
    cudaFree(G->inc);
    cudaFree(G->rec);
    free(G);
}

extern "C" int ibm_setup(const ibm_grid* g, const ibm_geom_params* gp, uint8_t* d_flags, const int64_t* d_face_id,
                         const double* d_t_lo, const double* d_t_hi, int64_t n_cut, ibm_geom** out, void* stream) {
    int rc = ibm_check_grid(g);
    if (rc) return rc;
    if (!gp || !d_flags || !out || n_cut < 0 || (n_cut > 0 && (!d_face_id || !d_t_lo || !d_t_hi)))
        return ibm_fail(IBM_E_INVALID, "ibm_setup: null or negative argument");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    ibm_geom* G = (ibm_geom*)calloc(1, sizeof(ibm_geom));
    if (!G) return ibm_fail(IBM_E_NOMEM, "ibm_setup: host allocation");
    G->grid = *g;
    G->gp = *gp;
    G->N = (long long)g->nx * g->ny * g->nz;
    G->n_cut = n_cut;
    G->flags = d_flags;
    long long* tiles = nullptr;
    int* d_err = nullptr;
    long long host[2] = {0, 0};
    int herr = 0;
    const long long nt = scan_tiles(G->N) + 1;
    cudaError_t e;
    if ((e = cudaMalloc(&G->cellrec, sizeof(int32_t) * G->N)) != cudaSuccess ||
        (e = cudaMalloc(&tiles, sizeof(long long) * (nt + 2))) != cudaSuccess ||
        (e = cudaMalloc(&d_err, sizeof(int))) != cudaSuccess) {
        cudaFree(tiles);
        cudaFree(d_err);
        ibm_geom_destroy(G);
        return ibm_fail(IBM_E_NOMEM, "ibm_setup: %s", cudaGetErrorString(e));
    }
    // inc list sized after the count is known: count into a scratch of N int32 first
    if ((e = cudaMalloc(&G->inc, sizeof(int32_t) * (G->N > 0 ? G->N : 1))) != cudaSuccess) goto nomem;
    k_region_bits<<<blocks_for(G->N, 256), 256, 0, s>>>(g->nx, g->ny, g->nz, d_flags);
    if ((e = scan_emit(G->N, RecCount{d_flags}, EmitCellrec{G->cellrec, G->inc}, tiles, tiles + nt, s)) != cudaSuccess)
        goto cuda_err;
    if ((e = cudaMemcpyAsync(host, tiles + nt, sizeof(long long), cudaMemcpyDeviceToHost, s)) != cudaSuccess) goto cuda_err;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) goto cuda_err;
    G->n_rec = host[0] & 0xffffffffLL;
    G->n_inc = host[0] >> 32;
    if (G->n_rec != 2 * n_cut) {
        cudaFree(tiles);
        cudaFree(d_err);
        ibm_geom_destroy(G);
        return ibm_fail(IBM_E_INVALID, "ibm_setup: flags name %lld cut links but the list has %lld faces",
                        (long long)host[0] & 0xffffffffLL, (long long)n_cut);
    }
    if ((e = cudaMalloc(&G->rec, sizeof(LinkRec) * (G->n_rec > 0 ? G->n_rec : 1))) != cudaSuccess) goto nomem;
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(int), s)) != cudaSuccess) goto cuda_err;
    if (G->n_inc > 0)
        k_build_records<<<blocks_for(G->n_inc, 128), 128, 0, s>>>(g->nx, g->ny, g->nz, d_flags, G->inc, G->n_inc,
                                                                  G->cellrec, d_face_id, d_t_lo, d_t_hi, n_cut,
                                                                  G->rec, d_err);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_err;
    if ((e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) goto cuda_err;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) goto cuda_err;
    cudaFree(tiles);
    cudaFree(d_err);
    if (herr) {
        ibm_geom_destroy(G);
        return ibm_fail(IBM_E_INVALID, "ibm_setup: a cut link has no entry in the cut-face list");
    }
    *out = G;
    return IBM_OK;
nomem:
    cudaFree(tiles);
    cudaFree(d_err);
    ibm_geom_destroy(G);
    return ibm_fail(IBM_E_NOMEM, "ibm_setup: %s", cudaGetErrorString(e));
cuda_err:
    cudaFree(tiles);
    cudaFree(d_err);
    ibm_geom_destroy(G);
    return ibm_cuda_check(e, "ibm_setup");
}

extern "C" int ibm_geom_info(const ibm_geom* G, int64_t* n_rec, int64_t* n_inc) {
    if (!G) return ibm_fail(IBM_E_INVALID, "ibm_geom_info: null geometry");
    if (n_rec) *n_rec = G->n_rec;
    if (n_inc) *n_inc = G->n_inc;
    return IBM_OK;
}

extern "C" int ibm_geom_export(const ibm_geom* G, int64_t* d_idx, double* d_coef, int64_t* d_cellrec, void* stream) {
    if (!G) return ibm_fail(IBM_E_INVALID, "ibm_geom_export: null geometry");
    cudaStream_t s = (cudaStream_t)stream;
    if ((d_idx || d_coef) && G->n_rec > 0) k_export<<<blocks_for(G->n_rec, 256), 256, 0, s>>>(G->rec, G->n_rec, d_idx, d_coef);
    if (d_cellrec && G->N > 0) k_export_cellrec<<<blocks_for(G->N, 256), 256, 0, s>>>(G->cellrec, G->N, d_cellrec);
    IBM_LAUNCHED("ibm_geom_export");
    return IBM_OK;
}

extern "C" int ibm_set_boundary_velocity(ibm_geom* G, const double* d_uib, void* stream) {
    if (!G) return ibm_fail(IBM_E_INVALID, "ibm_set_boundary_velocity: null geometry");
    if (G->n_rec > 0) k_set_uib<<<blocks_for(G->n_rec, 256), 256, 0, (cudaStream_t)stream>>>(G->rec, G->n_rec, d_uib);
    IBM_LAUNCHED("ibm_set_boundary_velocity");
    return IBM_OK;
}

// Accessors for the solver (api.cu).
void ibm_geom_device(const ibm_geom* G, const uint8_t** flags, const int32_t** cellrec, const LinkRec** rec,
                     const int32_t** inc, long long* n_rec, long long* n_inc) {
    *flags = G->flags;
    *cellrec = G->cellrec;
    *rec = G->rec;
    *inc = G->inc;
    *n_rec = G->n_rec;
    *n_inc = G->n_inc;
}
const ibm_grid* ibm_geom_grid(const ibm_geom* G) { return &G->grid; }
int ibm_geom_deadend(const ibm_geom* G) { return G->gp.deadend_on ? 1 : 0; }

// ------------------------------------------------------------------------------------------------
// Classification without any allocation, for callers that cannot call cudaMalloc.
//
// The scratch lives in a fixed device array of this file.  Its name in host code is only a host-side
// stand-in, so the device address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and cached; kernels receive that address.  The cache holds for the life of the
// device's context: a cudaDeviceReset invalidates it (documented in the header).

#include <mutex>

#define IBM_NOALLOC_SCRATCH_BYTES (32u << 20)   // 32 MiB, held by every GPU that loads the library
#define IBM_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[IBM_NOALLOC_SCRATCH_BYTES];

static void* g_noalloc_ptr[IBM_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

extern "C" int ibm_classify_noalloc(const ibm_grid* g, const float* d_tri, int64_t ntri, const ibm_geom_params* gp,
                                    uint8_t* d_flags, int64_t* d_face_id, double* d_t_lo, double* d_t_hi,
                                    int64_t cap, int64_t* n_cut, int64_t* n_tests, void* stream) {
    int rc = ibm_check_grid(g);
    if (rc) return rc;
    if (ntri < 0) return ibm_fail(IBM_E_INVALID, "ibm_classify_noalloc: negative triangle count");
    const size_t need = ibm_classify_workspace_bytes(g, ntri);
    if (need > IBM_NOALLOC_SCRATCH_BYTES)
        return ibm_fail(IBM_E_INVALID,
                        "ibm_classify_noalloc: this grid and soup need %zu bytes of scratch, more than the "
                        "%u bytes the library reserves; use ibm_classify with a caller workspace",
                        need, (unsigned)IBM_NOALLOC_SCRATCH_BYTES);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ibm_cuda_check(e, "ibm_classify_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= IBM_NOALLOC_MAX_DEVICES)
        return ibm_fail(IBM_E_INVALID, "ibm_classify_noalloc: device ordinal %d not supported", dev);
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return ibm_cuda_check(e, "ibm_classify_noalloc: cudaGetSymbolAddress");
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    // every part of the scratch that must start from a known value is initialised by ibm_classify
    return ibm_classify(g, d_tri, ntri, gp, d_flags, d_face_id, d_t_lo, d_t_hi, cap, n_cut, n_tests, scratch,
                        IBM_NOALLOC_SCRATCH_BYTES, stream);
}

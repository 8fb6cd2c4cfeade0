// common.cuh -- device-side conventions shared by the library's kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ibmles.h"

#define IBM_NSM 152                    // streaming multiprocessors of a GB300
#define IBM_TX 32                      // cell kernels: 32 x 8 threads over an (x, y) tile,
#define IBM_TY 8                       // each thread marching along z over a chunk of planes

// One cut link seen from the cell that reads across it (Sec. 2.4.1-2.4.2).
struct LinkRec {
    int32_t cell;      // P
    int32_t far;       // G = P + side e_axis (the cell behind the wall)
    int32_t opp;       // O = P - side e_axis when the lower ghost branch is used, else -1
    int8_t axis, side, branch, pad;
    double d;          // wall distance from P along the link, in units of dx
    double c_ib, c_p, c_o;
    double w_fluid, w_ghost;  // Eq. distribution_function at d: fluid branch, ghost branch (forcing)
    double uib[3];
};

// Everything a cell kernel needs to know about the grid, the boundaries and the immersed body.
struct Dom {
    int nx, ny, nz;
    int sy;            // nx
    long long sz;      // nx * ny
    long long N;
    double dx;
    double idx;                // 1 / dx
    float fdx, fidx;           // dx, 1 / dx rounded to FP32 (FP32 kernels do no FP64 arithmetic per cell)
    int bc[6];
    double u_in[3];
    const uint8_t* flags;      // may be null: no body
    const int32_t* cellrec;    // first record of each Omega_inc cell, -1 elsewhere
    const LinkRec* rec;
    int hom;                   // 1: ghost values without wall and inflow velocities (linear part)
    const uint8_t* fast;       // momentum flux: 1 where the tiled fast path applies (may be null)
    long long nrec;            // link records (two per cut face)
};

__device__ __forceinline__ int link_bit(int a, int s) { return 2 * a + (s > 0); }

// dx and 1/dx in the working precision (set on the host; GB300's FP64 rate is a small fraction of its
// FP32 rate, so a per-cell FP64 division would dominate an FP32 stencil).
template <class T> __device__ __forceinline__ T dom_dx(const Dom& D);
template <> __device__ __forceinline__ float dom_dx<float>(const Dom& D) { return D.fdx; }
template <> __device__ __forceinline__ double dom_dx<double>(const Dom& D) { return D.dx; }
template <class T> __device__ __forceinline__ T dom_idx(const Dom& D);
template <> __device__ __forceinline__ float dom_idx<float>(const Dom& D) { return D.fidx; }
template <> __device__ __forceinline__ double dom_idx<double>(const Dom& D) { return D.idx; }

__device__ __forceinline__ const LinkRec& link_record(const Dom& D, long long P, unsigned fl, int bit) {
    return D.rec[D.cellrec[P] + __popc(fl & 63u & ((1u << bit) - 1u))];
}

// Offset of neighbour P + s e_a, or 0x7fffffff... when it is beyond a non-periodic domain face.
// x_a is the cell's coordinate along a.
__device__ __forceinline__ bool nb_offset(const Dom& D, int a, int s, int xa, long long& off) {
    const int n = a == 0 ? D.nx : (a == 1 ? D.ny : D.nz);
    const long long st = a == 0 ? 1 : (a == 1 ? (long long)D.sy : D.sz);
    const int y = xa + s;
    if (y >= 0 && y < n) { off = s * st; return true; }
    if (D.bc[link_bit(a, s)] != IBM_BC_PERIODIC) return false;
    off = -(long long)s * (n - 1) * st;
    return true;
}

// Value of velocity component `comp` that cell P reads across link (a, s): the neighbour's value,
// the IB ghost of Eq. q_axis on a cut link, or the domain-boundary ghost.
template <class T>
__device__ __forceinline__ T vel_across(const Dom& D, const T* __restrict__ u, int comp, long long P,
                                        int xa, unsigned fl, int a, int s) {
    const long long cN = (long long)comp * D.N;
    const T uP = u[cN + P];
    const int bit = link_bit(a, s);
    if (fl & (1u << bit)) {
        const LinkRec& r = link_record(D, P, fl, bit);
        T v = (D.hom ? (T)0 : (T)r.c_ib * (T)r.uib[comp]) + (T)r.c_p * uP;
        if (r.opp >= 0) v = v + (T)r.c_o * u[cN + r.opp];
        return v;
    }
    long long off;
    if (nb_offset(D, a, s, xa, off)) return u[cN + P + off];
    switch (D.bc[bit]) {
        case IBM_BC_INFLOW: return (D.hom ? (T)0 : (T)2 * (T)D.u_in[comp]) - uP;
        case IBM_BC_OUTFLOW: return uP;
        case IBM_BC_SLIP: return comp == a ? -uP : uP;
        default: return -uP;
    }
}

// Pressure read across link (a, s): Neumann on cut links and walls/inflow, p = 0 at outflow faces.
template <class T>
__device__ __forceinline__ T p_across(const Dom& D, const T* __restrict__ p, long long P, int xa,
                                      unsigned fl, int a, int s) {
    const int bit = link_bit(a, s);
    if (fl & (1u << bit)) return p[P];
    long long off;
    if (nb_offset(D, a, s, xa, off)) return p[P + off];
    return D.bc[bit] == IBM_BC_OUTFLOW ? -p[P] : p[P];
}

// Face offsets in the concatenated Ux | Uy | Uz vector.
struct FaceLayout {
    long long off[3];
    int dim[3][3];   // dims of the face array of axis a: dim[a][0..2]
    __host__ __device__ long long index(int a, int i, int j, int k) const {
        return off[a] + i + (long long)dim[a][0] * (j + (long long)dim[a][1] * k);
    }
};

inline FaceLayout make_faces(int nx, int ny, int nz) {
    FaceLayout F;
    int d[3] = {nx, ny, nz};
    long long o = 0;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) F.dim[a][b] = d[b] + (a == b);
        F.off[a] = o;
        o += (long long)F.dim[a][0] * F.dim[a][1] * F.dim[a][2];
    }
    return F;
}

// Block-wide sum of a double (any block size that is a multiple of 32, <= 1024); result in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int w = tid >> 5;
    const int nw = (blockDim.x * blockDim.y * blockDim.z) >> 5;
    if ((tid & 31) == 0) sh[w] = v;
    (void)lane;
    __syncthreads();
    v = 0.0;
    if (tid < 32) {
        v = tid < nw ? sh[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// Block-wide sum of per-thread FP32 partials, in FP32 (GB300 runs FP64 at a small fraction of its
// FP32 rate, and an FP64 shuffle tree in every block of a one-cell-per-thread launch costs more than
// the kernel's own arithmetic); the block total is widened to FP64 for the grid stage.
__device__ __forceinline__ double block_sum(float v, double* sh) {
    float* shf = reinterpret_cast<float*>(sh);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int w = tid >> 5;
    const int nw = (blockDim.x * blockDim.y * blockDim.z) >> 5;
    if ((tid & 31) == 0) shf[w] = v;
    __syncthreads();
    v = 0.f;
    if (tid < 32) {
        v = tid < nw ? shf[tid] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return (double)v;
}

// Deterministic grid-wide reduction of `nv` values per block (double, or float summed in FP32 within
// the block): every block stores its partials in FP64, the last block to arrive sums them in block
// order and calls fin(totals).  `counter` must be zero on entry and is left zero.
template <int NV, class A, class Fin>
__device__ __forceinline__ void grid_reduce(A (&v)[NV], double* __restrict__ partials,
                                            unsigned int* counter, Fin fin) {
    __shared__ double sh[32];
    __shared__ bool last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = block_sum(v[q], sh);
        if (tid == 0) partials[(size_t)q * nblk + bid] = s;
    }
    if (tid == 0) {
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double tot[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = 0.0;
        for (unsigned b = tid; b < nblk; b += nthr) s += ((volatile double*)partials)[(size_t)q * nblk + b];
        tot[q] = block_sum(s, sh);
    }
    if (tid == 0) {
        fin(tot);
        *counter = 0u;
    }
}

// Flat launch of the stencil kernels: 32 x 8 threads over an (x, y) tile, each thread handling
// IBM_KU consecutive planes (loop fully unrolled, so all its loads are independent and in flight
// together).
#define IBM_KU 4
inline dim3 flat_grid(int nx, int ny, int nz, int planes = IBM_KU) {
    return dim3((unsigned)((nx + IBM_TX - 1) / IBM_TX), (unsigned)((ny + IBM_TY - 1) / IBM_TY),
                (unsigned)((nz + planes - 1) / planes));
}

// 7-point link sum  sum_links g (v_N - v_P) - d v_P  of a value function on the fine grid, with a
// fast path for a cell with no cut link away from the domain faces (g = 1 on all six links).
template <class T, class Get>
__device__ __forceinline__ T link_sum7(const Dom& D, long long P, int i, int j, int k, unsigned fl, T vP, Get get) {
    if (fl == 0u && i > 0 && i < D.nx - 1 && j > 0 && j < D.ny - 1 && k > 0 && k < D.nz - 1)
        return ((get(P - 1) + get(P + 1)) + (get(P - D.sy) + get(P + D.sy))) + (get(P - D.sz) + get(P + D.sz)) -
               (T)6 * vP;
    const int x[3] = {i, j, k};
    T sum = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            const int bit = 2 * a + (s > 0);
            if (fl & (1u << bit)) continue;
            long long off;
            if (nb_offset(D, a, s, x[a], off)) sum += get(P + off) - vP;
            else if (D.bc[bit] == IBM_BC_OUTFLOW) sum += -vP - vP;
        }
    return sum;
}

// Launch geometry of the cell kernels.
struct CellGrid {
    dim3 grid, block;
    int kchunk;
};

// Chooses the z-chunk so that the blocks fill whole waves of the SMs: with `res` resident blocks of
// 256 threads per SM, a launch takes ceil(blocks / (res * SMs)) waves of (kchunk + 1) plane steps
// (the +1 is the plane each column loads before its first one).
inline CellGrid cell_grid(int nx, int ny, int nz, int res = 4) {
    CellGrid g;
    g.block = dim3(IBM_TX, IBM_TY, 1);
    const long long gx = (nx + IBM_TX - 1) / IBM_TX, gy = (ny + IBM_TY - 1) / IBM_TY;
    const long long slots = (long long)res * IBM_NSM;
    long long best_cost = -1;
    int best_k = nz;
    for (int gz = 1; gz <= nz; ++gz) {
        const int kc = (nz + gz - 1) / gz;
        const long long gze = (nz + kc - 1) / kc;
        const long long blocks = gx * gy * gze;
        const long long waves = (blocks + slots - 1) / slots;
        const long long cost = waves * (kc + 1);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_k = kc;
        }
        if (kc == 1) break;
    }
    g.kchunk = best_k;
    g.grid = dim3((unsigned)gx, (unsigned)gy, (unsigned)((nz + best_k - 1) / best_k));
    return g;
}

inline unsigned cell_blocks(const CellGrid& g) { return g.grid.x * g.grid.y * g.grid.z; }

// Host-side error recording and argument checks (api.cu).
int ibm_fail(int code, const char* fmt, ...);
int ibm_check_grid(const ibm_grid* g);
int ibm_cuda_check(cudaError_t e, const char* what);
#define IBM_CUDA(call)                                                     \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ibm_cuda_check(e_, #call);           \
    } while (0)
#define IBM_LAUNCHED(what)                                                 \
    do {                                                                   \
        cudaError_t e_ = cudaGetLastError();                               \
        if (e_ != cudaSuccess) return ibm_cuda_check(e_, what);            \
    } while (0)

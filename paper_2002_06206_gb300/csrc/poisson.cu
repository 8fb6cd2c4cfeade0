// poisson.cu -- the pressure Poisson solve (Sec. 2.1, Eq. poisson): the link-masked 7-point operator,
// conjugate gradients in the working precision inside FP64 iterative refinement, BiCGStab and
// red-black SOR (the two solvers the paper names).
//
// The operator is symmetric by construction (a link carries a flux iff its face is uncut, and both
// cells of a face agree on that), so CG applies; it needs half the memory traffic of BiCGStab per
// iteration.  The Krylov scalars live on the device: each kernel reads alpha/beta from the previous
// kernel's grid reduction, and the host only reads the residual every check_every iterations.
// Kernels return at once when the device-side `done` flag is set, so launching a few iterations
// past convergence costs only launch latency.
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "solver.cuh"

namespace {

// sum over the six links of (v_N - v_P), Neumann on cut links and walls, v = 0 at outflow faces.
template <class T, class Get>
__device__ __forceinline__ T link_sum(const Dom& D, long long P, const int x[3], unsigned fl, T vP, Get get) {
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

__device__ __forceinline__ unsigned flags_at(const Dom& D, long long P) { return D.flags ? (unsigned)D.flags[P] : 0u; }

#define CELL_LOOP_BEGIN                                                             \
    const int i = blockIdx.x * IBM_TX + threadIdx.x, j = blockIdx.y * IBM_TY + threadIdx.y; \
    const bool active = i < D.nx && j < D.ny;                                     \
    const int k0 = blockIdx.z * kchunk, k1 = active ? min(D.nz, k0 + kchunk) : k0; \
    for (int k = k0; k < k1; ++k) {                                               \
        const long long P = i + (long long)D.sy * j + D.sz * k;                   \
        const int x[3] = {i, j, k};                                               \
        const unsigned fl = flags_at(D, P);
#define CELL_LOOP_END }

template <class T>
__global__ void __launch_bounds__(256) k_apply(Dom D, const T* __restrict__ p, T* __restrict__ Ap, T idx2, int kchunk) {
    CELL_LOOP_BEGIN
    const T vP = p[P];
    Ap[P] = link_sum<T>(D, P, x, fl, vP, [&](long long n) { return p[n]; }) * idx2;
    CELL_LOOP_END
}

// r = b - A x in FP64; stores r in the working precision; res2 = ||r||^2 (FP64), rr = ||(Tr) r||^2.
template <class Tr>
__global__ void __launch_bounds__(256) k_residual(Dom D, const double* __restrict__ b, const double* __restrict__ x64,
                                                  Tr* __restrict__ r, double idx2, SolveScal* sc, double* partials,
                                                  unsigned* counter) {
    Tr part0 = 0, part1 = 0;     // norms accumulated per thread in the working precision
    const int i = blockIdx.x * IBM_TX + threadIdx.x, j = blockIdx.y * IBM_TY + threadIdx.y;
    const int kb = blockIdx.z * IBM_KU;
    const bool active = i < D.nx && j < D.ny;
    auto xv = [&](long long n) { return x64[n]; };
#pragma unroll
    for (int u = 0; u < IBM_KU; ++u) {
        const int k = kb + u;
        if (active && k < D.nz) {
            const long long P = i + (long long)D.sy * j + D.sz * k;
            const unsigned fl = D.flags ? (unsigned)D.flags[P] : 0u;
            const double ap = link_sum7<double>(D, P, i, j, k, fl, x64[P], xv) * idx2;
            const double rv = b[P] - ap;
            const Tr rt = (Tr)rv;
            if (r) r[P] = rt;
            if constexpr (std::is_same<Tr, double>::value) part0 += rv * rv;
            else part0 += rt * rt;
            part1 += rt * rt;
        }
    }
    decltype(part0) acc[2] = {part0, part1};
    grid_reduce<2>(acc, partials, counter, [&](double* t) {
        sc->res2 = t[0];
        sc->rr = t[1];
        if (!isfinite(t[0])) sc->nonfinite = 1;
    });
}

__global__ void __launch_bounds__(256) k_dot_bb(Dom D, const double* __restrict__ b, SolveScal* sc, double* partials,
                                                unsigned* counter, int kchunk) {
    double acc[1] = {0.0};
    CELL_LOOP_BEGIN
    (void)fl;
    (void)x;
    acc[0] += b[P] * b[P];
    CELL_LOOP_END
    grid_reduce<1>(acc, partials, counter, [&](double* t) { sc->bb = t[0]; });
}

__global__ void k_begin_cycle(SolveScal* sc, double target2, int maxit) {
    sc->target2 = target2;
    sc->restart = 1;
    sc->maxit = maxit;
    sc->done = (sc->rr <= target2 || sc->iters >= maxit || sc->nonfinite) ? 1 : 0;
}

__global__ void k_add_iters(SolveScal* sc, int n) { sc->iters += n; }

__global__ void k_reset(SolveScal* sc) {
    sc->iters = 0;
    sc->nonfinite = 0;
    sc->done = 0;
    sc->dev_error = 0;
}

// CG, first half: direction p = r + beta p_old (recomputed where a neighbour needs it, so p never
// needs a pass of its own), q = A p, and (p, q).  Flat launch: each thread takes IBM_KU planes of one
// (i, j) column, unrolled, so its loads are all independent.
template <class T>
__global__ void __launch_bounds__(256) k_cg_dir_spmv(Dom D, const T* __restrict__ r, const T* __restrict__ pold,
                                                     T* __restrict__ pnew, T* __restrict__ q, T idx2, SolveScal* sc,
                                                     double* partials, unsigned* counter, int pcg) {
    if (sc->done) return;
    const T beta = sc->restart ? (T)0 : (T)(pcg ? sc->rz / sc->rz_old : sc->rr / sc->rr_old);
    const int i = blockIdx.x * IBM_TX + threadIdx.x, j = blockIdx.y * IBM_TY + threadIdx.y;
    const int kb = blockIdx.z * IBM_KU;
    const bool active = i < D.nx && j < D.ny;
    auto pv = [&](long long c) { return r[c] + beta * pold[c]; };
    T part = 0;       // per-thread partial sum in the working precision (FP64 arithmetic is slow here)
#pragma unroll
    for (int u = 0; u < IBM_KU; ++u) {
        const int k = kb + u;
        if (active && k < D.nz) {
            const long long P = i + (long long)D.sy * j + D.sz * k;
            const unsigned fl = D.flags ? (unsigned)D.flags[P] : 0u;
            const T pc = pv(P);
            const T qv = link_sum7<T>(D, P, i, j, k, fl, pc, pv) * idx2;
            pnew[P] = pc;
            q[P] = qv;
            part += pc * qv;
        }
    }
    decltype(part) acc[1] = {part};
    grid_reduce<1>(acc, partials, counter, [&](double* t) { sc->pq = t[0]; });
}

template <class T>
void launch_dir_spmv(const LesCtx& c, const T* src, const T* pold, T* pnew, T* q, T idx2, SolveScal* sc, int pcg,
                     cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (x4_ok(c)) {
            launch_cg_dir_spmv_x4(c, src, pold, pnew, q, idx2, sc, pcg, s);
            return;
        }
    }
    k_cg_dir_spmv<T><<<c.fgrid, c.cg.block, 0, s>>>(c.D, src, pold, pnew, q, idx2, sc, c.partials, c.counter, pcg);
}

// CG, second half: x += alpha p, r -= alpha q, (r, r), convergence and iteration cap.  A pure stream:
// 16-byte vector loads and stores when the arrays allow it.
template <class T>
struct Vec4;
template <>
struct Vec4<float> { using type = float4; };
template <>
struct Vec4<double> { using type = double2; };

template <class T>
__global__ void __launch_bounds__(256) k_cg_update(long long N, const T* __restrict__ p, const T* __restrict__ q,
                                                   T* __restrict__ x, T* __restrict__ r, SolveScal* sc,
                                                   double* partials, unsigned* counter, int pcg) {
    if (sc->done) return;
    const T alpha = (T)((pcg ? sc->rz : sc->rr) / sc->pq);
    T part = 0;
    using V = typename Vec4<T>::type;
    constexpr int W = sizeof(V) / sizeof(T);
    const bool aligned = ((((uintptr_t)p) | ((uintptr_t)q) | ((uintptr_t)x) | ((uintptr_t)r)) & 15u) == 0;
    const long long nv = aligned ? N / W : 0;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, nth = (long long)gridDim.x * blockDim.x;
    for (long long v = tid; v < nv; v += nth) {
        V pv = reinterpret_cast<const V*>(p)[v];
        V qv = reinterpret_cast<const V*>(q)[v];
        V xv = reinterpret_cast<V*>(x)[v];
        V rv = reinterpret_cast<V*>(r)[v];
        T* pe = reinterpret_cast<T*>(&pv);
        T* qe = reinterpret_cast<T*>(&qv);
        T* xe = reinterpret_cast<T*>(&xv);
        T* re = reinterpret_cast<T*>(&rv);
#pragma unroll
        for (int e = 0; e < W; ++e) {
            xe[e] = xe[e] + alpha * pe[e];
            re[e] = re[e] - alpha * qe[e];
            part += re[e] * re[e];
        }
        reinterpret_cast<V*>(x)[v] = xv;
        reinterpret_cast<V*>(r)[v] = rv;
    }
    for (long long c = nv * W + tid; c < N; c += nth) {
        x[c] = x[c] + alpha * p[c];
        const T rv = r[c] - alpha * q[c];
        r[c] = rv;
        part += rv * rv;
    }
    decltype(part) acc[1] = {part};
    grid_reduce<1>(acc, partials, counter, [&](double* t) {
        sc->rr_old = sc->rr;
        sc->rr = t[0];
        sc->restart = 0;
        sc->iters += 1;
        if (!isfinite(t[0])) {
            sc->nonfinite = 1;
            sc->done = 1;
        } else if (t[0] <= sc->target2 || sc->iters >= sc->maxit) {
            sc->done = 1;
        }
    });
}

__global__ void k_add_correction(long long N, double* __restrict__ x, const float* __restrict__ e) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        x[c] += (double)e[c];
}

// Red-black SOR sweep of one colour ((i + j + k) mod 2), in place on the FP64 iterate.
__global__ void __launch_bounds__(256) k_sor(Dom D, const double* __restrict__ b, double* __restrict__ xv, double idx2,
                                             double omega, int colour, int kchunk) {
    CELL_LOOP_BEGIN
    if (((i + j + k) & 1) != colour) continue;
    double diag = 0.0, off = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            const int bit = 2 * a + (s > 0);
            if (fl & (1u << bit)) continue;
            long long o;
            if (nb_offset(D, a, s, x[a], o)) {
                diag -= idx2;
                off += xv[P + o] * idx2;
            } else if (D.bc[bit] == IBM_BC_OUTFLOW) {
                diag -= 2.0 * idx2;
            }
        }
    if (diag == 0.0) continue;
    const double gs = (b[P] - off) / diag;
    xv[P] = (1.0 - omega) * xv[P] + omega * gs;
    CELL_LOOP_END
}

unsigned lin_blocks(long long n) {
    long long b = (n + 255) / 256;
    long long cap = 8LL * IBM_NSM;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

int read_scalars(PoissonWork& w, cudaStream_t s) {
    IBM_CUDA(cudaMemcpyAsync(w.hsc, w.sc, sizeof(SolveScal), cudaMemcpyDeviceToHost, s));
    IBM_CUDA(cudaEventRecord(w.ev, s));
    IBM_CUDA(cudaEventSynchronize(w.ev));
    return IBM_OK;
}

// CG iterations on A x = r0 (r already holds the residual, sc->rr its norm) until the device says done.
template <class T>
int cg_cycles(const LesCtx& c, PoissonWork& w, T* x, int check_every, cudaStream_t s) {
    const T idx2 = (T)(1.0 / (c.D.dx * c.D.dx));
    T* r = (T*)w.r;
    T* pa = (T*)w.pa;
    T* pb = (T*)w.pb;
    T* q = (T*)w.q;
    const unsigned nb = lin_blocks(c.D.N);
    for (int m = 0;;) {
        for (int it = 0; it < check_every; ++it, ++m) {
            T* pold = (m & 1) ? pb : pa;
            T* pnew = (m & 1) ? pa : pb;
            prof_begin(c.prof, PS_CG_SPMV, s);
            launch_dir_spmv<T>(c, r, pold, pnew, q, idx2, w.sc, 0, s);
            prof_end(c.prof, PS_CG_SPMV, s);
            prof_begin(c.prof, PS_CG_UPDATE, s);
            k_cg_update<T><<<nb, 256, 0, s>>>(c.D.N, pnew, q, x, r, w.sc, c.partials, c.counter, 0);
            prof_end(c.prof, PS_CG_UPDATE, s);
        }
        IBM_COUNT(c, 2 * check_every);
        IBM_LAUNCHED("cg iteration");
        int rc = read_scalars(w, s);
        if (rc) return rc;
        if (w.hsc->done) return IBM_OK;
    }
}

// ---- BiCGStab (Sec. 2.1) -------------------------------------------------------------------------
// Three kernels per iteration.  Each recomputes the vector its operator needs at the neighbours
// (p = r + beta (p_old - omega v_old), s = r - alpha v), so neither p nor s costs a pass of its own.

// Generic 7-point link sum of a value function on the z-marching layout (no register reuse: the
// BiCGStab operands combine three arrays).
template <class T, class Val>
__device__ __forceinline__ T apply_at(const Dom& D, long long P, const int x[3], unsigned fl, T vP, Val val) {
    return link_sum<T>(D, P, x, fl, vP, val);
}

template <class T>
__global__ void __launch_bounds__(256) k_bicg_pv(Dom D, const T* __restrict__ r, const T* __restrict__ rh,
                                                 const T* __restrict__ pold, const T* __restrict__ vold,
                                                 T* __restrict__ pnew, T* __restrict__ vnew, T idx2, SolveScal* sc,
                                                 double* partials, unsigned* counter, int kchunk) {
    if (sc->done) return;
    const bool restart = sc->restart != 0;
    const T beta = restart ? (T)0 : (T)((sc->rho / sc->rho_old) * (sc->alpha / sc->omega));
    const T om = restart ? (T)0 : (T)sc->omega;
    auto pv = [&](long long c) { return restart ? r[c] : r[c] + beta * (pold[c] - om * vold[c]); };
    T acc[1] = {(T)0};
    CELL_LOOP_BEGIN
    const T pc = pv(P);
    const T v = apply_at<T>(D, P, x, fl, pc, pv) * idx2;
    pnew[P] = pc;
    vnew[P] = v;
    acc[0] += rh[P] * v;
    CELL_LOOP_END
    grid_reduce<1>(acc, partials, counter, [&](double* t) {
        sc->rv = t[0];
        sc->alpha = t[0] != 0.0 ? sc->rho / t[0] : 0.0;
        if (t[0] == 0.0 || !isfinite(t[0])) sc->done = 1;          // breakdown: the host restarts
    });
}

template <class T>
__global__ void __launch_bounds__(256) k_bicg_st(Dom D, const T* __restrict__ r, const T* __restrict__ v,
                                                 T* __restrict__ sv, T* __restrict__ tv, T idx2, SolveScal* sc,
                                                 double* partials, unsigned* counter, int kchunk) {
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    auto sf = [&](long long c) { return r[c] - alpha * v[c]; };
    T acc[3] = {(T)0, (T)0, (T)0};
    CELL_LOOP_BEGIN
    const T sc_ = sf(P);
    const T t = apply_at<T>(D, P, x, fl, sc_, sf) * idx2;
    sv[P] = sc_;
    tv[P] = t;
    acc[0] += t * sc_;
    acc[1] += t * t;
    acc[2] += sc_ * sc_;
    CELL_LOOP_END
    grid_reduce<3>(acc, partials, counter, [&](double* t) {
        sc->ts = t[0];
        sc->tt = t[1];
        sc->ss = t[2];
        sc->omega = t[1] > 0.0 ? t[0] / t[1] : 0.0;
    });
}

template <class T>
__global__ void __launch_bounds__(256) k_bicg_xr(long long N, const T* __restrict__ p, const T* __restrict__ sv,
                                                 const T* __restrict__ tv, const T* __restrict__ rh, T* __restrict__ x,
                                                 T* __restrict__ r, SolveScal* sc, double* partials, unsigned* counter) {
    if (sc->done) return;
    const T alpha = (T)sc->alpha, om = (T)sc->omega;
    T acc[2] = {(T)0, (T)0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        x[c] = x[c] + alpha * p[c] + om * sv[c];
        const T rv = sv[c] - om * tv[c];
        r[c] = rv;
        acc[0] += rh[c] * rv;
        acc[1] += rv * rv;
    }
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
            sc->done = 1;                                           // converged, capped or broke down
        }
    });
}

__global__ void k_bicg_begin(SolveScal* sc) {
    sc->rho = sc->rr;            // (r_hat, r) with r_hat = r
    sc->rho_old = 1.0;
    sc->alpha = 1.0;
    sc->omega = 1.0;
}

template <class T>
int bicg_cycles(const LesCtx& c, PoissonWork& w, T* x, int check_every, cudaStream_t s) {
    const T idx2 = (T)(1.0 / (c.D.dx * c.D.dx));
    T* r = (T*)w.r;
    T* rh = (T*)w.rh;
    T* pa = (T*)w.pa;
    T* pb = (T*)w.pb;
    T* va = (T*)w.q;
    T* vb = (T*)w.vb;
    T* sv = (T*)w.sv;
    T* tv = (T*)w.tv;
    const unsigned nb = lin_blocks(c.D.N);
    IBM_CUDA(cudaMemcpyAsync(rh, r, sizeof(T) * c.D.N, cudaMemcpyDeviceToDevice, s));
    k_bicg_begin<<<1, 1, 0, s>>>(w.sc);
    IBM_COUNT(c, 1);
    for (int m = 0;;) {
        for (int it = 0; it < check_every; ++it, ++m) {
            T* pold = (m & 1) ? pb : pa;
            T* pnew = (m & 1) ? pa : pb;
            T* vold = (m & 1) ? vb : va;
            T* vnew = (m & 1) ? va : vb;
            prof_begin(c.prof, PS_CG_SPMV, s);
            k_bicg_pv<T><<<c.cg.grid, c.cg.block, 0, s>>>(c.D, r, rh, pold, vold, pnew, vnew, idx2, w.sc, c.partials,
                                                          c.counter, c.cg.kchunk);
            k_bicg_st<T><<<c.cg.grid, c.cg.block, 0, s>>>(c.D, r, vnew, sv, tv, idx2, w.sc, c.partials, c.counter,
                                                          c.cg.kchunk);
            prof_end(c.prof, PS_CG_SPMV, s);
            prof_begin(c.prof, PS_CG_UPDATE, s);
            k_bicg_xr<T><<<nb, 256, 0, s>>>(c.D.N, pnew, sv, tv, rh, x, r, w.sc, c.partials, c.counter);
            prof_end(c.prof, PS_CG_UPDATE, s);
        }
        IBM_LAUNCHED("bicgstab iteration");
        IBM_COUNT(c, 3 * check_every);
        int rc = read_scalars(w, s);
        if (rc) return rc;
        if (w.hsc->done) return IBM_OK;
    }
}

// Preconditioned CG: z = V-cycle(r) (which also forms (r, z)), then the same two kernels as CG with
// beta = (r,z)/(r,z)_old and alpha = (r,z)/(p,Ap).
template <class T>
int pcg_iteration(const LesCtx& c, PoissonWork& w, T* x, int m, cudaStream_t s) {
    const T idx2 = (T)(1.0 / (c.D.dx * c.D.dx));
    T* r = (T*)w.r;
    T* z = (T*)w.z;
    T* pold = (m & 1) ? (T*)w.pb : (T*)w.pa;
    T* pnew = (m & 1) ? (T*)w.pa : (T*)w.pb;
    T* q = (T*)w.q;
    int rc = mg_vcycle<T>(c, *c.mg, r, z, w.sc, s);
    if (rc) return rc;
    prof_begin(c.prof, PS_CG_SPMV, s);
    launch_dir_spmv<T>(c, z, pold, pnew, q, idx2, w.sc, 1, s);
    prof_end(c.prof, PS_CG_SPMV, s);
    prof_begin(c.prof, PS_CG_UPDATE, s);
    k_cg_update<T><<<lin_blocks(c.D.N), 256, 0, s>>>(c.D.N, pnew, q, x, r, w.sc, c.partials, c.counter, 1);
    prof_end(c.prof, PS_CG_UPDATE, s);
    IBM_LAUNCHED("pcg iteration");
    IBM_COUNT(c, 2);
    return IBM_OK;
}

// Captures two iterations (parities 0 and 1) into one executable graph, for solution vector x.
template <class T>
int pcg_capture(const LesCtx& c, PoissonWork& w, T* x) {
    if (w.gexec) {
        cudaGraphExecDestroy(w.gexec);
        w.gexec = nullptr;
    }
    long long before = c.nlaunch ? *c.nlaunch : 0;
    IBM_CUDA(cudaStreamBeginCapture(w.cap, cudaStreamCaptureModeThreadLocal));
    int rc = pcg_iteration<T>(c, w, x, 0, w.cap);
    if (!rc) rc = pcg_iteration<T>(c, w, x, 1, w.cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(w.cap, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return ibm_cuda_check(e, "pcg graph capture");
    e = cudaGraphInstantiate(&w.gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        w.gexec = nullptr;
        return ibm_cuda_check(e, "pcg graph instantiate");
    }
    w.glaunches = (c.nlaunch ? *c.nlaunch : 0) - before;
    if (c.nlaunch) *c.nlaunch = before;
    w.gkey = x;
    w.gprec = (int)sizeof(T);
    return IBM_OK;
}

template <class T>
int pcg_cycles(const LesCtx& c, PoissonWork& w, T* x, int check_every, cudaStream_t s) {
    const bool graphs = w.cap && !(c.prof && c.prof->on);
    if (graphs && (!w.gexec || w.gkey != (const void*)x || w.gprec != (int)sizeof(T))) {
        int rc = pcg_capture<T>(c, w, x);
        if (rc) return rc;
    }
    const int pairs = (check_every + 1) / 2;
    double rr_last = -1.0;
    for (int m = 0;;) {
        if (graphs) {
            for (int q = 0; q < pairs; ++q) IBM_CUDA(cudaGraphLaunch(w.gexec, s));
            IBM_COUNT(c, w.glaunches * pairs);
            m += 2 * pairs;
        } else {
            for (int it = 0; it < check_every; ++it, ++m) {
                int rc = pcg_iteration<T>(c, w, x, m, s);
                if (rc) return rc;
            }
        }
        int rc = read_scalars(w, s);
        if (rc) return rc;
        if (w.hsc->done) return IBM_OK;
        // an inner solve that has stopped converging (at the floor of its working precision) hands back
        // to the refinement: less than a factor 2 of residual norm over a whole check interval
        const double rr = w.hsc->rr;
        if (rr_last > 0.0 && rr > 0.25 * rr_last) return IBM_OK;
        rr_last = rr;
    }
}

}  // namespace

void launch_reset(SolveScal* sc, cudaStream_t s) { k_reset<<<1, 1, 0, s>>>(sc); }

// Residual norms of two candidate iterates in one pass: res2 of xa -> out[0], of xb -> out[1].
__global__ void __launch_bounds__(256) k_two_residuals(Dom D, const double* __restrict__ b, const double* __restrict__ xa,
                                                       const double* __restrict__ xb, double idx2, double* partials,
                                                       unsigned* counter, double* out) {
    const int i = blockIdx.x * IBM_TX + threadIdx.x, j = blockIdx.y * IBM_TY + threadIdx.y;
    const int kb = blockIdx.z * IBM_KU;
    const bool active = i < D.nx && j < D.ny;
    // only compares the two starting points, so FP32 arithmetic on the rounded iterates suffices
    float p0 = 0.f, p1 = 0.f;
    const float fidx2 = (float)idx2;
    auto va = [&](long long n) { return (float)xa[n]; };
    auto vb = [&](long long n) { return (float)xb[n]; };
#pragma unroll
    for (int u = 0; u < IBM_KU; ++u) {
        const int k = kb + u;
        if (active && k < D.nz) {
            const long long P = i + (long long)D.sy * j + D.sz * k;
            const unsigned fl = D.flags ? (unsigned)D.flags[P] : 0u;
            const float bp = (float)b[P];
            const float ra = bp - link_sum7<float>(D, P, i, j, k, fl, (float)xa[P], va) * fidx2;
            const float rb = bp - link_sum7<float>(D, P, i, j, k, fl, (float)xb[P], vb) * fidx2;
            p0 += ra * ra;
            p1 += rb * rb;
        }
    }
    decltype(p0) acc[2] = {p0, p1};
    grid_reduce<2>(acc, partials, counter, [&](double* t) {
        out[0] = t[0];
        out[1] = t[1];
    });
}

int launch_two_residuals(const LesCtx& c, const double* b, const double* xa, const double* xb, double* out,
                         cudaStream_t s) {
    k_two_residuals<<<c.fgrid, c.cg.block, 0, s>>>(c.D, b, xa, xb, 1.0 / (c.D.dx * c.D.dx), c.partials, c.counter, out);
    IBM_LAUNCHED("k_two_residuals");
    IBM_COUNT(c, 1);
    return IBM_OK;
}

int launch_apply64(const LesCtx& c, const double* p, double* Ap, cudaStream_t s) {
    k_apply<double><<<c.cg.grid, c.cg.block, 0, s>>>(c.D, p, Ap, 1.0 / (c.D.dx * c.D.dx), c.cg.kchunk);
    IBM_LAUNCHED("k_apply");
    IBM_COUNT(c, 1);
    return IBM_OK;
}

int run_poisson(const LesCtx& c, PoissonWork& w, const double* b, double* x, double tol, int maxit, int solver,
                int check_every, double inner_tol, double omega, les_stats* st, cudaStream_t s) {
    const double idx2 = 1.0 / (c.D.dx * c.D.dx);
    if (check_every <= 0) check_every = 16;
    if (inner_tol <= 0.0) inner_tol = 1e-4;
    if (omega <= 0.0) omega = 1.9;
    les_stats out = {};
    k_reset<<<1, 1, 0, s>>>(w.sc);
    k_dot_bb<<<c.cg.grid, c.cg.block, 0, s>>>(c.D, b, w.sc, c.partials, c.counter, c.cg.kchunk);
    IBM_LAUNCHED("k_dot_bb");
    IBM_COUNT(c, 2);
    int rc = IBM_OK;
    int outer = 0;
    const int max_outer = 64;
    for (;;) {
        // true residual in FP64; the Krylov residual array receives it in the working precision
        prof_begin(c.prof, PS_RESIDUAL, s);
        if (solver == IBM_SOLVER_RBSOR)
            k_residual<double><<<c.fgrid, c.cg.block, 0, s>>>(c.D, b, x, (double*)nullptr, idx2, w.sc, c.partials,
                                                              c.counter);
        else if (c.prec == IBM_FP64)
            k_residual<double><<<c.fgrid, c.cg.block, 0, s>>>(c.D, b, x, (double*)w.r, idx2, w.sc, c.partials,
                                                              c.counter);
        else
            k_residual<float><<<c.fgrid, c.cg.block, 0, s>>>(c.D, b, x, (float*)w.r, idx2, w.sc, c.partials, c.counter);
        prof_end(c.prof, PS_RESIDUAL, s);
        IBM_LAUNCHED("k_residual");
        IBM_COUNT(c, 1);
        if ((rc = read_scalars(w, s))) return rc;
        const SolveScal h = *w.hsc;
        if (h.dev_error) return ibm_fail(IBM_E_CUDA, "poisson_solve: a multigrid shared-memory load timed out");
        out.bnorm = sqrt(h.bb);
        out.relres = h.bb > 0.0 ? sqrt(h.res2 / h.bb) : 0.0;
        out.iters = h.iters;
        out.outer = outer;
        if (h.nonfinite || !isfinite(h.res2)) { rc = IBM_E_NONFINITE; break; }
        if (h.bb == 0.0 || h.res2 <= tol * tol * h.bb) { rc = IBM_OK; break; }
        if (h.iters >= maxit || (solver != IBM_SOLVER_RBSOR && outer >= max_outer)) { rc = IBM_E_NOCONV; break; }
        ++outer;
        if (solver == IBM_SOLVER_RBSOR) {
            for (int it = 0; it < check_every; ++it) {
                prof_begin(c.prof, PS_SOR, s);
                k_sor<<<c.cg.grid, c.cg.block, 0, s>>>(c.D, b, x, idx2, omega, 0, c.cg.kchunk);
                k_sor<<<c.cg.grid, c.cg.block, 0, s>>>(c.D, b, x, idx2, omega, 1, c.cg.kchunk);
                prof_end(c.prof, PS_SOR, s);
            }
            IBM_LAUNCHED("k_sor");
            k_add_iters<<<1, 1, 0, s>>>(w.sc, check_every);
            IBM_COUNT(c, 2 * check_every + 1);
            continue;
        }
        if (c.prec == IBM_FP64) {
            k_begin_cycle<<<1, 1, 0, s>>>(w.sc, 0.81 * tol * tol * h.bb, maxit);
            IBM_COUNT(c, 1);
            if (solver == IBM_SOLVER_BICGSTAB) {
                if ((rc = bicg_cycles<double>(c, w, x, check_every, s))) return rc;
            } else if (c.mg) {
                if ((rc = pcg_cycles<double>(c, w, x, check_every, s))) return rc;
            } else if ((rc = cg_cycles<double>(c, w, x, check_every, s))) {
                return rc;
            }
        } else {
            double t2 = inner_tol * inner_tol * h.rr;
            const double floor2 = 0.25 * tol * tol * h.bb;
            if (t2 < floor2) t2 = floor2;
            IBM_CUDA(cudaMemsetAsync(w.e, 0, sizeof(float) * c.D.N, s));
            k_begin_cycle<<<1, 1, 0, s>>>(w.sc, t2, maxit);
            IBM_COUNT(c, 1);
            if (solver == IBM_SOLVER_BICGSTAB) {
                if ((rc = bicg_cycles<float>(c, w, (float*)w.e, check_every, s))) return rc;
            } else if (c.mg) {
                if ((rc = pcg_cycles<float>(c, w, (float*)w.e, check_every, s))) return rc;
            } else if ((rc = cg_cycles<float>(c, w, (float*)w.e, check_every, s))) {
                return rc;
            }
            k_add_correction<<<lin_blocks(c.D.N), 256, 0, s>>>(c.D.N, x, (const float*)w.e);
            IBM_LAUNCHED("k_add_correction");
            IBM_COUNT(c, 1);
        }
    }
    out.status = rc;
    if (st) *st = out;
    return rc;
}

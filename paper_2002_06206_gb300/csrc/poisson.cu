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
                                                  unsigned* counter, int kchunk) {
    double acc[2] = {0.0, 0.0};
    CELL_LOOP_BEGIN
    const double vP = x64[P];
    const double ap = link_sum<double>(D, P, x, fl, vP, [&](long long n) { return x64[n]; }) * idx2;
    const double rv = b[P] - ap;
    const Tr rt = (Tr)rv;
    if (r) r[P] = rt;
    acc[0] += rv * rv;
    acc[1] += (double)rt * (double)rt;
    CELL_LOOP_END
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
}

// CG, first half: direction p = r + beta p_old (recomputed at the neighbours, so p never needs a
// separate pass), q = A p, and (p, q).
template <class T>
__global__ void __launch_bounds__(256) k_cg_dir_spmv(Dom D, const T* __restrict__ r, const T* __restrict__ pold,
                                                     T* __restrict__ pnew, T* __restrict__ q, T idx2, SolveScal* sc,
                                                     double* partials, unsigned* counter, int kchunk) {
    if (sc->done) return;
    const T beta = sc->restart ? (T)0 : (T)(sc->rr / sc->rr_old);
    double acc[1] = {0.0};
    CELL_LOOP_BEGIN
    const T pn = r[P] + beta * pold[P];
    const T qv = link_sum<T>(D, P, x, fl, pn, [&](long long n) { return r[n] + beta * pold[n]; }) * idx2;
    pnew[P] = pn;
    q[P] = qv;
    acc[0] += (double)pn * (double)qv;
    CELL_LOOP_END
    grid_reduce<1>(acc, partials, counter, [&](double* t) { sc->pq = t[0]; });
}

// CG, second half: x += alpha p, r -= alpha q, (r, r), convergence and iteration cap.
template <class T>
__global__ void __launch_bounds__(256) k_cg_update(long long N, const T* __restrict__ p, const T* __restrict__ q,
                                                   T* __restrict__ x, T* __restrict__ r, SolveScal* sc,
                                                   double* partials, unsigned* counter) {
    if (sc->done) return;
    const T alpha = (T)(sc->rr / sc->pq);
    double acc[1] = {0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        x[c] = x[c] + alpha * p[c];
        const T rv = r[c] - alpha * q[c];
        r[c] = rv;
        acc[0] += (double)rv * (double)rv;
    }
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
            k_cg_dir_spmv<T><<<c.cg.grid, c.cg.block, 0, s>>>(c.D, r, pold, pnew, q, idx2, w.sc, c.partials, c.counter,
                                                              c.cg.kchunk);
            prof_end(c.prof, PS_CG_SPMV, s);
            prof_begin(c.prof, PS_CG_UPDATE, s);
            k_cg_update<T><<<nb, 256, 0, s>>>(c.D.N, pnew, q, x, r, w.sc, c.partials, c.counter);
            prof_end(c.prof, PS_CG_UPDATE, s);
        }
        IBM_COUNT(c, 2 * check_every);
        IBM_LAUNCHED("cg iteration");
        int rc = read_scalars(w, s);
        if (rc) return rc;
        if (w.hsc->done) return IBM_OK;
    }
}

}  // namespace

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
            k_residual<double><<<c.cg.grid, c.cg.block, 0, s>>>(c.D, b, x, (double*)nullptr, idx2, w.sc, c.partials,
                                                                c.counter, c.cg.kchunk);
        else if (c.prec == IBM_FP64)
            k_residual<double><<<c.cg.grid, c.cg.block, 0, s>>>(c.D, b, x, (double*)w.r, idx2, w.sc, c.partials,
                                                                c.counter, c.cg.kchunk);
        else
            k_residual<float><<<c.cg.grid, c.cg.block, 0, s>>>(c.D, b, x, (float*)w.r, idx2, w.sc, c.partials, c.counter,
                                                               c.cg.kchunk);
        prof_end(c.prof, PS_RESIDUAL, s);
        IBM_LAUNCHED("k_residual");
        IBM_COUNT(c, 1);
        if ((rc = read_scalars(w, s))) return rc;
        const SolveScal h = *w.hsc;
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
            if ((rc = cg_cycles<double>(c, w, x, check_every, s))) return rc;
        } else {
            double t2 = inner_tol * inner_tol * h.rr;
            const double floor2 = 0.25 * tol * tol * h.bb;
            if (t2 < floor2) t2 = floor2;
            IBM_CUDA(cudaMemsetAsync(w.e, 0, sizeof(float) * c.D.N, s));
            k_begin_cycle<<<1, 1, 0, s>>>(w.sc, t2, maxit);
            IBM_COUNT(c, 1);
            if ((rc = cg_cycles<float>(c, w, (float*)w.e, check_every, s))) return rc;
            k_add_correction<<<lin_blocks(c.D.N), 256, 0, s>>>(c.D.N, x, (const float*)w.e);
            IBM_LAUNCHED("k_add_correction");
            IBM_COUNT(c, 1);
        }
    }
    out.status = rc;
    if (st) *st = out;
    return rc;
}

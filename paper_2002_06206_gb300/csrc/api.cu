// api.cu -- the C ABI of the library (declared in include/ibmles.h): argument checks, state and
// workspace management, and the composition of one fractional step from the kernels.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <math.h>
#include <string.h>

#include "solver.cuh"

static thread_local char g_err[512] = "";

int ibm_fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int ibm_cuda_check(cudaError_t e, const char* what) {
    snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? IBM_E_NOMEM : IBM_E_CUDA;
}

extern "C" const char* ibm_last_error(void) { return g_err; }

int ibm_check_grid(const ibm_grid* g) {
    if (!g) return ibm_fail(IBM_E_INVALID, "null grid");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return ibm_fail(IBM_E_INVALID, "grid %d x %d x %d: every extent must be >= 1", g->nx, g->ny, g->nz);
    const long long N = (long long)g->nx * g->ny * g->nz;
    if (N > (1LL << 31) / 3) return ibm_fail(IBM_E_INVALID, "grid of %lld cells exceeds 2^31/3", N);
    if (!(g->dx > 0.0)) return ibm_fail(IBM_E_INVALID, "dx must be positive");
    return IBM_OK;
}

void ibm_geom_device(const ibm_geom* G, const uint8_t** flags, const int32_t** cellrec, const LinkRec** rec,
                     const int32_t** inc, long long* n_rec, long long* n_inc);
const ibm_grid* ibm_geom_grid(const ibm_geom* G);
int ibm_geom_deadend(const ibm_geom* G);

void prof_begin(Prof* p, int slot, cudaStream_t s) {
    if (!p || !p->on) return;
    if (p->used[slot] == p->cap) {          // flush this slot's finished pairs
        cudaEventSynchronize(p->ev[slot][2 * p->cap - 1]);
        for (int q = 0; q < p->cap; ++q) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p->ev[slot][2 * q], p->ev[slot][2 * q + 1]) == cudaSuccess) p->ms[slot] += ms;
        }
        p->used[slot] = 0;
    }
    cudaEventRecord(p->ev[slot][2 * p->used[slot]], s);
}

void prof_end(Prof* p, int slot, cudaStream_t s) {
    if (!p || !p->on) return;
    cudaEventRecord(p->ev[slot][2 * p->used[slot] + 1], s);
    p->used[slot] += 1;
    p->launches[slot] += 1;
}

static void prof_free(Prof* p) {
    if (!p) return;
    for (int q = 0; q < PS_COUNT; ++q) {
        if (!p->ev[q]) continue;
        for (int e = 0; e < 2 * p->cap; ++e) cudaEventDestroy(p->ev[q][e]);
        free(p->ev[q]);
    }
    free(p);
}

struct les_state {
    ibm_grid grid;
    les_params prm;
    LesCtx c;
    PoissonWork w;
    void* nut;
    void* ustar;
    void* Ustar;
    double* b;
    double* out4;
    double* hfs;        // pinned: forcing sums of the last step
    size_t s;           // bytes of a field value
    long long nlaunch;  // kernel launches since creation or the last les_profile(st, 1)
    ibm_net* net;       // learned initial guess, or null
    double* p_prev;     // p^{n-1}
    double* p_keep;     // p^n kept across the solve
    double* x_guess;
    double* two_res;    // [2] residual norms of p^n and of the guess
    long long steps;    // steps taken (the guess needs p^{n-1})
};

static void free_state(les_state* S) {
    if (!S) return;
    cudaFree(S->nut);
    cudaFree(S->ustar);
    cudaFree(S->Ustar);
    cudaFree(S->b);
    cudaFree(S->out4);
    cudaFree(S->w.r);
    cudaFree(S->w.pa);
    cudaFree(S->w.pb);
    cudaFree(S->w.q);
    cudaFree(S->w.e);
    cudaFree(S->w.rh);
    cudaFree(S->w.sv);
    cudaFree(S->w.tv);
    cudaFree(S->w.vb);
    cudaFree(S->w.sc);
    cudaFreeHost(S->w.hsc);
    cudaFreeHost(S->hfs);
    if (S->w.ev) cudaEventDestroy(S->w.ev);
    if (S->w.gexec) cudaGraphExecDestroy(S->w.gexec);
    if (S->w.cap) cudaStreamDestroy(S->w.cap);
    cudaFree(S->c.partials);
    cudaFree(S->c.counter);
    cudaFree(S->c.fscal);
    cudaFree(S->c.fdelta);
    cudaFree(S->w.z);
    cudaFree(S->p_prev);
    cudaFree(S->p_keep);
    cudaFree(S->x_guess);
    cudaFree(S->two_res);
    cudaFree(S->c.general);
    cudaFree(S->c.fastmask);
    if (S->c.cn) {
        CNWork* w = S->c.cn;
        cudaFree(w->r); cudaFree(w->rh); cudaFree(w->p); cudaFree(w->v); cudaFree(w->sv); cudaFree(w->tv);
        cudaFree(w->x); cudaFree(w->sc);
        cudaFreeHost(w->hsc);
        free(w);
    }
    if (S->c.mg) {
        mg_free(*S->c.mg);
        free(S->c.mg);
    }
    prof_free(S->c.prof);
    free(S);
}

extern "C" void les_destroy(les_state* S) { free_state(S); }

static int check_params(const les_params* p) {
    if (!p) return ibm_fail(IBM_E_INVALID, "null params");
    if (p->precision != IBM_FP64 && p->precision != IBM_FP32_REFINE64)
        return ibm_fail(IBM_E_INVALID, "unknown precision %d", p->precision);
    if (p->solver < IBM_SOLVER_CG || p->solver > IBM_SOLVER_RBSOR)
        return ibm_fail(IBM_E_INVALID, "unknown solver %d", p->solver);
    for (int f = 0; f < 6; ++f)
        if (p->bc[f] < IBM_BC_PERIODIC || p->bc[f] > IBM_BC_NOSLIP)
            return ibm_fail(IBM_E_INVALID, "unknown boundary type %d on face %d", p->bc[f], f);
    for (int a = 0; a < 3; ++a)
        if ((p->bc[2 * a] == IBM_BC_PERIODIC) != (p->bc[2 * a + 1] == IBM_BC_PERIODIC))
            return ibm_fail(IBM_E_INVALID, "periodic boundary on axis %d must be set on both faces", a);
    if (!(p->dt > 0.0) || !(p->nu >= 0.0)) return ibm_fail(IBM_E_INVALID, "dt must be > 0 and nu >= 0");
    if (!(p->tol > 0.0)) return ibm_fail(IBM_E_INVALID, "tol must be > 0");
    if (p->precond != 0 && p->precond != 1) return ibm_fail(IBM_E_INVALID, "unknown preconditioner %d", p->precond);
    if (p->precond && p->mg_omega != 0.0 && !(p->mg_omega > 0.0 && p->mg_omega < 2.0))
        return ibm_fail(IBM_E_INVALID, "mg_omega must lie in (0, 2) for a symmetric positive preconditioner");
    if (p->precond && p->mg_sweeps < 0) return ibm_fail(IBM_E_INVALID, "mg_sweeps must be >= 0");
    if (p->mg_passes != 0 && p->mg_passes != 1) return ibm_fail(IBM_E_INVALID, "mg_passes must be 0 or 1");
    if (!(p->quick >= 0.0 && p->quick <= 1.0)) return ibm_fail(IBM_E_INVALID, "quick must lie in [0, 1]");
    if (p->integrator != IBM_ADAMS_BASHFORTH && p->integrator != IBM_CRANK_NICOLSON)
        return ibm_fail(IBM_E_INVALID, "unknown integrator %d", p->integrator);
    if (p->integrator == IBM_CRANK_NICOLSON && (!(p->mom_tol >= 0.0) || p->mom_max_iter < 0))
        return ibm_fail(IBM_E_INVALID, "mom_tol must be >= 0 and mom_max_iter >= 0");
    return IBM_OK;
}

#define ALLOC(ptr, bytes)                                                                \
    do {                                                                                 \
        cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes) > 0 ? (bytes) : 16);          \
        if (e_ != cudaSuccess) {                                                         \
            free_state(S);                                                               \
            return ibm_fail(IBM_E_NOMEM, "les_create: %s (%zu bytes)", cudaGetErrorString(e_), (size_t)(bytes)); \
        }                                                                                \
    } while (0)

extern "C" int les_create(const ibm_grid* g, const les_params* p, const ibm_geom* geom, les_state** out) {
    int rc = ibm_check_grid(g);
    if (rc) return rc;
    if ((rc = check_params(p))) return rc;
    if (!out) return ibm_fail(IBM_E_INVALID, "les_create: null output");
    *out = nullptr;
    if (geom) {
        const ibm_grid* gg = ibm_geom_grid(geom);
        if (gg->nx != g->nx || gg->ny != g->ny || gg->nz != g->nz)
            return ibm_fail(IBM_E_INVALID, "les_create: geometry grid differs from the solver grid");
    }
    les_state* S = (les_state*)calloc(1, sizeof(les_state));
    if (!S) return ibm_fail(IBM_E_NOMEM, "les_create: host allocation");
    S->grid = *g;
    S->prm = *p;
    LesCtx& c = S->c;
    c.D.nx = g->nx;
    c.D.ny = g->ny;
    c.D.nz = g->nz;
    c.D.sy = g->nx;
    c.D.sz = (long long)g->nx * g->ny;
    c.D.N = (long long)g->nx * g->ny * g->nz;
    c.D.dx = g->dx;
    c.D.idx = 1.0 / g->dx;
    c.D.fdx = (float)g->dx;
    c.D.fidx = (float)(1.0 / g->dx);
    for (int f = 0; f < 6; ++f) c.D.bc[f] = p->bc[f];
    for (int a = 0; a < 3; ++a) c.D.u_in[a] = p->u_in[a];
    if (geom) {
        ibm_geom_device(geom, &c.D.flags, &c.D.cellrec, &c.D.rec, &c.inc, &c.n_rec, &c.n_inc);
        c.D.nrec = c.n_rec;
    }
    c.F = make_faces(g->nx, g->ny, g->nz);
    c.NF = c.F.off[2] + (long long)c.F.dim[2][0] * c.F.dim[2][1] * c.F.dim[2][2];
    c.cg = cell_grid(g->nx, g->ny, g->nz);
    c.fgrid = flat_grid(g->nx, g->ny, g->nz);
    c.pgrid = flat_grid(g->nx, g->ny, g->nz, 1);
    c.cgrid = flat_grid(g->nx, g->ny, g->nz, 2 * IBM_KU);
    c.prec = p->precision;
    c.nu = p->nu;
    c.dt = p->dt;
    c.quick = p->quick;
    c.integrator = p->integrator;
    c.csm_on = p->csm_on;
    c.forcing_on = p->forcing_on;
    c.deadend_on = geom ? ibm_geom_deadend(geom) : 0;
    S->s = p->precision == IBM_FP64 ? 8 : 4;
    const size_t N = (size_t)c.D.N, s = S->s;
    ALLOC(S->nut, N * s);
    ALLOC(S->ustar, 3 * N * s);
    ALLOC(S->Ustar, (size_t)c.NF * s);
    ALLOC(S->b, N * 8);
    ALLOC(S->out4, 8 * 8);
    ALLOC(S->w.r, N * s);
    ALLOC(S->w.pa, N * s);
    ALLOC(S->w.pb, N * s);
    ALLOC(S->w.q, N * s);
    if (p->precision != IBM_FP64) ALLOC(S->w.e, N * 4);
    if (p->solver == IBM_SOLVER_BICGSTAB) {
        ALLOC(S->w.rh, N * s);
        ALLOC(S->w.sv, N * s);
        ALLOC(S->w.tv, N * s);
        ALLOC(S->w.vb, N * s);
    }
    ALLOC(S->w.sc, sizeof(SolveScal));
    size_t nblk = cell_blocks(c.cg);
    const size_t nflat = (size_t)c.fgrid.x * c.fgrid.y * c.fgrid.z;   // >= the 4-cell launches' blocks
    if (nblk < nflat) nblk = nflat;
    if (nblk < 32 * IBM_NSM) nblk = 32 * IBM_NSM;
    ALLOC(c.partials, nblk * 8 * sizeof(double));
    ALLOC(c.counter, 16 * sizeof(unsigned));
    ALLOC(c.fscal, 8 * sizeof(double));
    ALLOC(c.fdelta, 3 * (size_t)(c.n_inc > 0 ? c.n_inc : 1) * sizeof(double));
    cudaError_t e;
    if ((e = cudaMallocHost((void**)&S->w.hsc, sizeof(SolveScal))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&S->hfs, 16 * sizeof(double))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&S->w.ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMemset(c.counter, 0, 16 * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(S->nut, 0, N * s)) != cudaSuccess ||
        (e = cudaMemset(S->w.sc, 0, sizeof(SolveScal))) != cudaSuccess ||
        (e = cudaMemset(c.fscal, 0, 8 * sizeof(double))) != cudaSuccess) {
        free_state(S);
        return ibm_cuda_check(e, "les_create");
    }
    memset(S->hfs, 0, 16 * sizeof(double));
    S->c.nlaunch = &S->nlaunch;
    {
        int rc1 = flux_kernels_setup();
        if (!rc1) rc1 = build_general_list(S->c, 0);
        if (rc1) {
            free_state(S);
            return rc1;
        }
    }
    if (p->integrator == IBM_CRANK_NICOLSON) {
        CNWork* w = (CNWork*)calloc(1, sizeof(CNWork));
        if (!w) {
            free_state(S);
            return ibm_fail(IBM_E_NOMEM, "les_create: host allocation");
        }
        S->c.cn = w;
        w->tol = p->mom_tol > 0.0 ? p->mom_tol : (p->precision == IBM_FP64 ? 1e-10 : 1e-6);
        w->maxit = p->mom_max_iter > 0 ? p->mom_max_iter : 200;
        ALLOC(w->r, 3 * N * s);
        ALLOC(w->rh, 3 * N * s);
        ALLOC(w->p, 3 * N * s);
        ALLOC(w->v, 3 * N * s);
        ALLOC(w->sv, 3 * N * s);
        ALLOC(w->tv, 3 * N * s);
        ALLOC(w->x, 3 * N * s);
        ALLOC(w->sc, sizeof(SolveScal));
        if ((e = cudaMallocHost((void**)&w->hsc, sizeof(SolveScal))) != cudaSuccess ||
            (e = cudaMemset(w->sc, 0, sizeof(SolveScal))) != cudaSuccess ||
            (e = cudaMemset(w->p, 0, 3 * N * s)) != cudaSuccess ||
            (e = cudaMemset(w->v, 0, 3 * N * s)) != cudaSuccess) {
            free_state(S);
            return ibm_cuda_check(e, "les_create: crank-nicolson workspace");
        }
    }
    if (p->precond == 1) {
        // MG holds 64-byte aligned tensor maps
        const size_t mgb = (sizeof(MG) + 63) & ~(size_t)63;
        MG* mg = (MG*)aligned_alloc(64, mgb);
        if (mg) memset(mg, 0, mgb);
        if (!mg) {
            free_state(S);
            return ibm_fail(IBM_E_NOMEM, "les_create: host allocation");
        }
        S->c.mg = mg;
        mg->sweeps = p->mg_sweeps > 0 ? p->mg_sweeps : 2;
        mg->omega = p->mg_omega > 0.0 ? p->mg_omega : 1.6;
        mg->coarse_sweeps = 8;
        mg->allow_fused = p->mg_passes == 0;
        ALLOC(S->w.z, N * s);
        if ((e = cudaStreamCreateWithFlags(&S->w.cap, cudaStreamNonBlocking)) != cudaSuccess) {
            free_state(S);
            return ibm_cuda_check(e, "les_create: capture stream");
        }
        int rc2 = mg_setup(S->c, *mg, (int)s);
        if (!rc2 && (e = cudaDeviceSynchronize()) != cudaSuccess) rc2 = ibm_cuda_check(e, "les_create: multigrid set-up");
        if (rc2) {
            free_state(S);
            return rc2;
        }
    }
    *out = S;
    return IBM_OK;
}

#define NEED(x) \
    if (!(x)) return ibm_fail(IBM_E_INVALID, "%s: null argument (%s)", __func__, #x)

extern "C" int les_attach_guess(les_state* S, ibm_net* net) {
    NEED(S);
    if (net && !S->p_prev) {
        const size_t N = (size_t)S->c.D.N;
        cudaError_t e;
        if ((e = cudaMalloc(&S->p_prev, N * 8)) != cudaSuccess || (e = cudaMalloc(&S->p_keep, N * 8)) != cudaSuccess ||
            (e = cudaMalloc(&S->x_guess, N * 8)) != cudaSuccess || (e = cudaMalloc(&S->two_res, 2 * 8)) != cudaSuccess)
            return ibm_fail(IBM_E_NOMEM, "les_attach_guess: %s", cudaGetErrorString(e));
        S->steps = 0;
    }
    S->net = net;
    return IBM_OK;
}

extern "C" int les_last_rhs(les_state* S, double* d_b, void* stream) {
    NEED(S); NEED(d_b);
    IBM_CUDA(cudaMemcpyAsync(d_b, S->b, (size_t)S->c.D.N * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return IBM_OK;
}

extern "C" int les_init_faces(les_state* S, const void* u, void* U, void* stream) {
    NEED(S); NEED(u); NEED(U);
    return launch_faces(S->c, u, U, (cudaStream_t)stream);
}

extern "C" int les_profile(les_state* S, int32_t on) {
    NEED(S);
    Prof* p = S->c.prof;
    if (!p) {
        S->nlaunch = 0;
        if (!on) return IBM_OK;
        p = (Prof*)calloc(1, sizeof(Prof));
        if (!p) return ibm_fail(IBM_E_NOMEM, "les_profile: host allocation");
        p->cap = 2048;
        for (int q = 0; q < PS_COUNT; ++q) {
            p->ev[q] = (cudaEvent_t*)calloc(2 * p->cap, sizeof(cudaEvent_t));
            for (int e = 0; e < 2 * p->cap; ++e) {
                cudaError_t err = cudaEventCreate(&p->ev[q][e]);
                if (err != cudaSuccess) {
                    p->cap = e / 2;
                    prof_free(p);
                    return ibm_cuda_check(err, "les_profile: cudaEventCreate");
                }
            }
        }
        S->c.prof = p;
    }
    for (int q = 0; q < PS_COUNT; ++q) {
        p->used[q] = 0;
        p->ms[q] = 0.0;
        p->launches[q] = 0;
    }
    p->on = on ? 1 : 0;
    S->nlaunch = 0;
    return IBM_OK;
}

extern "C" int64_t les_kernel_launches(const les_state* S) { return S ? S->nlaunch : -1; }

extern "C" int les_profile_read(les_state* S, double* ms, int64_t* launches) {
    NEED(S); NEED(ms); NEED(launches);
    Prof* p = S->c.prof;
    for (int q = 0; q < PS_COUNT; ++q) {
        ms[q] = 0.0;
        launches[q] = 0;
    }
    if (!p) return IBM_OK;
    for (int q = 0; q < PS_COUNT; ++q) {
        if (p->used[q] > 0) {
            IBM_CUDA(cudaEventSynchronize(p->ev[q][2 * p->used[q] - 1]));
            for (int e = 0; e < p->used[q]; ++e) {
                float t = 0.f;
                IBM_CUDA(cudaEventElapsedTime(&t, p->ev[q][2 * e], p->ev[q][2 * e + 1]));
                p->ms[q] += t;
            }
            p->used[q] = 0;
        }
        ms[q] = p->ms[q];
        launches[q] = p->launches[q];
    }
    return IBM_OK;
}

extern "C" int les_csm(les_state* S, const void* u, void* nut, void* stream) {
    NEED(S); NEED(u); NEED(nut);
    return launch_csm(S->c, u, nut, (cudaStream_t)stream);
}

extern "C" int les_predict(les_state* S, const void* u, const void* U, const void* nut, const void* Hprev, void* H,
                           void* ustar, int32_t first, void* stream) {
    NEED(S); NEED(u); NEED(U); NEED(nut); NEED(H); NEED(ustar);
    if (!first && !Hprev) return ibm_fail(IBM_E_INVALID, "les_predict: Hprev needed after the first step");
    return launch_predict(S->c, u, U, nut, Hprev ? Hprev : H, H, ustar, first ? 1 : 0, (cudaStream_t)stream);
}

extern "C" int les_predict_cn(les_state* S, const void* u, const void* U, const void* nut, void* H, void* ustar,
                              int32_t* iters, void* stream) {
    NEED(S); NEED(u); NEED(U); NEED(nut); NEED(H); NEED(ustar);
    int it = 0;
    int rc = launch_predict_cn(S->c, u, U, nut, H, ustar, &it, (cudaStream_t)stream);
    if (iters) *iters = it;
    return rc;
}

extern "C" int les_forcing(les_state* S, void* ustar, double* fsum, void* stream) {
    NEED(S); NEED(ustar);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_forcing(S->c, ustar, s);
    if (rc) return rc;
    if (fsum) {
        IBM_CUDA(cudaMemcpyAsync(S->hfs, S->c.fscal, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        IBM_CUDA(cudaStreamSynchronize(s));
        memcpy(fsum, S->hfs, 3 * sizeof(double));
    }
    return IBM_OK;
}

extern "C" int les_faces(les_state* S, const void* ustar, void* Ustar, void* stream) {
    NEED(S); NEED(ustar); NEED(Ustar);
    return launch_faces(S->c, ustar, Ustar, (cudaStream_t)stream);
}

extern "C" int les_rhs(les_state* S, const void* Ustar, double* b, void* stream) {
    NEED(S); NEED(Ustar); NEED(b);
    return launch_rhs(S->c, Ustar, b, (cudaStream_t)stream);
}

extern "C" int les_correct(les_state* S, const void* ustar, const void* Ustar, const double* p, void* u, void* U,
                           void* stream) {
    NEED(S); NEED(ustar); NEED(Ustar); NEED(p); NEED(u); NEED(U);
    return launch_correct(S->c, ustar, Ustar, p, u, U, (cudaStream_t)stream);
}

extern "C" int poisson_apply(les_state* S, const double* p, double* Ap, void* stream) {
    NEED(S); NEED(p); NEED(Ap);
    return launch_apply64(S->c, p, Ap, (cudaStream_t)stream);
}

extern "C" int poisson_solve(les_state* S, const double* b, double* p, double tol, int32_t max_it, int32_t solver,
                             les_stats* st, void* stream) {
    NEED(S); NEED(b); NEED(p);
    if (!(tol > 0.0) || max_it < 0 || solver < IBM_SOLVER_CG || solver > IBM_SOLVER_RBSOR)
        return ibm_fail(IBM_E_INVALID, "poisson_solve: bad tol/max_it/solver");
    if (solver == IBM_SOLVER_BICGSTAB && !S->w.rh)
        return ibm_fail(IBM_E_INVALID, "poisson_solve: BiCGStab needs a state created with solver = IBM_SOLVER_BICGSTAB");
    int rc = run_poisson(S->c, S->w, b, p, tol, max_it, solver, S->prm.check_every, S->prm.inner_tol,
                         S->prm.sor_omega, st, (cudaStream_t)stream);
    if (rc == IBM_E_NOCONV) ibm_fail(rc, "poisson_solve: no convergence within %d iterations", max_it);
    if (rc == IBM_E_NONFINITE) ibm_fail(rc, "poisson_solve: residual is not finite");
    return rc;
}

extern "C" int poisson_precond(les_state* S, const void* r, void* z, void* stream) {
    NEED(S); NEED(r); NEED(z);
    if (!S->c.mg) return ibm_fail(IBM_E_INVALID, "poisson_precond: the state has no multigrid preconditioner");
    if ((((uintptr_t)r) | ((uintptr_t)z)) & 15u)
        return ibm_fail(IBM_E_INVALID, "poisson_precond: r and z must be 16-byte aligned");
    if (r == z) return ibm_fail(IBM_E_INVALID, "poisson_precond: r and z must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    launch_reset(S->w.sc, s);
    int rc = S->c.prec == IBM_FP64 ? mg_vcycle<double>(S->c, *S->c.mg, (const double*)r, (double*)z, S->w.sc, s)
                                  : mg_vcycle<float>(S->c, *S->c.mg, (const float*)r, (float*)z, S->w.sc, s);
    if (rc) return rc;
    IBM_CUDA(cudaMemcpyAsync(S->w.hsc, S->w.sc, sizeof(SolveScal), cudaMemcpyDeviceToHost, s));
    IBM_CUDA(cudaStreamSynchronize(s));
    if (S->w.hsc->dev_error) return ibm_fail(IBM_E_CUDA, "poisson_precond: a multigrid shared-memory load timed out");
    return IBM_OK;
}

extern "C" int les_mg_info(const les_state* S, int64_t* out, int32_t n) {
    NEED(S); NEED(out);
    if (n < 2) return ibm_fail(IBM_E_INVALID, "les_mg_info: n must be >= 2");
    for (int q = 0; q < n; ++q) out[q] = 0;
    if (!S->c.mg) return IBM_OK;
    const MG& mg = *S->c.mg;
    out[0] = mg.nlev;
    out[1] = mg.fused;
    for (int l = 0; l < mg.nlev && 2 + l < n; ++l) out[2 + l] = mg.lev[l].M;
    return IBM_OK;
}

extern "C" int les_step(les_state* S, void* u, void* U, double* p, void* H, int32_t first, les_stats* st,
                        void* stream) {
    NEED(S); NEED(u); NEED(U); NEED(p); NEED(H);
    cudaStream_t s = (cudaStream_t)stream;
    const LesCtx& c = S->c;
    int rc;
    if (c.csm_on) {
        prof_begin(c.prof, PS_CSM, s);
        if ((rc = launch_csm(c, u, S->nut, s))) return rc;
        prof_end(c.prof, PS_CSM, s);
    }
    int mom_iters = 0;
    if (c.integrator == IBM_CRANK_NICOLSON) {
        if ((rc = launch_predict_cn(c, u, U, S->nut, H, S->ustar, &mom_iters, s))) return rc;
    } else {
        prof_begin(c.prof, PS_PREDICT, s);
        if ((rc = launch_predict(c, u, U, S->nut, H, H, S->ustar, first ? 1 : 0, s))) return rc;
        prof_end(c.prof, PS_PREDICT, s);
    }
    const bool forcing = c.forcing_on && c.D.flags && c.n_inc > 0;
    if (!forcing) S->hfs[0] = S->hfs[1] = S->hfs[2] = 0.0;
    if (forcing) {
        prof_begin(c.prof, PS_FORCING, s);
        if ((rc = launch_forcing(c, S->ustar, s))) return rc;
        prof_end(c.prof, PS_FORCING, s);
        IBM_CUDA(cudaMemcpyAsync(S->hfs, c.fscal, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    prof_begin(c.prof, PS_FACES, s);
    if ((rc = launch_faces(c, S->ustar, S->Ustar, s))) return rc;
    prof_end(c.prof, PS_FACES, s);
    prof_begin(c.prof, PS_RHS, s);
    if ((rc = launch_rhs(c, S->Ustar, S->b, s))) return rc;
    prof_end(c.prof, PS_RHS, s);
    const int solver = S->prm.solver;
    les_stats ps = {};
    int guess_used = 0;
    double r0 = -1.0, rg = -1.0;
    if (S->net) {
        // learned initial guess: start from it only if its residual is below that of p^n
        const size_t nb = (size_t)c.D.N * 8;
        IBM_CUDA(cudaMemcpyAsync(S->p_keep, p, nb, cudaMemcpyDeviceToDevice, s));
        if (S->steps >= 1) {
            if ((rc = net_guess(S->net, &S->grid, S->b, p, S->p_prev, c.D.flags, S->x_guess, s))) return rc;
            if ((rc = launch_two_residuals(c, S->b, p, S->x_guess, S->two_res, s))) return rc;
            double h[2];
            IBM_CUDA(cudaMemcpyAsync(h, S->two_res, sizeof(h), cudaMemcpyDeviceToHost, s));
            IBM_CUDA(cudaStreamSynchronize(s));
            r0 = h[0];
            rg = h[1];
            if (h[1] < h[0]) {
                IBM_CUDA(cudaMemcpyAsync(p, S->x_guess, nb, cudaMemcpyDeviceToDevice, s));
                guess_used = 1;
            }
        }
    }
    int prc = run_poisson(c, S->w, S->b, p, S->prm.tol, S->prm.max_iter > 0 ? S->prm.max_iter : 100000, solver,
                          S->prm.check_every, S->prm.inner_tol, S->prm.sor_omega, &ps, s);
    if (prc != IBM_OK && prc != IBM_E_NOCONV) return prc;
    prof_begin(c.prof, PS_CORRECT, s);
    if ((rc = launch_correct(c, S->ustar, S->Ustar, p, u, U, s))) return rc;
    prof_end(c.prof, PS_CORRECT, s);
    if (S->net) {
        IBM_CUDA(cudaMemcpyAsync(S->p_prev, S->p_keep, (size_t)c.D.N * 8, cudaMemcpyDeviceToDevice, s));
        S->steps += 1;
    }
    if (st) {
        *st = ps;
        st->guess_used = guess_used;
        st->relres0 = (r0 >= 0.0 && ps.bnorm > 0.0) ? sqrt(r0) / ps.bnorm : -1.0;
        st->relres_guess = (rg >= 0.0 && ps.bnorm > 0.0) ? sqrt(rg) / ps.bnorm : -1.0;
        for (int q = 0; q < 3; ++q) st->fsum[q] = forcing ? S->hfs[q] : 0.0;
        st->mom_iters = mom_iters;
    }
    if (prc == IBM_E_NOCONV) return ibm_fail(prc, "les_step: pressure solve did not converge");
    return IBM_OK;
}

extern "C" int forces(les_state* S, const float* tri, int64_t ntri, const double* p, const void* u, double out[12],
                      void* stream) {
    NEED(S); NEED(p); NEED(out);
    if (ntri < 0 || (ntri > 0 && !tri)) return ibm_fail(IBM_E_INVALID, "forces: bad soup");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_forces(S->c, tri, ntri, p, S->out4, s);
    if (rc) return rc;
    if (u) {
        if ((rc = launch_viscous_force(S->c, u, S->out4 + 4, s))) return rc;
    } else {
        IBM_CUDA(cudaMemsetAsync(S->out4 + 4, 0, 4 * sizeof(double), s));
    }
    IBM_CUDA(cudaMemcpyAsync(S->hfs + 4, S->out4, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    IBM_CUDA(cudaStreamSynchronize(s));
    memcpy(out, S->hfs + 4, 8 * sizeof(double));
    // momentum-forcing estimate of the last step: the forcing added sum(du dx^3) to the fluid in dt
    for (int q = 0; q < 3; ++q) out[8 + q] = -S->hfs[q] / S->c.dt;
    out[11] = 0.0;
    return IBM_OK;
}

// Stable accessors used by the Python binding to size buffers.
extern "C" int64_t les_num_faces(const ibm_grid* g) {
    if (ibm_check_grid(g)) return -1;
    FaceLayout F = make_faces(g->nx, g->ny, g->nz);
    return F.off[2] + (long long)F.dim[2][0] * F.dim[2][1] * F.dim[2][2];
}

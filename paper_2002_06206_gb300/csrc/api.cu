// api.cu -- the C ABI of the library (declared in include/ibmles.h): argument checks, state and
// workspace management, and the composition of one fractional step from the kernels.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
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
    cudaFree(S->w.sc);
    cudaFreeHost(S->w.hsc);
    cudaFreeHost(S->hfs);
    if (S->w.ev) cudaEventDestroy(S->w.ev);
    cudaFree(S->c.partials);
    cudaFree(S->c.counter);
    cudaFree(S->c.fscal);
    cudaFree(S->c.fdelta);
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
    for (int f = 0; f < 6; ++f) c.D.bc[f] = p->bc[f];
    for (int a = 0; a < 3; ++a) c.D.u_in[a] = p->u_in[a];
    if (geom) {
        ibm_geom_device(geom, &c.D.flags, &c.D.cellrec, &c.D.rec, &c.inc, &c.n_rec, &c.n_inc);
    }
    c.F = make_faces(g->nx, g->ny, g->nz);
    c.NF = c.F.off[2] + (long long)c.F.dim[2][0] * c.F.dim[2][1] * c.F.dim[2][2];
    c.cg = cell_grid(g->nx, g->ny, g->nz);
    c.prec = p->precision;
    c.nu = p->nu;
    c.dt = p->dt;
    c.csm_on = p->csm_on;
    c.forcing_on = p->forcing_on;
    c.deadend_on = geom ? ibm_geom_deadend(geom) : 0;
    S->s = p->precision == IBM_FP64 ? 8 : 4;
    const size_t N = (size_t)c.D.N, s = S->s;
    ALLOC(S->nut, N * s);
    ALLOC(S->ustar, 3 * N * s);
    ALLOC(S->Ustar, (size_t)c.NF * s);
    ALLOC(S->b, N * 8);
    ALLOC(S->out4, 4 * 8);
    ALLOC(S->w.r, N * s);
    ALLOC(S->w.pa, N * s);
    ALLOC(S->w.pb, N * s);
    ALLOC(S->w.q, N * s);
    if (p->precision != IBM_FP64) ALLOC(S->w.e, N * 4);
    ALLOC(S->w.sc, sizeof(SolveScal));
    size_t nblk = cell_blocks(c.cg);
    if (nblk < 32 * IBM_NSM) nblk = 32 * IBM_NSM;
    ALLOC(c.partials, nblk * 8 * sizeof(double));
    ALLOC(c.counter, 16 * sizeof(unsigned));
    ALLOC(c.fscal, 8 * sizeof(double));
    ALLOC(c.fdelta, 3 * (size_t)(c.n_inc > 0 ? c.n_inc : 1) * sizeof(double));
    cudaError_t e;
    if ((e = cudaMallocHost((void**)&S->w.hsc, sizeof(SolveScal))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&S->hfs, 8 * sizeof(double))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&S->w.ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMemset(c.counter, 0, 16 * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(S->nut, 0, N * s)) != cudaSuccess ||
        (e = cudaMemset(S->w.sc, 0, sizeof(SolveScal))) != cudaSuccess ||
        (e = cudaMemset(c.fscal, 0, 8 * sizeof(double))) != cudaSuccess) {
        free_state(S);
        return ibm_cuda_check(e, "les_create");
    }
    memset(S->hfs, 0, 8 * sizeof(double));
    S->c.nlaunch = &S->nlaunch;
    *out = S;
    return IBM_OK;
}

#define NEED(x) \
    if (!(x)) return ibm_fail(IBM_E_INVALID, "%s: null argument (%s)", __func__, #x)

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
    if (solver == IBM_SOLVER_BICGSTAB) return ibm_fail(IBM_E_INVALID, "poisson_solve: BiCGStab is not built yet");
    int rc = run_poisson(S->c, S->w, b, p, tol, max_it, solver, S->prm.check_every, S->prm.inner_tol,
                         S->prm.sor_omega, st, (cudaStream_t)stream);
    if (rc == IBM_E_NOCONV) ibm_fail(rc, "poisson_solve: no convergence within %d iterations", max_it);
    if (rc == IBM_E_NONFINITE) ibm_fail(rc, "poisson_solve: residual is not finite");
    return rc;
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
    prof_begin(c.prof, PS_PREDICT, s);
    if ((rc = launch_predict(c, u, U, S->nut, H, H, S->ustar, first ? 1 : 0, s))) return rc;
    prof_end(c.prof, PS_PREDICT, s);
    const bool forcing = c.forcing_on && c.D.flags && c.n_inc > 0;
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
    const int solver = S->prm.solver == IBM_SOLVER_BICGSTAB ? IBM_SOLVER_CG : S->prm.solver;
    les_stats ps = {};
    int prc = run_poisson(c, S->w, S->b, p, S->prm.tol, S->prm.max_iter > 0 ? S->prm.max_iter : 100000, solver,
                          S->prm.check_every, S->prm.inner_tol, S->prm.sor_omega, &ps, s);
    if (prc != IBM_OK && prc != IBM_E_NOCONV) return prc;
    prof_begin(c.prof, PS_CORRECT, s);
    if ((rc = launch_correct(c, S->ustar, S->Ustar, p, u, U, s))) return rc;
    prof_end(c.prof, PS_CORRECT, s);
    if (st) {
        *st = ps;
        for (int q = 0; q < 3; ++q) st->fsum[q] = forcing ? S->hfs[q] : 0.0;
    }
    if (prc == IBM_E_NOCONV) return ibm_fail(prc, "les_step: pressure solve did not converge");
    return IBM_OK;
}

extern "C" int forces(les_state* S, const float* tri, int64_t ntri, const double* p, double out[4], void* stream) {
    NEED(S); NEED(p); NEED(out);
    if (ntri < 0 || (ntri > 0 && !tri)) return ibm_fail(IBM_E_INVALID, "forces: bad soup");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_forces(S->c, tri, ntri, p, S->out4, s);
    if (rc) return rc;
    IBM_CUDA(cudaMemcpyAsync(S->hfs + 4, S->out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    IBM_CUDA(cudaStreamSynchronize(s));
    memcpy(out, S->hfs + 4, 4 * sizeof(double));
    return IBM_OK;
}

// Stable accessors used by the Python binding to size buffers.
extern "C" int64_t les_num_faces(const ibm_grid* g) {
    if (ibm_check_grid(g)) return -1;
    FaceLayout F = make_faces(g->nx, g->ny, g->nz);
    return F.off[2] + (long long)F.dim[2][0] * F.dim[2][1] * F.dim[2][2];
}

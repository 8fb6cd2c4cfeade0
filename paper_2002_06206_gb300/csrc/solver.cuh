// solver.cuh -- the flow solver's internal context and the launchers of its kernels.
#pragma once
#include "common.cuh"

// Scalars the pressure solve keeps on the device (read by the host only at check points).
struct SolveScal {
    double rr, rr_old, pq, target2;     // Krylov: (r,r), previous (r,r), (p,Ap), stop threshold
    double bb, res2, rr32;              // ||b||^2, ||b - A x||^2 in FP64, ||r||^2 of the FP32 copy
    double rho, rho_old, alpha, omega;  // BiCGStab
    double ts, tt, ss, rv;              // BiCGStab inner products
    int done, iters, restart, nonfinite;
    int maxit, pad0, pad1, pad2;
};

// Optional per-kernel timing with CUDA events on the launching stream (les_profile).
enum ProfSlot {
    PS_CSM = 0, PS_PREDICT, PS_FORCING, PS_FACES, PS_RHS, PS_RESIDUAL, PS_CG_SPMV, PS_CG_UPDATE, PS_CORRECT,
    PS_SOR, PS_COUNT
};
struct Prof {
    int on;
    int cap;                       // event pairs per slot before a flush
    cudaEvent_t* ev[PS_COUNT];     // 2 * cap events per slot
    int used[PS_COUNT];
    double ms[PS_COUNT];
    long long launches[PS_COUNT];
};
void prof_begin(Prof* p, int slot, cudaStream_t s);
void prof_end(Prof* p, int slot, cudaStream_t s);

struct LesCtx {
    Dom D;
    FaceLayout F;
    CellGrid cg;
    int prec;                 // IBM_FP64 / IBM_FP32_REFINE64
    double nu, dt;
    int csm_on, forcing_on, deadend_on;
    const int32_t* inc;       // Omega_inc cells
    long long n_inc, n_rec;
    long long NF;
    double* partials;         // grid-reduction partials (cell_blocks * 8 doubles)
    unsigned int* counter;    // grid-reduction arrival counter (zero between kernels)
    double* fscal;            // [8] face-flux / forcing sums
    double* fdelta;           // [3 * n_inc] forcing increments
    Prof* prof;               // null unless profiling
    long long* nlaunch;       // running count of kernel launches (host memory)
};

#define IBM_COUNT(c, n) \
    do { if ((c).nlaunch) *(c).nlaunch += (n); } while (0)

// les.cu
int launch_csm(const LesCtx& c, const void* u, void* nut, cudaStream_t s);
int launch_predict(const LesCtx& c, const void* u, const void* U, const void* nut, const void* Hprev, void* H,
                   void* ustar, int first, cudaStream_t s);
int launch_forcing(const LesCtx& c, void* ustar, cudaStream_t s);   // sums in c.fscal[0..2]
int launch_faces(const LesCtx& c, const void* ustar, void* Ustar, cudaStream_t s);
int launch_rhs(const LesCtx& c, const void* Ustar, double* b, cudaStream_t s);
int launch_correct(const LesCtx& c, const void* ustar, const void* Ustar, const double* p, void* u, void* U,
                   cudaStream_t s);
int launch_forces(const LesCtx& c, const float* tri, long long ntri, const double* p, double* d_out4,
                  cudaStream_t s);

// poisson.cu
struct PoissonWork {
    void* r;        // Krylov vectors of the working precision
    void* pa;
    void* pb;
    void* q;
    void* e;        // FP32 correction (mixed mode)
    void* rh;       // BiCGStab shadow residual
    void* sv;       // BiCGStab s
    void* tv;       // BiCGStab t
    SolveScal* sc;  // device scalars
    SolveScal* hsc; // pinned host copy
    cudaEvent_t ev;
};
int launch_apply64(const LesCtx& c, const double* p, double* Ap, cudaStream_t s);
int run_poisson(const LesCtx& c, PoissonWork& w, const double* b, double* x, double tol, int maxit, int solver,
                int check_every, double inner_tol, double omega, les_stats* st, cudaStream_t s);

// solver.cuh -- the flow solver's internal context and the launchers of its kernels.
#pragma once
#include <cuda.h>

#include "common.cuh"

// Scalars the pressure solve keeps on the device (read by the host only at check points).
struct SolveScal {
    double rr, rr_old, pq, target2;     // Krylov: (r,r), previous (r,r), (p,Ap), stop threshold
    double bb, res2, rr32;              // ||b||^2, ||b - A x||^2 in FP64, ||r||^2 of the FP32 copy
    double rho, rho_old, alpha, omega;  // BiCGStab
    double ts, tt, ss, rv;              // BiCGStab inner products
    double rz, rz_old;                  // preconditioned CG: (r, z) and its previous value
    int done, iters, restart, nonfinite;
    int maxit, dev_error, pad1, pad2;   // dev_error: a bounded device wait gave up (fused multigrid)
    double part[2];                     // partial sums handed from a fast kernel to its general partner
};

// Optional per-kernel timing with CUDA events on the launching stream (les_profile).
enum ProfSlot {
    PS_CSM = 0, PS_PREDICT, PS_FORCING, PS_FACES, PS_RHS, PS_RESIDUAL, PS_CG_SPMV, PS_CG_UPDATE, PS_CORRECT,
    PS_SOR, PS_MG_FINE, PS_MG_TRANSFER, PS_MG_COARSE, PS_MOMENTUM, PS_COUNT
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

// One level of the multigrid preconditioner (mg.cu).  Level 0 is the fine grid (its links are in the
// flags).  A position of level l >= 1 is a block of 2^l x 2^l x 2^l fine cells; its unknowns are the
// connected parts of the block (connected through links inside the block), so an aggregate never
// spans a wall.  Unknowns are numbered by colour (parity of the position), then position, then part;
// the links of unknown u are col/g[rp[u] .. rp[u+1]).
#define IBM_MG_MAXLEV 16
struct MGLev {
    int px, py, pz;      // positions along x, y, z
    long long P;         // positions
    long long M, M0;     // unknowns; the first M0 have colour 0
    long long nnz;       // stored links (each link once from either end)
    int32_t* off;        // [P] first unknown of each position
    int32_t* cnt;        // [P] unknowns (parts) of each position
    int32_t* pos;        // [M] position of each unknown
    int32_t* rp;         // [M + 1] first link of each unknown
    int32_t* col;        // [nnz] neighbour unknown
    float* g;            // [nnz] conductance: sum of the fine conductances between the two aggregates
    float* d;            // [M] Dirichlet (outflow) diagonal term
    float* invdg;        // [M] 1 / (sum of g + d), 0 for an isolated unknown
    int32_t* parent;     // [M] unknown of level l + 1 that contains this one
    int32_t* cp;         // [M + 1] first child (levels >= 2: children are unknowns of level l - 1)
    int32_t* ch;         // [M of level l - 1] children, grouped by parent
    void* b;             // right-hand side (working precision)
    void* x;             // iterate
};
struct MG {
    int nlev;
    int sweeps;          // red-black passes before and after the coarse correction on the fine grid
    int coarse_sweeps;   // symmetric sweeps on the coarsest level
    double omega;        // coarse-correction factor, 0 < omega < 2
    MGLev lev[IBM_MG_MAXLEV];
    // fused fine-grid passes (FP32, two sweeps, nx a multiple of 4, no periodic axis): tensor maps of
    // r, z and the flags for the TMA plane loads, made for the vectors last passed to the V-cycle
    int allow_fused;     // les_params.mg_passes == 0
    int fused;           // 1: the fused kernels apply to this grid and configuration
    int fz_chunk;        // planes per z-chunk of a fused launch (even)
    dim3 fgrid;          // tiles x, tiles y, z-chunks
    void* z2;            // [N] working precision: pre-smoothed and prolongated z, read by the post-smoothing
                         // pass (which writes z): no block reads what another block of the pass writes
    const void* tm_r_ptr;
    CUtensorMap tm_r, tm_z2, tm_f;
};

// Crank-Nicolson predictor workspace: BiCGStab vectors over the stacked three components (3N values
// of the working precision each) and its device-side scalars.
struct CNWork {
    void *r, *rh, *p, *v, *sv, *tv, *x;
    SolveScal* sc;            // device
    SolveScal* hsc;           // pinned host copy
    double tol;
    int maxit;
    int have_x;               // x holds the last converged increment (the next solve starts from it)
};

struct LesCtx {
    Dom D;
    FaceLayout F;
    CellGrid cg;
    dim3 fgrid;               // flat launch (IBM_KU planes per thread)
    dim3 pgrid;               // flat launch, one cell per thread
    dim3 cgrid;               // flat launch over same-colour cell pairs (2 * IBM_KU planes per thread)
    int prec;                 // IBM_FP64 / IBM_FP32_REFINE64
    double nu, dt;
    double quick;             // QUICK fraction of the advected face value (hybrid scheme)
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
    MG* mg;                   // multigrid preconditioner, null for plain CG
    int integrator;           // IBM_ADAMS_BASHFORTH or IBM_CRANK_NICOLSON
    CNWork* cn;               // Crank-Nicolson workspace, null for Adams-Bashforth
    int32_t* general;         // cells the momentum flux evaluates with the general rules
    long long n_general;
    uint8_t* fastmask;        // N bytes: 1 for the cells of the tiled fast path
};
// les.cu: list of the cells that are not fast_cell for the momentum flux (c.general, c.n_general).
int build_general_list(LesCtx& c, cudaStream_t s);
// les.cu: kernel attributes of the tiled momentum-flux kernels (once per process and device).
int flux_kernels_setup();

#define IBM_COUNT(c, n) \
    do { if ((c).nlaunch) *(c).nlaunch += (n); } while (0)

// les.cu
int launch_csm(const LesCtx& c, const void* u, void* nut, cudaStream_t s);
int launch_predict(const LesCtx& c, const void* u, const void* U, const void* nut, const void* Hprev, void* H,
                   void* ustar, int first, cudaStream_t s);
// Crank-Nicolson predictor: H = L(u), ustar = u + delta; *iters = momentum BiCGStab iterations.
int launch_predict_cn(const LesCtx& c, const void* u, const void* U, const void* nut, void* H, void* ustar,
                      int* iters, cudaStream_t s);
int launch_forcing(const LesCtx& c, void* ustar, cudaStream_t s);   // sums in c.fscal[0..2]
int launch_faces(const LesCtx& c, const void* ustar, void* Ustar, cudaStream_t s);
int launch_rhs(const LesCtx& c, const void* Ustar, double* b, cudaStream_t s);
int launch_correct(const LesCtx& c, const void* ustar, const void* Ustar, const double* p, void* u, void* U,
                   cudaStream_t s);
// viscous force on the body from the cut links: d_out4 = {Fx, Fy, Fz, links}
int launch_viscous_force(const LesCtx& c, const void* u, double* d_out4, cudaStream_t s);
int launch_forces(const LesCtx& c, const float* tri, long long ntri, const double* p, double* d_out4,
                  cudaStream_t s);

// stencil4.cu: FP32 fine-grid kernels with 4 cells per thread (nx a multiple of 4)
bool x4_ok(const LesCtx& c);
void launch_cg_dir_spmv_x4(const LesCtx& c, const float* src, const float* pold, float* pnew, float* q, float idx2,
                           SolveScal* sc, int pcg, cudaStream_t s);
void launch_mg_smooth0_x4(const LesCtx& c, const float* r, float* z, float scale, int col, int zero, int fin,
                          SolveScal* sc, cudaStream_t s);

// Builds the levels (allocates them; synchronises the device).  mg.sweeps, omega and coarse_sweeps
// must be set; mg_free releases what mg_setup allocated (also after a failed set-up).
int mg_setup(const LesCtx& c, MG& mg, int precision_bytes);
void mg_free(MG& mg);
template <class T>
int mg_vcycle(const LesCtx& c, const MG& mg, const T* r, T* z, SolveScal* sc, cudaStream_t s);

struct PoissonWork {
    void* z;        // preconditioned residual (MG-PCG)
    void* r;        // Krylov vectors of the working precision
    void* pa;
    void* pb;
    void* q;
    void* e;        // FP32 correction (mixed mode)
    void* rh;       // BiCGStab shadow residual
    void* sv;       // BiCGStab s
    void* tv;       // BiCGStab t
    void* vb;       // BiCGStab second v buffer (v is read at the neighbours while the next is written)
    SolveScal* sc;  // device scalars
    SolveScal* hsc; // pinned host copy
    cudaEvent_t ev;
    // CUDA graph of two preconditioned iterations (both ping-pong parities), replayed while the
    // per-kernel profiler is off; captured on `cap` for the solution vector `gkey` in precision `gprec`
    cudaStream_t cap;
    cudaGraphExec_t gexec;
    const void* gkey;
    int gprec;
    long long glaunches;
};
int launch_apply64(const LesCtx& c, const double* p, double* Ap, cudaStream_t s);
void launch_reset(SolveScal* sc, cudaStream_t s);   // clears the solve's device flags
int launch_two_residuals(const LesCtx& c, const double* b, const double* xa, const double* xb, double* out,
                         cudaStream_t s);
// learn.cu
int net_guess(ibm_net* n, const ibm_grid* g, const double* b, const double* p, const double* pprev,
              const uint8_t* flags, double* xg, cudaStream_t s);
int run_poisson(const LesCtx& c, PoissonWork& w, const double* b, double* x, double tol, int maxit, int solver,
                int check_every, double inner_tol, double omega, les_stats* st, cudaStream_t s);

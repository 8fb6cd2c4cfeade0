/* ibmles.h -- C ABI of the GB300 (sm_103a) topology-free immersed-boundary LES library.
 *
 * The library implements one fractional time step of the immersed-boundary LES of Onishi & Tsubokura
 * (arXiv 2002.06206) on a uniform Cartesian grid, plus the per-geometry fluid/solid classification of
 * a raw triangle soup, as hand-written CUDA kernels.  Every pointer named d_* is a device pointer
 * owned by the caller; `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * All calls are asynchronous on `stream` unless their comment names a host synchronisation.
 *
 * Layout conventions (shared by every call):
 *   grid      nx*ny*nz cells of size dx; cell (i,j,k) has index c = i + nx*(j + ny*k) and its centre
 *             at ((i+1/2)dx, (j+1/2)dx, (k+1/2)dx).  At most 2^31/3 cells.
 *   cell      fields are component-major: u[comp*N + c] (comp 0,1,2 = x,y,z).
 *   face      fields are one concatenated vector Ux | Uy | Uz of length
 *             NF = (nx+1)ny nz + nx(ny+1)nz + nx ny(nz+1); Ux index i + (nx+1)(j + ny k) is the face at
 *             x = i dx, Uy index i + nx(j + (ny+1)k), Uz index i + nx(j + ny k).
 *   soup      float32 [ntri][3][3] vertex coordinates in grid units (position / dx), no connectivity.
 *   flags     one byte per cell: bits 0-5 = cut link towards -x,+x,-y,+y,-z,+z; bit 6 = Omega_inc
 *             (the cell has a cut link); bit 7 = Omega_adj (not Omega_inc, next to an Omega_inc cell).
 *   face id   a cut face between cell c and c + e_a has id a*N + c.
 *   precision IBM_FP64: cell/face fields and H are double.  IBM_FP32_REFINE64: they are float; the
 *             pressure p and the right-hand side b are double in both modes.
 *
 * Errors: every int-returning call returns an ibm_status; ibm_last_error() describes the last
 * failure of the calling thread.  No call aborts or traps on bad input.
 */
#ifndef IBMLES_H
#define IBMLES_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IBM_OK = 0,
    IBM_E_INVALID = 1,    /* bad argument (null pointer, size, mode, unsupported grid) */
    IBM_E_NOMEM = 2,      /* device allocation failed */
    IBM_E_CUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    IBM_E_NOCONV = 4,     /* the pressure solve hit max_iter; the best iterate is left in p */
    IBM_E_NONFINITE = 5,  /* a residual norm became NaN or Inf */
    IBM_E_CAPACITY = 6    /* the cut-face buffer is too small; *n_cut holds the required size */
} ibm_status;

enum { IBM_BC_PERIODIC = 0, IBM_BC_INFLOW = 1, IBM_BC_OUTFLOW = 2, IBM_BC_SLIP = 3, IBM_BC_NOSLIP = 4 };
enum { IBM_FP64 = 0, IBM_FP32_REFINE64 = 1 };
enum { IBM_SOLVER_CG = 0, IBM_SOLVER_BICGSTAB = 1, IBM_SOLVER_RBSOR = 2 };
enum { IBM_ADAMS_BASHFORTH = 0, IBM_CRANK_NICOLSON = 1 };

typedef struct { int32_t nx, ny, nz, reserved; double dx; } ibm_grid;

typedef struct {
    double eps_edge;     /* edge tolerance of the ray/triangle predicate, relative to |W| (1e-9) */
    double eps_det;      /* determinant threshold: |W| <= eps_det is "parallel" (0) */
    int32_t deadend_on;  /* dead-end filter of the IB forcing (Sec. 3.4, Eq. deadend_filter) */
    int32_t reserved;
} ibm_geom_params;

typedef struct {
    double nu;           /* kinematic viscosity (1/Re in non-dimensional units) */
    double dt;           /* time step */
    double u_in[3];      /* inflow velocity (Dirichlet faces of type IBM_BC_INFLOW) */
    int32_t bc[6];       /* domain-face types, order x-, x+, y-, y+, z-, z+ (periodic must pair) */
    int32_t csm_on;      /* coherent-structure eddy viscosity (Sec. 2.3) */
    int32_t forcing_on;  /* distributed direct forcing (Sec. 2.1/2.4.2) */
    int32_t precision;   /* IBM_FP64 or IBM_FP32_REFINE64 */
    int32_t solver;      /* IBM_SOLVER_* for the pressure Poisson equation */
    double tol;          /* stop at ||b - A p||_2 <= tol ||b||_2 */
    int32_t max_iter;    /* cap on Krylov (or SOR) iterations per solve, summed over refinements */
    int32_t check_every; /* iterations between host reads of the residual (0 = 16) */
    double inner_tol;    /* FP32 inner solve: relative reduction per FP64 refinement (0 = 1e-4) */
    double sor_omega;    /* over-relaxation factor of red-black SOR (0 = 1.9) */
    int32_t precond;     /* CG preconditioner: 0 none, 1 geometric multigrid V-cycle */
    int32_t mg_sweeps;   /* red-black Gauss-Seidel sweeps on the fine grid before and after the coarse
                            correction (0 = 2); the coarse levels take one sweep each way */
    double mg_omega;     /* multigrid coarse-correction factor in (0, 2) (0 = 1.6) */
    double quick;        /* fraction of QUICK in the advected face value, [0, 1] (Sec. 3.1/3.3: 0.05-0.1) */
    int32_t integrator;  /* IBM_ADAMS_BASHFORTH (explicit, Euler first step) or IBM_CRANK_NICOLSON
                            (Eq. crank-nicolson, implicit momentum solve by BiCGStab) */
    int32_t mom_max_iter;/* Crank-Nicolson: BiCGStab iteration cap per step (0 = 200) */
    double mom_tol;      /* Crank-Nicolson: stop at ||r|| <= mom_tol ||dt L(u^n)|| (0 = 1e-6 in
                            FP32_REFINE64 mode, 1e-10 in FP64 mode) */
    int32_t mg_passes;   /* multigrid fine-grid passes: 0 = fused where the grid allows (FP32, mg_sweeps 2,
                            nx a multiple of 16, no periodic axis, a body present: the four half-sweeps
                            before the coarse correction and the restriction in one pass, the four after
                            it and (r, z) in another), 1 = one kernel per half-sweep.  Same V-cycle. */
    int32_t reserved;
} les_params;

typedef struct {
    int32_t iters;       /* inner iterations of the last pressure solve */
    int32_t outer;       /* FP64 refinement passes of the last pressure solve */
    int32_t status;      /* ibm_status of the solve */
    int32_t guess_used;  /* 1 if the solve started from the learned guess */
    double relres;       /* ||b - A p|| / ||b|| at exit, computed in FP64 */
    double bnorm;        /* ||b||_2 */
    double fsum[3];      /* momentum added by the IB forcing this step: sum of du * dx^3 */
    double relres0;      /* with a learned guess attached: initial ||b - A p^n|| / ||b|| (else -1), in FP32 */
    double relres_guess; /* with a learned guess attached: the same for the guess (else -1), in FP32 */
    int32_t mom_iters;   /* Crank-Nicolson: momentum BiCGStab iterations of the step (0 for AB2) */
    int32_t reserved;
} les_stats;

typedef struct ibm_geom ibm_geom;
typedef struct les_state les_state;
typedef struct ibm_net ibm_net;

/* ---------------------------------------------------------------------------------------------- */
/* Geometry: classification (Sec. 2.4.1: ray tracing from the cell centres along the grid lines,    */
/* Moller-Trumbore with a determinant tolerance).                                                   */

/* Device workspace ibm_classify needs for this grid and soup size (bytes). */
size_t ibm_classify_workspace_bytes(const ibm_grid* grid, int64_t ntri);

/* For each axis a and each grid line through cell centres parallel to a, decide with an exactly
 * specified FP64 predicate which triangles of d_tri cross it; a crossing at x_hit belongs to the
 * interior face f = floor(x_hit/dx - 1/2) at position t = x_hit/dx - 1/2 - f in [0,1) along the
 * centre-to-centre segment.  Writes d_flags bits 0-5 (bits 6-7 cleared) and the cut-face list sorted
 * by face id with t_lo = min t, t_hi = max t per face.  d_flags[N], d_face_id/d_t_lo/d_t_hi[cap].
 * Host synchronisation: reads the cut count back; *n_cut (host) = number of cut faces.  Returns
 * IBM_E_CAPACITY if *n_cut > cap (then only the first cap entries are written; call again with a
 * buffer of *n_cut).  Triangles with non-finite vertices are skipped.  d_workspace must hold ibm_classify_workspace_bytes() bytes.
 * *n_tests (host, may be NULL) = number of (triangle, grid line) predicate evaluations. */
int ibm_classify(const ibm_grid* grid, const float* d_tri, int64_t ntri, const ibm_geom_params* gp,
                 uint8_t* d_flags, int64_t* d_face_id, double* d_t_lo, double* d_t_hi, int64_t cap,
                 int64_t* n_cut, int64_t* n_tests, void* d_workspace, size_t ws_bytes, void* stream);

/* ibm_classify without any device allocation, for callers that cannot call cudaMalloc -- for
 * example code that runs under a host framework owning every device allocation through its own
 * pool, or code that must not trigger the implicit device synchronisation an allocation can cause.
 * The paper has no counterpart: this is a packaging variant of ibm_classify (same arguments and
 * results, no d_workspace).  Its scratch is a fixed 32 MiB device array inside the library, held by
 * every GPU that loads the library until the process exits; grids and soups whose
 * ibm_classify_workspace_bytes() exceed it are rejected with IBM_E_INVALID before any device work.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and keeps it for the life of the process; make that first call before any
 * stream capture.  cudaDeviceReset destroys the device's context and with it that address: after a
 * reset this entry point must not be called again in the same process.  All calls share the one
 * array: calls that overlap on the GPU (other streams or threads, same device) race and must be
 * serialised by the caller.  Each call re-initialises what it needs, so earlier contents do not
 * matter. */
int ibm_classify_noalloc(const ibm_grid* grid, const float* d_tri, int64_t ntri, const ibm_geom_params* gp,
                         uint8_t* d_flags, int64_t* d_face_id, double* d_t_lo, double* d_t_hi, int64_t cap,
                         int64_t* n_cut, int64_t* n_tests, void* stream);

/* Setup (Sec. 2.4.1 Eq. dummy_cell_region, Sec. 2.4.2 Eq. q_axis and Eq. distribution_function):
 * sets flags bits 6-7 in place and builds two link records per cut face (one per side) with the
 * ghost branch, its coefficients and the forcing weights.  The returned geometry owns its device
 * memory; d_flags must stay alive and unchanged while the geometry is used. */
int ibm_setup(const ibm_grid* grid, const ibm_geom_params* gp, uint8_t* d_flags,
              const int64_t* d_face_id, const double* d_t_lo, const double* d_t_hi, int64_t n_cut,
              ibm_geom** out, void* stream);
int ibm_geom_info(const ibm_geom* geom, int64_t* n_rec, int64_t* n_inc);
/* Copy the records out: d_idx[n_rec][6] = cell, far, opp, axis, side, branch; d_coef[n_rec][6] =
 * d/dx, c_ib, c_p, c_o, w_fluid, w_ghost; d_cellrec[N] = first record of each cell or -1. */
int ibm_geom_export(const ibm_geom* geom, int64_t* d_idx, double* d_coef, int64_t* d_cellrec,
                    void* stream);
/* Wall velocity u_IB (Eq. forcing_term) per record, d_uib[n_rec][3] in FP64 in record order, copied
 * on `stream`; NULL resets it to zero.  It enters the ghost values of Eq. q_axis, the forcing target,
 * and the flux of each cut face: the mean of u_IB.e_a over the face's two records.  A nonzero value
 * therefore lets fluid cross the wall at the wall's own velocity, as in the prescribed-velocity
 * Taylor-Green verification of Sec. 2.5.  The cut faces of a sealed pocket must then carry zero net
 * flux, or its Poisson block has no solution and the solve ends with IBM_E_NOCONV. */
int ibm_set_boundary_velocity(ibm_geom* geom, const double* d_uib, void* stream);
void ibm_geom_destroy(ibm_geom* geom);

/* ---------------------------------------------------------------------------------------------- */
/* Flow solver.  les_create allocates every workspace once; no later call allocates. `geom` may be  */
/* NULL (no immersed body); it must outlive the state.                                             */

int les_create(const ibm_grid* grid, const les_params* params, const ibm_geom* geom, les_state** out);
void les_destroy(les_state* st);

/* Face velocity from a cell field with the face rule of les_faces (no mass correction skipped). */
int les_init_faces(les_state* st, const void* d_u, void* d_U, void* stream);

/* One fractional step (Sec. 2.1; Adams-Bashforth 2 or Crank-Nicolson per params.integrator): CSM eddy
 * viscosity, predictor, IB forcing,
 * face velocities, RHS, pressure solve, correction.  In/out: d_u[3N], d_U[NF], d_p[N] (double; x0
 * of the solve), d_H[3N] (holds H^{n-1} on entry and H^n on exit).  first_step != 0 takes an Euler
 * step.  Host synchronisation: the pressure solve reads its residual every check_every iterations.
 * `stats` (host, may be NULL) receives the solve's figures. */
int les_step(les_state* st, void* d_u, void* d_U, double* d_p, void* d_H, int32_t first_step,
             les_stats* stats, void* stream);

/* The step's operators, exposed one by one (les_step calls exactly these). */
/* Eq. Smagorinsky/Q/FCS: nu_t per cell from central velocity gradients (ghost values on cut links). */
int les_csm(les_state* st, const void* d_u, void* d_nut, void* stream);
/* Adams-Bashforth predictor: H = L(u) = -div(U u) + div((nu + nu_t) grad u) + div(nu_t grad u^T);
 * u* = u + dt(3/2 H - 1/2 Hprev) (u + dt H on the first step). */
int les_predict(les_state* st, const void* d_u, const void* d_U, const void* d_nut,
                const void* d_Hprev, void* d_H, void* d_ustar, int32_t first_step, void* stream);
/* Crank-Nicolson predictor (Eq. crank-nicolson) with U = U^n and nu_t = nu_t(u^n) in both halves:
 * delta = u* - u solves delta - (dt/2) L_0(delta) = dt L(u), L_0 the linear part of L (ghost values
 * without wall and inflow velocities), by BiCGStab over the stacked three components, starting from the
 * increment of the previous converged call on this state (from 0 on the first call or after a failure).
 * d_H[3N] receives L(u), d_ustar[3N] the predicted field; *iters (host, may be NULL) the iterations.
 * Needs a state created with integrator = IBM_CRANK_NICOLSON.  Synchronises every 4 iterations.
 * Returns IBM_E_NOCONV at mom_max_iter (d_ustar then holds the last iterate), IBM_E_NONFINITE. */
int les_predict_cn(les_state* st, const void* d_u, const void* d_U, const void* d_nut, void* d_H, void* d_ustar,
                   int32_t* iters, void* stream);
/* Eq. forcing_term + Eq. discrete_forcing_term: in-place forcing of d_ustar; fsum (host, may be
 * NULL, synchronises) = momentum added, sum of du * dx^3. */
int les_forcing(les_state* st, void* d_ustar, double* fsum, void* stream);
/* Face velocities U* of the intermediate field: the mean of the two cells on uncut interior faces, the
 * wall's normal velocity on cut faces (see ibm_set_boundary_velocity; 0 for a stationary body), the
 * boundary value on domain faces, outflow faces shifted to zero net boundary flux. */
int les_faces(les_state* st, const void* d_ustar, void* d_Ustar, void* stream);
/* Eq. poisson right-hand side b = div(U*)/dt (double). */
int les_rhs(les_state* st, const void* d_Ustar, double* d_b, void* stream);
/* Eq. correction: cell velocity from the central pressure gradient, face velocity from the compact one
 * on uncut interior faces; cut faces and wall/inflow faces keep their U* value. */
int les_correct(les_state* st, const void* d_ustar, const void* d_Ustar, const double* d_p,
                void* d_u, void* d_U, void* stream);

/* Eq. poisson operator in FP64: (A p)_c = sum over uncut links of (p_n - p_c)/dx^2, outflow faces
 * p = 0, cut links, walls and inflow faces Neumann. */
int poisson_apply(les_state* st, const double* d_p, double* d_Ap, void* stream);
/* Solve A p = b to ||b - A p|| <= tol ||b|| with x0 = d_p (in/out).  solver = IBM_SOLVER_*; in
 * FP32_REFINE64 mode the Krylov iterations run in FP32 inside FP64 iterative refinement.
 * Host synchronisation as les_step.  Returns IBM_E_NOCONV after max_it iterations. */
int poisson_solve(les_state* st, const double* d_b, double* d_p, double tol, int32_t max_it,
                  int32_t solver, les_stats* stats, void* stream);

/* The multigrid preconditioner of the pressure solve (not in the paper, whose solvers are BiCGStab and
 * red-black SOR): d_z[N] = one V-cycle applied to d_r[N], in the state's working precision (float in
 * FP32_REFINE64 mode, double in FP64 mode), for the unscaled system  sum_links g (z_N - z_P) - d z_P =
 * dx^2 r  whose operator is dx^2 times the Eq. poisson operator.  Both arrays are 16-byte aligned and
 * distinct.  Needs a state created with precond = 1.  Synchronises (reads a device error word). */
int poisson_precond(les_state* st, const void* d_r, void* d_z, void* stream);
/* Multigrid hierarchy of a state (host, no synchronisation): out[0] = levels (0 without multigrid),
 * out[1] = 1 when the fused fine-grid passes are used, out[2 + l] = unknowns of level l (level 0 =
 * cells), for the first n - 2 levels.  n >= 2. */
int les_mg_info(const les_state* st, int64_t* out, int32_t n);

/* Forces on the body (Sec. 3.2-3.3), out (host) = 12 doubles; synchronises.
 *  out[0..2]  Eq. force: Shepard inverse-distance pressure on the front/back of every triangle,
 *             F = sum_tri area (p_back - p_front) n;  out[3] = triangles used (both sides found);
 *  out[4..6]  viscous force (reading; the paper integrates pressure): the molecular diffusive flux
 *             nu (u_P - u_G) dx through every cut link, u_G the Eq. q_axis ghost value;
 *             out[7] = links used (0 when d_u is NULL);
 *  out[8..10] momentum-forcing estimate of the last les_step: -(sum of the forcing's du dx^3) / dt;
 *  out[11]    0.
 * d_u (may be NULL) is the cell velocity in the working precision. */
int forces(les_state* st, const float* d_tri, int64_t ntri, const double* d_p, const void* d_u, double out[12],
           void* stream);

/* Per-kernel timing with CUDA events recorded on the launching stream around each kernel group of
 * les_step / poisson_solve.  les_profile(st, 1) enables and resets the counters, (st, 0) disables.
 * les_profile_read (synchronises) fills ms[14] (total milliseconds) and launches[14] per group, in
 * the order: csm, predict, forcing, faces, rhs, residual, cg_dir_spmv, cg_update, correct, sor,
 * mg_fine (fine-grid smoothing passes), mg_transfer (fine-grid restriction and prolongation),
 * mg_coarse (everything on the coarse levels, one group per V-cycle), momentum (the Crank-Nicolson
 * BiCGStab after its first operator evaluation, which counts as predict). */
int les_profile(les_state* st, int32_t on);
int les_profile_read(les_state* st, double* ms, int64_t* launches);
/* Kernels this state launched since les_create or the last les_profile(st, 1) (host counter). */
int64_t les_kernel_launches(const les_state* st);

/* ---------------------------------------------------------------------------------------------- */
/* Surface pressure per triangle side (Eq. force) with the thin-plate filter of Eq. force_filter    */
/* (Sec. 3.3), which the paper prints garbled.  Reading: a cell centre x of the 2x2x2 block around  */
/* the centroid X of a triangle takes part in the Shepard average of X's side only if the open      */
/* segment X-x crosses no other triangle of the soup, so points behind a second surface closer than  */
/* a cell (the inner faces of a plate thinner than dx, a duplicated skin) are cancelled.  Cp follows */
/* as (p_side - p_ref) / (U0^2 / 2).                                                                */
typedef struct ibm_surface ibm_surface;
/* Bins the triangles (float32 [ntri][3][3], grid units, device; the caller keeps d_tri alive and
 * unchanged while the object lives) into 2x2x2-cell bins.  Allocates; synchronises `stream`. */
int ibm_surface_create(const ibm_grid* grid, const float* d_tri, int64_t ntri, void* stream, ibm_surface** out);
void ibm_surface_destroy(ibm_surface* surf);
/* Number of (bin, triangle) entries of the binning (for sizing and tests), -1 for NULL. */
int64_t ibm_surface_bin_entries(const ibm_surface* surf);
/* d_pside[2 ntri] (device, double) = front (n.(x - X) > 0) and back Shepard pressure of every
 * triangle, NaN where a side has no point (degenerate or non-finite triangles: both NaN).  zfilter
 * != 0 applies the filter.  h_out4 (host, may be NULL; synchronises) = sum over the sides that have
 * a value of -area p n (front) or +area p n (back), and the number of such sides.  No allocation. */
int ibm_surface_pressure(ibm_surface* surf, const double* d_p, int32_t zfilter, double* d_pside, double* h_out4,
                         void* stream);

/* ---------------------------------------------------------------------------------------------- */
/* Learned initial guess of the pressure solve.  Not in the paper: a small 3-D convolutional network  */
/* (3x3x3 kernels, 8 -> 8 -> 8 -> 1 channels, ReLU) that maps, per cell, the right-hand side b dx^2,  */
/* the last pressure change p^n - p^{n-1} (both divided by s = RMS of p^n - p^{n-1}) and the solid    */
/* mask (cells with a cut link) to the deviation of p^{n+1} from the linear extrapolation,           */
/* (p^{n+1} - 2 p^n + p^{n-1}) / s.  BF16 weights and activations, FP32 accumulation on the tensor  */
/* cores; a zero network leaves the extrapolation.  Parameters: W1[8][27][8], W2[8][27][8], W3[1][27][8], b1[8],    */
/* b2[8], b3[1] (ibm_net_num_params() floats), tap = 9 (dz+1) + 3 (dy+1) + (dx+1).                    */

int ibm_net_num_params(void);
/* h_params (host, may be NULL for zeros): initial parameters. */
int ibm_net_create(const float* h_params, ibm_net** out);
void ibm_net_destroy(ibm_net* net);
int ibm_net_get_params(const ibm_net* net, float* h_params);
/* Gradients of the last ibm_net_train_step (mean squared error), same layout as the parameters. */
int ibm_net_get_grads(const ibm_net* net, float* h_grads);
/* d_out[N] (float) = network output for the snapshot (b, p, p_prev, flags); *scale (host, may be NULL,
 * synchronises) = s.  d_flags may be NULL (no body). */
int ibm_net_forward(ibm_net* net, const ibm_grid* grid, const double* d_b, const double* d_p,
                    const double* d_pprev, const uint8_t* d_flags, float* d_out, double* scale, void* stream);
/* The training target of a snapshot: d_target[N] (float) = (p^{n+1} - 2 p^n + p^{n-1}) / s, formed in
 * FP64 on the device; s > 0 is the scale ibm_net_forward returned for (b, p^n, p^{n-1}).  All arrays are
 * device arrays of N = nx ny nz values owned by the caller.  IBM_E_INVALID on a null array or s <= 0. */
int ibm_net_target(const ibm_grid* grid, const double* d_pnext, const double* d_p, const double* d_pprev,
                   double s, float* d_target, void* stream);
/* One Adam step (betas 0.9, 0.999) on the mean squared error against
 * d_target[N] = (p^{n+1} - 2 p^n + p^{n-1}) / s (ibm_net_target);
 * lr = 0 only computes the gradients.  *loss (host, synchronises) = the loss before the update. */
int ibm_net_train_step(ibm_net* net, const ibm_grid* grid, const double* d_b, const double* d_p,
                       const double* d_pprev, const uint8_t* d_flags, const float* d_target, float lr,
                       double* loss, void* stream);
/* Attach (or detach with NULL) a network to a solver state: from the second step on, each les_step
 * starts the pressure solve from 2 p^n - p^{n-1} + s net(...) when that iterate has the smaller
 * residual, else from p^n.  The state keeps p^{n-1}.  The network must stay alive while attached. */
int les_attach_guess(les_state* st, ibm_net* net);
/* Copy the right-hand side b of the last les_step / les_rhs into d_b[N]. */
int les_last_rhs(les_state* st, double* d_b, void* stream);

/* Measured fused multiply-add rate of the current GPU in TFLOP/s (2 flops per FMA), FP64
 * (precision = IBM_FP64) or FP32 (IBM_FP32_REFINE64): independent FMA chains on every SM, best of three
 * launches timed with CUDA events on `stream`.  Not in the paper: the arithmetic roof beside the HBM
 * roof in performance reports.  Allocates 16 bytes (stream-ordered); synchronises. */
int ibm_probe_fma_rate(int32_t precision, double* tflops, void* stream);

/* Number of faces NF of the concatenated face vector for this grid (-1 for an invalid grid). */
int64_t les_num_faces(const ibm_grid* grid);

const char* ibm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif

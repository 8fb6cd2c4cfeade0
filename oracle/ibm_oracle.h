/* ibm_oracle.h -- plain FP64 CPU oracle of the topology-free immersed-boundary LES step.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct definition that the CUDA library is
 * checked against.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it; the product path never does.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * Grid: nx*ny*nz cells of size dx; cell (i,j,k) has index i + nx*(j + ny*k) and centre
 * ((i+1/2)dx, (j+1/2)dx, (k+1/2)dx).  Cell fields are component-major: u[comp*N + cell].
 * Face fields are concatenated Ux | Uy | Uz with Ux[(nx+1)*ny*nz] (index i + (nx+1)*(j + ny*k),
 * face at x = i*dx), Uy[nx*(ny+1)*nz], Uz[nx*ny*(nz+1)].
 * Triangle soups are float32 [ntri][3 vertices][xyz] in grid units (dx = 1 in the soup).
 *
 * Readings and their pins: where the paper is silent the oracle states a reading, and each one has
 * a check beyond the oracle's own definition.  The dead-end filter (or_forcing) is pinned to the
 * printed threshold; the placement of the forcing (or_forcing) by its d = 0 limit and by the
 * Taylor-Green convergence of Sec. 2.5; the transpose SGS term on cut faces (or_predict,
 * or_momentum_operator) by the vanishing stress divergence of a linear field at a wall (any choice
 * exact for linear fields would pass); the inflow, slip and no-slip velocity ghosts by their
 * exactness for linear fields; the zero-gradient outflow velocity ghost by an x-invariant field,
 * whose operator next to the outflow face equals the interior one (the inflow, slip and no-slip
 * ghosts fail that check); the pressure part of the outer boundaries by a manufactured solution at
 * second order.
 */
#ifndef IBM_ORACLE_H
#define IBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { int32_t nx, ny, nz, pad_; double dx; } or_grid;

enum { OR_BC_PERIODIC = 0, OR_BC_INFLOW = 1, OR_BC_OUTFLOW = 2, OR_BC_SLIP = 3, OR_BC_NOSLIP = 4 };
enum { OR_SOLVER_BICGSTAB = 0, OR_SOLVER_CG = 1, OR_SOLVER_RBSOR = 2 };
enum { OR_ADAMS_BASHFORTH = 0, OR_CRANK_NICOLSON = 1 };

typedef struct {
    double nu;            /* kinematic viscosity (1/Re in the paper's non-dimensional form) */
    double dt;            /* time step */
    double u_in[3];       /* inflow velocity (Dirichlet) */
    int32_t bc[6];        /* domain-face types, order x-, x+, y-, y+, z-, z+ */
    int32_t csm_on;       /* coherent-structure model on (Sec. 2.3) */
    int32_t forcing_on;   /* distributed forcing on (Eq. discrete_forcing_term) */
    int32_t deadend_on;   /* dead-end filter B (Eq. deadend_filter) */
    int32_t integrator;   /* OR_ADAMS_BASHFORTH (AB2, Euler first step) or OR_CRANK_NICOLSON */
    double quick;         /* weight of the QUICK face value in the advective flux (hybrid scheme), 0..1 */
    double mom_tol;       /* Crank-Nicolson: relative residual of the momentum solve */
    int32_t mom_maxit;    /* Crank-Nicolson: BiCGStab iteration cap */
    int32_t pad_;
} or_params;

/* One link record: the cut link of cell `cell` in direction side*e_axis (Sec. 2.4.1, Eq. q_axis). */
typedef struct {
    int64_t cell;    /* P: the cell that reads across the cut link */
    int64_t far;     /* G = P + side*e_axis: the cell on the other side of the wall */
    int64_t opp;     /* O = P - side*e_axis for branch B, else -1 */
    int64_t axis;    /* 0, 1, 2 */
    int64_t side;    /* -1 or +1 */
    int64_t branch;  /* 0 = A (d >= 1/2), 1 = B (d < 1/2, O usable), 2 = C (d < 1/2, O unusable) */
    double d;        /* wall distance from P's centre along the link, in units of dx */
    double c_ib, c_p, c_o;   /* ghost = c_ib*q_IB + c_p*q_P + c_o*q_O */
    double w_fluid, w_ghost;    /* Eq. distribution_function at d: fluid branch, ghost branch */
    double uib[3];           /* wall velocity at the intersection (0 for stationary bodies) */
} or_record;

typedef struct {
    int32_t iters;       /* Krylov / SOR iterations of the pressure solve */
    int32_t status;      /* 0 converged, 4 not converged */
    double relres;       /* ||b - A p|| / ||b|| at exit */
    double bnorm;        /* ||b|| */
    double fsum[3];      /* momentum added by the IB forcing this step, sum over cells of du * dx^3 */
    int32_t mom_iters;   /* Crank-Nicolson momentum BiCGStab iterations (0 for AB2) */
    int32_t pad_;
} or_stats;

/* Classification (Sec. 2.4.1): exact axis-aligned ray/triangle predicate.  Writes flags bits 0-5 and
 * the cut-face list sorted by face id (axis*N + lower cell).  Returns the number of cut faces (only
 * the first `cap` are written), or -1 on allocation failure.  *n_skipped counts non-finite triangles. */
int64_t or_classify(const or_grid* g, const float* tri, int64_t ntri, double eps_edge, double eps_det,
                    uint8_t* flags, int64_t* face_id, double* t_lo, double* t_hi, int64_t cap,
                    int64_t* n_skipped, int64_t* n_tests);

/* Literal Moller-Trumbore cross-check: number of (triangle, grid line) pairs on which MT and the
 * exact predicate disagree about a hit, or whose hit positions differ by more than 1e-9. */
int64_t or_mt_disagreements(const or_grid* g, const float* tri, int64_t ntri, double eps_edge,
                            double eps_det);

/* Setup (Sec. 2.4.1-2.4.2): Omega_inc (bit 6), Omega_adj (bit 7), two link records per cut face,
 * cellrec[P] = first record of cell P (-1 if none), inc_list = Omega_inc cells in index order.
 * Returns the number of records (2*n_cut) or -1 if a cut face is missing from the list. */
int64_t or_setup(const or_grid* g, uint8_t* flags, const int64_t* face_id, const double* t_lo,
                 const double* t_hi, int64_t n_cut, or_record* rec, int64_t* cellrec,
                 int64_t* inc_list, int64_t* n_inc);

/* Ghost value of velocity component `comp` read by cell P across link (axis, side). */
double or_velocity_across(const or_grid* g, const or_params* pr, const uint8_t* flags,
                          const or_record* rec, const int64_t* cellrec, const double* u,
                          int comp, int64_t P, int axis, int side);

void or_csm(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
            const int64_t* cellrec, const double* u, double* nut);
void or_predict(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                const int64_t* cellrec, const double* u, const double* U, const double* nut,
                const double* Hprev, double* H, double* ustar, int first_step);
/* L(u) per cell (advection + diffusion + SGS stress divergence per unit volume), U and nu_t fixed;
 * hom != 0 drops the wall and inflow velocities from the ghost values (the linear part of L). */
void or_momentum_operator(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                          const int64_t* cellrec, const double* u, const double* U, const double* nut,
                          int hom, double* L);
/* Crank-Nicolson predictor (Eq. crank-nicolson); returns BiCGStab iterations or -1 at maxit. */
int or_predict_cn(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                  const int64_t* cellrec, const double* u, const double* U, const double* nut, double* H,
                  double* ustar, double tol, int32_t maxit);
void or_forcing(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                int64_t nrec, const double* ustar_in, double* ustar_out, double fsum[3]);
void or_faces(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
              const int64_t* cellrec, const double* ustar, double* Ustar);
void or_rhs(const or_grid* g, const or_params* pr, const double* Ustar, double* b);
void or_apply(const or_grid* g, const or_params* pr, const uint8_t* flags, const double* p, double* Ap);
int or_solve(const or_grid* g, const or_params* pr, const uint8_t* flags, const double* b, double* p,
             double tol, int32_t maxit, int32_t solver, double omega, or_stats* st);
void or_correct(const or_grid* g, const or_params* pr, const uint8_t* flags, const double* ustar,
                const double* Ustar, const double* p, double* u, double* U);
/* One fractional step: CSM -> predictor (AB2 or Crank-Nicolson per pr->integrator) -> forcing ->
 * faces -> RHS -> solve -> correction. */
int or_step(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
            int64_t nrec, const int64_t* cellrec, double* u, double* U, double* p, double* Hprev,
            int first_step, double tol, int32_t maxit, int32_t solver, double omega, or_stats* st);

/* Near-field surface force (Eq. force): Shepard inverse-distance average of p on the front and back
 * side of every triangle, F = sum_tri A (p_back - p_front) n.  out[0..2] = force, out[3] = the number
 * of triangles that contributed. */
void or_forces(const or_grid* g, const float* tri, int64_t ntri, const double* p, double out[4]);

/* Viscous force on the body: sum over cut links of nu (u_P - u_G) dx (u_G the Eq. q_axis ghost);
 * out[0..2] = force, out[3] = links used. */
void or_viscous_force(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                      int64_t nrec, const int64_t* cellrec, const double* u, double out[4]);

/* Surface pressure per triangle side (Eq. force) with, if zfilter, the thin-plate filter of
 * Eq. force_filter read as: a cell centre counts for node X only if the open segment from X to it
 * crosses no other triangle.  pside[2t] = front, pside[2t+1] = back Shepard average (NaN if that
 * side has no point).  out[0..2] = sum over sides with a value of -/+ area p n (front/back),
 * out[3] = number of such sides. */
void or_surface_pressure(const or_grid* g, const float* tri, int64_t ntri, const double* p, int zfilter,
                         double* pside, double out[4]);

#ifdef __cplusplus
}
#endif
#endif

/* ibm_oracle.c -- plain FP64 CPU oracle of the topology-free immersed-boundary LES step
 * (Onishi & Tsubokura, "Topology-free immersed boundary method for incompressible turbulence flows").
 *
 * TEST INFRASTRUCTURE ONLY: the definition the CUDA library is checked against and the timed CPU
 * baseline.  Single-threaded loops in the paper's order, no blocking, no fusion.  Compile with
 * -ffp-contract=off so that every product and sum is rounded separately (the classification
 * predicate must be reproducible bit for bit).
 *
 * Readings of points the paper leaves open are marked "Reading:" where they are applied.
 */
#include "ibm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Candidate grid lines of a triangle: its projected bounding box widened by this margin (grid
 * units).  An edge tolerance eps_edge*|W| admits points at most eps_edge * (triangle height) outside
 * the triangle, far below this margin for any triangle smaller than 1e5 cells. */
#define LINE_MARGIN 1e-4

/* ------------------------------------------------------------------------------------------------ */
/* grid helpers                                                                                      */

static int64_t ncells(const or_grid* g) { return (int64_t)g->nx * g->ny * g->nz; }
static int64_t extent(const or_grid* g, int a) { return a == 0 ? g->nx : (a == 1 ? g->ny : g->nz); }
static int64_t stride(const or_grid* g, int a) {
    return a == 0 ? 1 : (a == 1 ? (int64_t)g->nx : (int64_t)g->nx * g->ny);
}
static void coords(const or_grid* g, int64_t c, int64_t x[3]) {
    x[0] = c % g->nx;
    x[1] = (c / g->nx) % g->ny;
    x[2] = c / ((int64_t)g->nx * g->ny);
}
static int64_t cell_at(const or_grid* g, const int64_t x[3]) {
    return x[0] + (int64_t)g->nx * (x[1] + (int64_t)g->ny * x[2]);
}
static int64_t nfaces_axis(const or_grid* g, int a) {
    int64_t d[3] = {g->nx, g->ny, g->nz};
    d[a] += 1;
    return d[0] * d[1] * d[2];
}
/* Face on axis a at position x[a] in [0, n_a] (the low face of cell x when x[a] < n_a). */
static int64_t face_at(const or_grid* g, int a, const int64_t x[3]) {
    int64_t d[3] = {g->nx, g->ny, g->nz};
    d[a] += 1;
    int64_t off = 0;
    for (int b = 0; b < a; ++b) off += nfaces_axis(g, b);
    return off + x[0] + d[0] * (x[1] + d[1] * x[2]);
}
static int link_bit(int a, int s) { return 2 * a + (s > 0 ? 1 : 0); }
static int is_cut(const uint8_t* flags, int64_t P, int a, int s) {
    return (flags[P] >> link_bit(a, s)) & 1;
}
static int popcount6(unsigned m) {
    int n = 0;
    for (int b = 0; b < 6; ++b) n += (m >> b) & 1;
    return n;
}
static int bc_of(const or_params* pr, int a, int s) { return pr->bc[link_bit(a, s)]; }

/* Neighbour P + s e_a: 1 and its index if it is a cell (inside, or across a periodic seam);
 * 0 if it lies beyond a non-periodic domain face. */
static int neighbour(const or_grid* g, const or_params* pr, int64_t P, int a, int s, int64_t* N) {
    int64_t x[3];
    coords(g, P, x);
    int64_t y = x[a] + s, n = extent(g, a);
    if (y < 0 || y >= n) {
        if (bc_of(pr, a, s) != OR_BC_PERIODIC) return 0;
        y = (y + n) % n;
    }
    x[a] = y;
    *N = cell_at(g, x);
    return 1;
}

static const or_record* link_record(const uint8_t* flags, const or_record* rec, const int64_t* cellrec,
                                     int64_t P, int a, int s) {
    unsigned below = (unsigned)(flags[P] & 63) & ((1u << link_bit(a, s)) - 1u);
    return &rec[cellrec[P] + popcount6(below)];
}

/* ------------------------------------------------------------------------------------------------ */
/* Classification: Sec. 2.4.1 (ray tracing from the cell centres along the grid lines).              */
/* The grid line through (q_b, q_c) = (j+1/2, k+1/2) parallel to axis a meets triangle (A,B,C) where  */
/* its 2-D barycentric weights in the (b,c) projection are non-negative.  orient(P,Q,q) is twice the  */
/* signed area of (P,Q,q) in that projection; W = w0 + w1 + w2 is the determinant of Moller-Trumbore */
/* for the direction e_a (up to sign); W == 0 (|W| <= eps_det) means the line is parallel to the     */
/* triangle's plane and is rejected.                                                                 */

static double orient(double Pb, double Pc, double Qb, double Qc, double qb, double qc) {
    double l = (Qb - Pb) * (qc - Pc);
    double r = (Qc - Pc) * (qb - Pb);
    return l - r;
}

typedef struct { int64_t fid; double t; } hit_t;

static int hit_cmp(const void* x, const void* y) {
    const hit_t* a = (const hit_t*)x;
    const hit_t* b = (const hit_t*)y;
    if (a->fid != b->fid) return a->fid < b->fid ? -1 : 1;
    if (a->t != b->t) return a->t < b->t ? -1 : 1;
    return 0;
}

/* Exact predicate for one line; returns 1 and x_hit if the line hits the triangle. */
static int line_hit(const double A[3], const double B[3], const double C[3], int a, double qb, double qc,
                    double eps_edge, double eps_det, double* x_hit) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    double w0 = orient(B[b], B[c], C[b], C[c], qb, qc);
    double w1 = orient(C[b], C[c], A[b], A[c], qb, qc);
    double w2 = orient(A[b], A[c], B[b], B[c], qb, qc);
    double W = (w0 + w1) + w2;
    if (!(fabs(W) > eps_det)) return 0;
    double thr = eps_edge * fabs(W);
    double s0 = W > 0 ? w0 : -w0, s1 = W > 0 ? w1 : -w1, s2 = W > 0 ? w2 : -w2;
    if (!(s0 >= -thr && s1 >= -thr && s2 >= -thr)) return 0;
    double num = (w0 * A[a] + w1 * B[a]) + w2 * C[a];
    *x_hit = num / W;
    return 1;
}

static int64_t clamp_line(double v, int64_t n) {
    if (!(v > -1.0)) return -1;
    if (v > (double)n) return n;
    return (int64_t)v;
}

/* Candidate line range [lo, hi] along transverse axis b for coordinates in [mn, mx]. */
static void line_range(double mn, double mx, int64_t n, int64_t* lo, int64_t* hi) {
    double l = ceil(mn - LINE_MARGIN - 0.5);
    double h = floor(mx + LINE_MARGIN - 0.5);
    int64_t L = l < 0.0 ? 0 : clamp_line(l, n);
    int64_t H = clamp_line(h, n);
    if (H > n - 1) H = n - 1;
    *lo = L;
    *hi = H;
}

static int tri_load(const float* t, double A[3], double B[3], double C[3]) {
    for (int d = 0; d < 3; ++d) {
        A[d] = (double)t[d];
        B[d] = (double)t[3 + d];
        C[d] = (double)t[6 + d];
        if (!isfinite(A[d]) || !isfinite(B[d]) || !isfinite(C[d])) return 0;
    }
    return 1;
}

int64_t or_classify(const or_grid* g, const float* tri, int64_t ntri, double eps_edge, double eps_det,
                    uint8_t* flags, int64_t* face_id, double* t_lo, double* t_hi, int64_t cap,
                    int64_t* n_skipped, int64_t* n_tests) {
    const int64_t N = ncells(g);
    int64_t nh = 0, caph = 1024, skipped = 0, tests = 0;
    hit_t* hits = (hit_t*)malloc((size_t)caph * sizeof(hit_t));
    if (!hits) return -1;
    for (int64_t t = 0; t < ntri; ++t) {
        double A[3], B[3], C[3];
        if (!tri_load(tri + 9 * t, A, B, C)) { ++skipped; continue; }
        for (int a = 0; a < 3; ++a) {
            int b = (a + 1) % 3, c = (a + 2) % 3;
            int64_t jb0, jb1, jc0, jc1;
            line_range(fmin(fmin(A[b], B[b]), C[b]), fmax(fmax(A[b], B[b]), C[b]), extent(g, b), &jb0, &jb1);
            line_range(fmin(fmin(A[c], B[c]), C[c]), fmax(fmax(A[c], B[c]), C[c]), extent(g, c), &jc0, &jc1);
            for (int64_t jc = jc0; jc <= jc1; ++jc)
                for (int64_t jb = jb0; jb <= jb1; ++jb) {
                    double xh;
                    ++tests;
                    if (!line_hit(A, B, C, a, (double)jb + 0.5, (double)jc + 0.5, eps_edge, eps_det, &xh))
                        continue;
                    /* Reading: a hit belongs to the interior face whose centre-to-centre segment
                     * [f+1/2, f+3/2) contains it; t in [0,1) is its position on that segment. */
                    double xm = xh - 0.5;
                    double f = floor(xm);
                    if (!(f >= 0.0 && f <= (double)(extent(g, a) - 2))) continue;
                    double tt = xm - f;
                    int64_t x[3];
                    x[a] = (int64_t)f;
                    x[b] = jb;
                    x[c] = jc;
                    if (nh == caph) {
                        caph *= 2;
                        hit_t* nhits = (hit_t*)realloc(hits, (size_t)caph * sizeof(hit_t));
                        if (!nhits) { free(hits); return -1; }
                        hits = nhits;
                    }
                    hits[nh].fid = (int64_t)a * N + cell_at(g, x);
                    hits[nh].t = tt;
                    ++nh;
                }
        }
    }
    qsort(hits, (size_t)nh, sizeof(hit_t), hit_cmp);
    for (int64_t c = 0; c < N; ++c) flags[c] = 0;
    int64_t ncut = 0;
    for (int64_t h = 0; h < nh;) {
        int64_t e = h;
        double lo = hits[h].t, hi = hits[h].t;
        while (e < nh && hits[e].fid == hits[h].fid) {
            if (hits[e].t < lo) lo = hits[e].t;
            if (hits[e].t > hi) hi = hits[e].t;
            ++e;
        }
        int64_t fid = hits[h].fid;
        if (ncut < cap) {
            face_id[ncut] = fid;
            t_lo[ncut] = lo;
            t_hi[ncut] = hi;
        }
        int a = (int)(fid / N);
        int64_t lower = fid % N;
        flags[lower] |= (uint8_t)(1u << link_bit(a, +1));
        flags[lower + stride(g, a)] |= (uint8_t)(1u << link_bit(a, -1));
        ++ncut;
        h = e;
    }
    free(hits);
    if (n_skipped) *n_skipped = skipped;
    if (n_tests) *n_tests = tests;
    return ncut;
}

/* Moller-Trumbore (1997) with ray origin at the line's point on the plane x_a = 0 and direction e_a. */
static int mt_hit(const double A[3], const double B[3], const double C[3], int a, double qb, double qc,
                  double eps, double* x_hit) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    double O[3], D[3] = {0, 0, 0}, e1[3], e2[3], h[3], s[3], q[3];
    O[a] = 0.0; O[b] = qb; O[c] = qc;
    D[a] = 1.0;
    for (int d = 0; d < 3; ++d) { e1[d] = B[d] - A[d]; e2[d] = C[d] - A[d]; s[d] = O[d] - A[d]; }
    h[0] = D[1] * e2[2] - D[2] * e2[1];
    h[1] = D[2] * e2[0] - D[0] * e2[2];
    h[2] = D[0] * e2[1] - D[1] * e2[0];
    double det = e1[0] * h[0] + e1[1] * h[1] + e1[2] * h[2];
    if (fabs(det) <= eps) return 0;
    double inv = 1.0 / det;
    double u = inv * (s[0] * h[0] + s[1] * h[1] + s[2] * h[2]);
    if (u < 0.0 || u > 1.0) return 0;
    q[0] = s[1] * e1[2] - s[2] * e1[1];
    q[1] = s[2] * e1[0] - s[0] * e1[2];
    q[2] = s[0] * e1[1] - s[1] * e1[0];
    double v = inv * (D[0] * q[0] + D[1] * q[1] + D[2] * q[2]);
    if (v < 0.0 || u + v > 1.0) return 0;
    *x_hit = inv * (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]);
    return 1;
}

int64_t or_mt_disagreements(const or_grid* g, const float* tri, int64_t ntri, double eps_edge,
                            double eps_det) {
    int64_t bad = 0;
    for (int64_t t = 0; t < ntri; ++t) {
        double A[3], B[3], C[3];
        if (!tri_load(tri + 9 * t, A, B, C)) continue;
        for (int a = 0; a < 3; ++a) {
            int b = (a + 1) % 3, c = (a + 2) % 3;
            int64_t jb0, jb1, jc0, jc1;
            line_range(fmin(fmin(A[b], B[b]), C[b]), fmax(fmax(A[b], B[b]), C[b]), extent(g, b), &jb0, &jb1);
            line_range(fmin(fmin(A[c], B[c]), C[c]), fmax(fmax(A[c], B[c]), C[c]), extent(g, c), &jc0, &jc1);
            for (int64_t jc = jc0; jc <= jc1; ++jc)
                for (int64_t jb = jb0; jb <= jb1; ++jb) {
                    double x1 = 0, x2 = 0;
                    int h1 = line_hit(A, B, C, a, jb + 0.5, jc + 0.5, eps_edge, eps_det, &x1);
                    int h2 = mt_hit(A, B, C, a, jb + 0.5, jc + 0.5, 1e-300, &x2);
                    if (h1 != h2 || (h1 && fabs(x1 - x2) > 1e-9)) ++bad;
                }
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------------------------------ */
/* Setup: Omega_inc / Omega_adj (Eq. dummy_cell_region), ghost branches (Eq. q_axis), D (Eq.          */
/* distribution_function).                                                                          */

static int64_t find_face(const int64_t* face_id, int64_t n, int64_t fid) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (face_id[mid] == fid) return mid;
        if (face_id[mid] < fid) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

int64_t or_setup(const or_grid* g, uint8_t* flags, const int64_t* face_id, const double* t_lo,
                 const double* t_hi, int64_t n_cut, or_record* rec, int64_t* cellrec,
                 int64_t* inc_list, int64_t* n_inc) {
    const int64_t N = ncells(g);
    for (int64_t P = 0; P < N; ++P) {
        flags[P] &= 63;
        if (flags[P]) flags[P] |= 64;                      /* Omega_inc: the cell has a cut link */
    }
    for (int64_t P = 0; P < N; ++P) {
        if (flags[P] & 64) continue;
        int64_t x[3];
        coords(g, P, x);
        int adj = 0;
        for (int a = 0; a < 3; ++a)
            for (int s = -1; s <= 1; s += 2) {
                int64_t y = x[a] + s;
                if (y < 0 || y >= extent(g, a)) continue;
                if (flags[P + s * stride(g, a)] & 64) adj = 1;
            }
        if (adj) flags[P] |= 128;                           /* Omega_adj */
    }
    int64_t k = 0, ninc = 0;
    for (int64_t P = 0; P < N; ++P) {
        if (!(flags[P] & 64)) { cellrec[P] = -1; continue; }
        cellrec[P] = k;
        inc_list[ninc++] = P;
        int64_t x[3];
        coords(g, P, x);
        for (int bit = 0; bit < 6; ++bit) {
            if (!((flags[P] >> bit) & 1)) continue;
            int a = bit / 2, s = (bit & 1) ? +1 : -1;
            int64_t lower = s > 0 ? P : P - stride(g, a);
            int64_t idx = find_face(face_id, n_cut, (int64_t)a * N + lower);
            if (idx < 0) return -1;
            or_record* r = &rec[k++];
            double d = s > 0 ? t_lo[idx] : 1.0 - t_hi[idx];
            r->cell = P;
            r->far = P + s * stride(g, a);
            r->axis = a;
            r->side = s;
            r->d = d;
            int64_t yo = x[a] - s;
            int o_ok = (yo >= 0 && yo < extent(g, a)) && !is_cut(flags, P, a, -s);
            if (d >= 0.5) {                     /* Eq. q_axis, upper branch */
                r->branch = 0;
                r->opp = -1;
                r->c_ib = 1.0 / d;
                r->c_p = (d - 1.0) / d;
                r->c_o = 0.0;
            } else if (o_ok) {                  /* Eq. q_axis, lower branch */
                r->branch = 1;
                r->opp = P - s * stride(g, a);
                r->c_ib = 2.0;
                r->c_o = 2.0 * d - 1.0;
                r->c_p = -2.0 * d;
            } else {
                /* Reading: the lower branch needs the opposite neighbour O; when O is itself behind a
                 * wall or outside the domain, fall back to the upper branch evaluated at d = 1/2. */
                r->branch = 2;
                r->opp = -1;
                r->c_ib = 2.0;
                r->c_p = -1.0;
                r->c_o = 0.0;
            }
            /* Eq. distribution_function at the near cell's distance d: fluid and ghost branch. */
            r->w_fluid = d / (1.0 + d);
            r->w_ghost = (1.0 - d) / (1.0 + d);
            r->uib[0] = r->uib[1] = r->uib[2] = 0.0;
        }
    }
    *n_inc = ninc;
    return k;
}

/* ------------------------------------------------------------------------------------------------ */
/* Values read across a link: neighbour, IB ghost (Eq. q_axis / Neumann), or domain-boundary ghost.   */

/* Value of component comp read by P across link (a, s).  hom != 0 drops the inhomogeneous parts of
 * the ghost values (wall velocity u_IB, inflow velocity), which leaves the linear part used by the
 * implicit operator of the Crank-Nicolson predictor. */
static double velocity_across_h(const or_grid* g, const or_params* pr, const uint8_t* flags,
                                const or_record* rec, const int64_t* cellrec, const double* u,
                                int comp, int64_t P, int a, int s, int hom) {
    const int64_t N = ncells(g);
    double uP = u[comp * N + P];
    if (is_cut(flags, P, a, s)) {
        const or_record* r = link_record(flags, rec, cellrec, P, a, s);
        double v = (hom ? 0.0 : r->c_ib * r->uib[comp]) + r->c_p * uP;
        if (r->opp >= 0) v = v + r->c_o * u[comp * N + r->opp];
        return v;
    }
    int64_t Nb;
    if (neighbour(g, pr, P, a, s, &Nb)) return u[comp * N + Nb];
    /* Reading of the outer boundary conditions (the paper omits them). */
    switch (bc_of(pr, a, s)) {
        case OR_BC_INFLOW: return (hom ? 0.0 : 2.0 * pr->u_in[comp]) - uP;
        case OR_BC_OUTFLOW: return uP;
        case OR_BC_SLIP: return comp == a ? -uP : uP;
        default: return -uP; /* no-slip */
    }
}

double or_velocity_across(const or_grid* g, const or_params* pr, const uint8_t* flags,
                          const or_record* rec, const int64_t* cellrec, const double* u,
                          int comp, int64_t P, int a, int s) {
    return velocity_across_h(g, pr, flags, rec, cellrec, u, comp, P, a, s, 0);
}

static double p_across(const or_grid* g, const or_params* pr, const uint8_t* flags, const double* p,
                       int64_t P, int a, int s) {
    if (is_cut(flags, P, a, s)) return p[P];        /* Neumann on the IB: zeta = 1, eta = 0 */
    int64_t Nb;
    if (neighbour(g, pr, P, a, s, &Nb)) return p[Nb];
    return bc_of(pr, a, s) == OR_BC_OUTFLOW ? -p[P] : p[P];
}

/* grad[a][b] = d u_b / d x_a by central differences through the link values. */
static void velocity_gradient_h(const or_grid* g, const or_params* pr, const uint8_t* flags,
                                const or_record* rec, const int64_t* cellrec, const double* u,
                                int64_t P, double grad[3][3], int hom) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double up = velocity_across_h(g, pr, flags, rec, cellrec, u, b, P, a, +1, hom);
            double um = velocity_across_h(g, pr, flags, rec, cellrec, u, b, P, a, -1, hom);
            grad[a][b] = (up - um) / (2.0 * g->dx);
        }
}

static void velocity_gradient(const or_grid* g, const or_params* pr, const uint8_t* flags,
                              const or_record* rec, const int64_t* cellrec, const double* u,
                              int64_t P, double grad[3][3]) {
    velocity_gradient_h(g, pr, flags, rec, cellrec, u, P, grad, 0);
}

/* ------------------------------------------------------------------------------------------------ */
/* CSM eddy viscosity: Eq. Smagorinsky, Eq. Q, Eq. FCS (Sec. 2.3).                                   */

void or_csm(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
            const int64_t* cellrec, const double* u, double* nut) {
    const int64_t N = ncells(g);
    const double delta = g->dx;   /* (dx dy dz)^(1/3) on a uniform grid */
    for (int64_t P = 0; P < N; ++P) {
        double G[3][3], SS = 0.0, WW = 0.0;
        velocity_gradient(g, pr, flags, rec, cellrec, u, P, G);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double S = 0.5 * (G[a][b] + G[b][a]);
                double W = 0.5 * (G[a][b] - G[b][a]);
                SS += S * S;
                WW += W * W;
            }
        double Q = 0.5 * (WW - SS);
        double E = 0.5 * (WW + SS);
        double F = E > 0.0 ? Q / E : 0.0;            /* reading: F_CS = 0 where E = 0 */
        double C = (1.0 / 20.0) * (fabs(F) * sqrt(fabs(F)));
        nut[P] = C * delta * delta * sqrt(SS);      /* |S| = sqrt(S_ij S_ij) as printed */
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Momentum predictor: flux-form central differences with face velocity U (Sec. 2.1), SGS stress     */
/* divergence of 2 nu_t S (Eq. SGSstress), Adams-Bashforth 2 in time (Sec. 2.5).                     */

static double face_velocity(const or_grid* g, const double* U, int64_t P, int a, int s) {
    int64_t x[3];
    coords(g, P, x);
    if (s > 0) x[a] += 1;
    return U[face_at(g, a, x)];
}

/* Advected value on the face of P towards side s along axis a (Sec. 3.1/3.3: central differencing
 * blended with a fraction `quick` of QUICK, the "hybrid" scheme).  With L the lower and R the upper
 * cell of the face, QUICK takes (6 upwind + 3 downwind - far upwind)/8, the far upwind value read
 * across the upwind cell's outer link (neighbour, ghost or boundary value).  Both cells of a face get
 * the same value, so the advective fluxes still telescope. */
static double face_advected(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                            const int64_t* cellrec, const double* u, int comp, int64_t P, int a, int s,
                            double uP, double uN, double Uf, int hom) {
    const int64_t N = ncells(g);
    double central = 0.5 * (uP + uN);
    if (pr->quick == 0.0) return central;
    int64_t Nb;
    if (is_cut(flags, P, a, s) || !neighbour(g, pr, P, a, s, &Nb)) return central;
    int64_t Lc = s > 0 ? P : Nb, Rc = s > 0 ? Nb : P;
    double uL = u[comp * N + Lc], uR = u[comp * N + Rc], q;
    if (Uf >= 0.0) {
        double far = velocity_across_h(g, pr, flags, rec, cellrec, u, comp, Lc, a, -1, hom);
        q = (6.0 * uL + 3.0 * uR - far) / 8.0;
    } else {
        double far = velocity_across_h(g, pr, flags, rec, cellrec, u, comp, Rc, a, +1, hom);
        q = (6.0 * uR + 3.0 * uL - far) / 8.0;
    }
    return (1.0 - pr->quick) * central + pr->quick * q;
}

/* L(u) of cell P: flux-form advection with the face velocity U, diffusion with nu + nu_t and the
 * transpose part of the SGS stress, summed over the six faces and divided by dx (per unit volume).
 * U and nu_t are held fixed, so L is affine in u; hom != 0 gives its linear part. */
static void momentum_flux(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                          const int64_t* cellrec, const double* u, const double* U, const double* nut,
                          int64_t P, int hom, double out[3]) {
    const int64_t N = ncells(g);
    const double dx = g->dx, nu = pr->nu;
    double GP[3][3], h[3] = {0.0, 0.0, 0.0};
    velocity_gradient_h(g, pr, flags, rec, cellrec, u, P, GP, hom);
    for (int a = 0; a < 3; ++a)
        for (int s = -1; s <= 1; s += 2) {
            double Uf = face_velocity(g, U, P, a, s);
            int64_t Nb = -1;
            int interior = !is_cut(flags, P, a, s) && neighbour(g, pr, P, a, s, &Nb);
            double nutf = interior ? 0.5 * (nut[P] + nut[Nb]) : nut[P];
            double GN[3][3];
            if (interior) velocity_gradient_h(g, pr, flags, rec, cellrec, u, Nb, GN, hom);
            for (int i = 0; i < 3; ++i) {
                double uP = u[i * N + P];
                double uN = velocity_across_h(g, pr, flags, rec, cellrec, u, i, P, a, s, hom);
                double D1 = (uN - uP) / dx;
                /* transpose part of 2 S: (d u_a / d x_i) on the face, oriented along +e_a */
                double T;
                if (i == a) T = D1;
                else if (interior) T = (double)s * 0.5 * (GP[i][a] + GN[i][a]);
                else T = (double)s * GP[i][a];
                double conv = -(double)s * Uf * face_advected(g, pr, flags, rec, cellrec, u, i, P, a, s, uP, uN, Uf, hom);
                h[i] += conv + (nu + nutf) * D1 + nutf * T;
            }
        }
    for (int i = 0; i < 3; ++i) out[i] = h[i] / dx;
}

void or_momentum_operator(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                          const int64_t* cellrec, const double* u, const double* U, const double* nut,
                          int hom, double* L) {
    const int64_t N = ncells(g);
    for (int64_t P = 0; P < N; ++P) {
        double h[3];
        momentum_flux(g, pr, flags, rec, cellrec, u, U, nut, P, hom, h);
        for (int i = 0; i < 3; ++i) L[i * N + P] = h[i];
    }
}

void or_predict(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                const int64_t* cellrec, const double* u, const double* U, const double* nut,
                const double* Hprev, double* H, double* ustar, int first_step) {
    const int64_t N = ncells(g);
    const double dt = pr->dt;
    or_momentum_operator(g, pr, flags, rec, cellrec, u, U, nut, 0, H);
    for (int64_t P = 0; P < N; ++P)
        for (int i = 0; i < 3; ++i) {
            double hi = H[i * N + P], uP = u[i * N + P];
            if (first_step)
                ustar[i * N + P] = uP + dt * hi;
            else
                ustar[i * N + P] = uP + dt * (1.5 * hi - 0.5 * Hprev[i * N + P]);
        }
}

/* Crank-Nicolson predictor (Eq. crank-nicolson): (u* - u^n)/dt = (L(u*) + L(u^n))/2 with U = U^n and
 * nu_t = nu_t(u^n) in both halves.  With delta = u* - u^n and L_0 the linear part of L this is
 *   M delta = delta - (dt/2) L_0(delta) = dt L(u^n),
 * one system over the stacked three components (the transpose SGS term couples them), solved by
 * BiCGStab (the paper's Krylov solver) from delta = 0 to ||dt L(u^n) - M delta|| <= tol ||dt L(u^n)||.
 * H receives L(u^n).  Returns the BiCGStab iterations, or -1 if maxit was reached. */
static void cn_matvec(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                      const int64_t* cellrec, const double* U, const double* nut, const double* x, double* y) {
    const int64_t n3 = 3 * ncells(g);
    or_momentum_operator(g, pr, flags, rec, cellrec, x, U, nut, 1, y);
    for (int64_t i = 0; i < n3; ++i) y[i] = x[i] - 0.5 * pr->dt * y[i];
}

int or_predict_cn(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                  const int64_t* cellrec, const double* u, const double* U, const double* nut, double* H,
                  double* ustar, double tol, int32_t maxit) {
    const int64_t n3 = 3 * ncells(g);
    double* b = (double*)malloc((size_t)n3 * sizeof(double));
    double* x = (double*)calloc((size_t)n3, sizeof(double));
    double* r = (double*)malloc((size_t)n3 * sizeof(double));
    double* rh = (double*)malloc((size_t)n3 * sizeof(double));
    double* p = (double*)calloc((size_t)n3, sizeof(double));
    double* v = (double*)calloc((size_t)n3, sizeof(double));
    double* sv = (double*)malloc((size_t)n3 * sizeof(double));
    double* t = (double*)malloc((size_t)n3 * sizeof(double));
    or_momentum_operator(g, pr, flags, rec, cellrec, u, U, nut, 0, H);
    for (int64_t i = 0; i < n3; ++i) b[i] = pr->dt * H[i];
    double bn = 0.0;
    for (int64_t i = 0; i < n3; ++i) bn += b[i] * b[i];
    bn = sqrt(bn);
    int it = 0, ok = 1;
    memcpy(r, b, (size_t)n3 * sizeof(double));          /* x0 = 0 */
    memcpy(rh, r, (size_t)n3 * sizeof(double));
    double rho = 1.0, alpha = 1.0, omega = 1.0, rn = bn;
    while (bn > 0.0 && rn > tol * bn) {
        if (it >= maxit) { ok = 0; break; }
        double rho1 = 0.0;
        for (int64_t i = 0; i < n3; ++i) rho1 += rh[i] * r[i];
        double beta = (rho1 / rho) * (alpha / omega);
        for (int64_t i = 0; i < n3; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        cn_matvec(g, pr, flags, rec, cellrec, U, nut, p, v);
        double rv = 0.0;
        for (int64_t i = 0; i < n3; ++i) rv += rh[i] * v[i];
        alpha = rho1 / rv;
        for (int64_t i = 0; i < n3; ++i) sv[i] = r[i] - alpha * v[i];
        cn_matvec(g, pr, flags, rec, cellrec, U, nut, sv, t);
        double ts = 0.0, tt = 0.0;
        for (int64_t i = 0; i < n3; ++i) { ts += t[i] * sv[i]; tt += t[i] * t[i]; }
        omega = tt > 0.0 ? ts / tt : 0.0;
        rn = 0.0;
        for (int64_t i = 0; i < n3; ++i) {
            x[i] += alpha * p[i] + omega * sv[i];
            r[i] = sv[i] - omega * t[i];
            rn += r[i] * r[i];
        }
        rn = sqrt(rn);
        rho = rho1;
        ++it;
        if (omega == 0.0) break;
    }
    for (int64_t i = 0; i < n3; ++i) ustar[i] = u[i] + x[i];
    free(b); free(x); free(r); free(rh); free(p); free(v); free(sv); free(t);
    return ok ? it : -1;
}

/* ------------------------------------------------------------------------------------------------ */
/* Distributed direct forcing: Eq. forcing_term, Eq. discrete_forcing_term, Eq. distribution_function,*/
/* dead-end filter Eq. deadend_filter.  Reading: the velocity at the intersection X is the linear     */
/* interpolant of the background u* between P and the cell G behind the wall, and the force          */
/* (u_IB - u*_X)/dt is spread to P with the ghost branch of D, (dx - d)/(dx + d).  Three facts give    */
/* this reading.  P is a ghost cell of the dummy stencil of the cell across the wall.  At d = 0 the   */
/* weight is 1, so P lands on u_IB exactly: Gibou's imposition, which the paper says D follows.  And  */
/* P's push stays in proportion to its share (1 - d/dx) of u*_X, so every push also corrects u*_X.    */
/* The fluid branch d/(dx + d) lacks that last property: at d -> dx it pushes P by half the mismatch  */
/* while P no longer enters u*_X, and on the Taylor-Green case of Sec. 2.5 with a wall through cell   */
/* centres that drift grows without bound.  G is forced through its own records.  All records use the */
/* background u*.                                                                                   */

void or_forcing(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                int64_t nrec, const double* ustar_in, double* ustar_out, double fsum[3]) {
    const int64_t N = ncells(g);
    const double dt = pr->dt, vol = g->dx * g->dx * g->dx;
    double* delta = (double*)calloc((size_t)(3 * N), sizeof(double));
    double* wsum = (double*)calloc((size_t)N, sizeof(double));
    fsum[0] = fsum[1] = fsum[2] = 0.0;
    for (int64_t r = 0; r < nrec; ++r) {
        const or_record* R = &rec[r];
        int64_t P = R->cell, G = R->far;
        int dead_P = pr->deadend_on && popcount6(flags[P] & 63) >= 5;
        if (!dead_P) wsum[P] += R->w_ghost;
        for (int i = 0; i < 3; ++i) {
            double uX = (1.0 - R->d) * ustar_in[i * N + P] + R->d * ustar_in[i * N + G];
            double F = (R->uib[i] - uX) / dt;
            if (!dead_P) delta[i * N + P] += dt * R->w_ghost * F;
        }
    }
    /* Reading: a cell crossed by several IB points receives the sum of their spread forces; where the
     * printed weights add up to more than 1 the sum is divided by that total, so that the explicit
     * update stays a relaxation towards u_IB (unnormalised sums over-correct and grow step by step). */
    for (int i = 0; i < 3; ++i)
        for (int64_t P = 0; P < N; ++P) {
            double dlt = wsum[P] > 1.0 ? delta[i * N + P] / wsum[P] : delta[i * N + P];
            ustar_out[i * N + P] = ustar_in[i * N + P] + dlt;
            fsum[i] += dlt * vol;
        }
    free(delta);
    free(wsum);
}

/* ------------------------------------------------------------------------------------------------ */
/* Face velocities of the intermediate field (the interface velocity U of Sec. 2.1).                 */
/* Reading (Rhie-Chow, the paper gives no formula): U*_f is the average of the two cell values on    */
/* uncut interior faces, the boundary value on inflow/wall faces and the adjacent cell value on       */
/* outflow faces, which are then shifted uniformly so that the net boundary flux is zero.             */
/* Reading (cut faces): the wall's own normal velocity, the mean of u_IB.e_a over the face's two link */
/* records (one per side; a side without a record is left out).  It is zero for a stationary body,   */
/* so every sealed pocket's right-hand side sums to zero.  With a prescribed wall velocity, as in the */
/* Taylor-Green verification of Sec. 2.5, fluid crosses the wall at that velocity.                   */

static double cut_face_velocity(const uint8_t* flags, const or_record* rec, const int64_t* cellrec,
                                int64_t L, int64_t R, int a) {
    double sum = link_record(flags, rec, cellrec, L, a, +1)->uib[a];
    double n = 1.0;
    if (is_cut(flags, R, a, -1)) {
        sum += link_record(flags, rec, cellrec, R, a, -1)->uib[a];
        n = 2.0;
    }
    return sum / n;
}

void or_faces(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
              const int64_t* cellrec, const double* ustar, double* Ustar) {
    const int64_t N = ncells(g);
    double phi_other = 0.0, phi_out = 0.0;
    int64_t n_out = 0;
    for (int a = 0; a < 3; ++a) {
        int64_t n = extent(g, a);
        int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int64_t jc = 0; jc < extent(g, c); ++jc)
            for (int64_t jb = 0; jb < extent(g, b); ++jb)
                for (int64_t f = 0; f <= n; ++f) {
                    int64_t x[3];
                    x[a] = f; x[b] = jb; x[c] = jc;
                    int64_t fi = face_at(g, a, x);
                    if (f > 0 && f < n) {
                        int64_t xl[3] = {x[0], x[1], x[2]};
                        xl[a] = f - 1;
                        int64_t L = cell_at(g, xl), R = cell_at(g, x);
                        Ustar[fi] = is_cut(flags, L, a, +1) ? cut_face_velocity(flags, rec, cellrec, L, R, a)
                                                            : 0.5 * (ustar[a * N + L] + ustar[a * N + R]);
                        continue;
                    }
                    int s = f == 0 ? -1 : +1;
                    int bc = bc_of(pr, a, s);
                    int64_t xin[3] = {x[0], x[1], x[2]};
                    xin[a] = f == 0 ? 0 : n - 1;
                    int64_t Pin = cell_at(g, xin);
                    double v;
                    if (bc == OR_BC_PERIODIC) {
                        int64_t xl[3] = {x[0], x[1], x[2]}, xr[3] = {x[0], x[1], x[2]};
                        xl[a] = n - 1; xr[a] = 0;
                        v = 0.5 * (ustar[a * N + cell_at(g, xl)] + ustar[a * N + cell_at(g, xr)]);
                    } else if (bc == OR_BC_INFLOW) {
                        v = pr->u_in[a];
                        phi_other += (double)s * v;
                    } else if (bc == OR_BC_OUTFLOW) {
                        v = ustar[a * N + Pin];
                        phi_out += (double)s * v;
                        ++n_out;
                    } else {
                        v = 0.0;
                    }
                    Ustar[fi] = v;
                }
    }
    if (n_out > 0) {
        double shift = (-phi_other - phi_out) / (double)n_out;   /* outward flux per outflow face */
        for (int a = 0; a < 3; ++a) {
            int64_t n = extent(g, a);
            int b = (a + 1) % 3, c = (a + 2) % 3;
            for (int s = -1; s <= 1; s += 2) {
                if (bc_of(pr, a, s) != OR_BC_OUTFLOW) continue;
                for (int64_t jc = 0; jc < extent(g, c); ++jc)
                    for (int64_t jb = 0; jb < extent(g, b); ++jb) {
                        int64_t x[3];
                        x[a] = s < 0 ? 0 : n; x[b] = jb; x[c] = jc;
                        Ustar[face_at(g, a, x)] += (double)s * shift;
                    }
            }
        }
    }
}

/* Eq. poisson right-hand side: b = div(U*) / dt (finite-volume divergence over the six faces). */
void or_rhs(const or_grid* g, const or_params* pr, const double* Ustar, double* b) {
    const int64_t N = ncells(g);
    for (int64_t P = 0; P < N; ++P) {
        int64_t x[3];
        coords(g, P, x);
        double div = 0.0;
        for (int a = 0; a < 3; ++a) {
            int64_t xh[3] = {x[0], x[1], x[2]};
            xh[a] += 1;
            div += Ustar[face_at(g, a, xh)] - Ustar[face_at(g, a, x)];
        }
        b[P] = div / (g->dx * pr->dt);
    }
}

/* Eq. poisson operator: (A p)_P = sum over the six links of (p_N - p_P)/dx^2, where a cut link or a   */
/* wall/inflow face carries no flux (Neumann) and an outflow face holds p = 0 (ghost -p_P).          */
void or_apply(const or_grid* g, const or_params* pr, const uint8_t* flags, const double* p, double* Ap) {
    const int64_t N = ncells(g);
    const double idx2 = 1.0 / (g->dx * g->dx);
    for (int64_t P = 0; P < N; ++P) {
        double s_ = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int s = -1; s <= 1; s += 2) {
                if (is_cut(flags, P, a, s)) continue;
                int64_t Nb;
                if (neighbour(g, pr, P, a, s, &Nb)) s_ += p[Nb] - p[P];
                else if (bc_of(pr, a, s) == OR_BC_OUTFLOW) s_ += -p[P] - p[P];
            }
        Ap[P] = s_ * idx2;
    }
}

static double dot(const double* x, const double* y, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

/* Residual r = b - A p; returns ||r||_2. */
static double residual(const or_grid* g, const or_params* pr, const uint8_t* flags, const double* b,
                       const double* p, double* r, double* tmp) {
    const int64_t N = ncells(g);
    or_apply(g, pr, flags, p, tmp);
    for (int64_t i = 0; i < N; ++i) r[i] = b[i] - tmp[i];
    return sqrt(dot(r, r, N));
}

/* Pressure solve (Sec. 2.1: BiCGStab or red-black SOR over the whole domain; CG is added because the */
/* operator is symmetric).  Stops at ||b - A p||_2 <= tol ||b||_2 (reading: relative to ||b||).       */
int or_solve(const or_grid* g, const or_params* pr, const uint8_t* flags, const double* b, double* p,
             double tol, int32_t maxit, int32_t solver, double omega, or_stats* st) {
    const int64_t N = ncells(g);
    double* r = (double*)malloc((size_t)N * sizeof(double));
    double* w = (double*)malloc((size_t)N * sizeof(double));
    double* d = (double*)malloc((size_t)N * sizeof(double));
    double* v = (double*)malloc((size_t)N * sizeof(double));
    double* s = (double*)malloc((size_t)N * sizeof(double));
    double* t = (double*)malloc((size_t)N * sizeof(double));
    double* rh = (double*)malloc((size_t)N * sizeof(double));
    double bn = sqrt(dot(b, b, N));
    double rn = residual(g, pr, flags, b, p, r, w);
    int it = 0, status = 0;
    st->bnorm = bn;
    if (bn == 0.0 || rn <= tol * bn) goto done;
    if (solver == OR_SOLVER_CG) {
        memcpy(d, r, (size_t)N * sizeof(double));
        double rr = dot(r, r, N);
        while (it < maxit) {
            or_apply(g, pr, flags, d, w);
            double alpha = rr / dot(d, w, N);
            for (int64_t i = 0; i < N; ++i) { p[i] += alpha * d[i]; r[i] -= alpha * w[i]; }
            double rr2 = dot(r, r, N);
            ++it;
            if (sqrt(rr2) <= tol * bn) {
                rn = residual(g, pr, flags, b, p, r, w);   /* confirm on the true residual */
                if (rn <= tol * bn) break;
                rr2 = rn * rn;
                memcpy(d, r, (size_t)N * sizeof(double));
                rr = rr2;
                continue;
            }
            double beta = rr2 / rr;
            for (int64_t i = 0; i < N; ++i) d[i] = r[i] + beta * d[i];
            rr = rr2;
        }
    } else if (solver == OR_SOLVER_BICGSTAB) {
        double rho = 1.0, alpha = 1.0, om = 1.0;
        memcpy(rh, r, (size_t)N * sizeof(double));
        memset(v, 0, (size_t)N * sizeof(double));
        memset(d, 0, (size_t)N * sizeof(double));
        while (it < maxit) {
            double rho2 = dot(rh, r, N);
            if (rho2 == 0.0 || om == 0.0) {              /* breakdown: restart from the true residual */
                rn = residual(g, pr, flags, b, p, r, w);
                memcpy(rh, r, (size_t)N * sizeof(double));
                memset(v, 0, (size_t)N * sizeof(double));
                memset(d, 0, (size_t)N * sizeof(double));
                rho = alpha = om = 1.0;
                rho2 = dot(rh, r, N);
                if (rho2 == 0.0) break;
            }
            double beta = (rho2 / rho) * (alpha / om);
            for (int64_t i = 0; i < N; ++i) d[i] = r[i] + beta * (d[i] - om * v[i]);
            or_apply(g, pr, flags, d, v);
            alpha = rho2 / dot(rh, v, N);
            for (int64_t i = 0; i < N; ++i) s[i] = r[i] - alpha * v[i];
            ++it;
            if (sqrt(dot(s, s, N)) <= tol * bn) {
                for (int64_t i = 0; i < N; ++i) p[i] += alpha * d[i];
                rn = residual(g, pr, flags, b, p, r, w);
                if (rn <= tol * bn) break;
                om = 0.0;                                  /* force a restart */
                rho = rho2;
                continue;
            }
            or_apply(g, pr, flags, s, t);
            double tt = dot(t, t, N);
            om = tt > 0.0 ? dot(t, s, N) / tt : 0.0;
            for (int64_t i = 0; i < N; ++i) { p[i] += alpha * d[i] + om * s[i]; r[i] = s[i] - om * t[i]; }
            rho = rho2;
            if (sqrt(dot(r, r, N)) <= tol * bn) {
                rn = residual(g, pr, flags, b, p, r, w);
                if (rn <= tol * bn) break;
                om = 0.0;
            }
        }
    } else {
        /* Red-black SOR: colour (i+j+k) mod 2, red first. */
        const double idx2 = 1.0 / (g->dx * g->dx);
        while (it < maxit) {
            for (int colour = 0; colour < 2; ++colour)
                for (int64_t P = 0; P < N; ++P) {
                    int64_t x[3];
                    coords(g, P, x);
                    if (((x[0] + x[1] + x[2]) & 1) != colour) continue;
                    double diag = 0.0, off = 0.0;
                    for (int a = 0; a < 3; ++a)
                        for (int sd = -1; sd <= 1; sd += 2) {
                            if (is_cut(flags, P, a, sd)) continue;
                            int64_t Nb;
                            if (neighbour(g, pr, P, a, sd, &Nb)) { diag -= idx2; off += p[Nb] * idx2; }
                            else if (bc_of(pr, a, sd) == OR_BC_OUTFLOW) diag -= 2.0 * idx2;
                        }
                    if (diag == 0.0) continue;
                    double gs = (b[P] - off) / diag;
                    p[P] = (1.0 - omega) * p[P] + omega * gs;
                }
            ++it;
            rn = residual(g, pr, flags, b, p, r, w);
            if (rn <= tol * bn) break;
        }
    }
    rn = residual(g, pr, flags, b, p, r, w);
    if (!(rn <= tol * bn)) status = 4;
done:
    st->iters = it;
    st->status = status;
    st->relres = bn > 0.0 ? rn / bn : 0.0;
    free(r); free(w); free(d); free(v); free(s); free(t); free(rh);
    return status;
}

/* Eq. correction: u = u* - dt grad p.  Cell values use the central gradient through the link values, */
/* face values the compact gradient across the face (reading of the Rhie-Chow interpolation), so     */
/* that div U^{n+1} = dt (b - A p) cell by cell.                                                    */
void or_correct(const or_grid* g, const or_params* pr, const uint8_t* flags, const double* ustar,
                const double* Ustar, const double* p, double* u, double* U) {
    const int64_t N = ncells(g);
    const double dx = g->dx, dt = pr->dt;
    for (int64_t P = 0; P < N; ++P)
        for (int a = 0; a < 3; ++a) {
            double pp = p_across(g, pr, flags, p, P, a, +1);
            double pm = p_across(g, pr, flags, p, P, a, -1);
            u[a * N + P] = ustar[a * N + P] - dt * (pp - pm) / (2.0 * dx);
        }
    for (int a = 0; a < 3; ++a) {
        int64_t n = extent(g, a);
        int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int64_t jc = 0; jc < extent(g, c); ++jc)
            for (int64_t jb = 0; jb < extent(g, b); ++jb)
                for (int64_t f = 0; f <= n; ++f) {
                    int64_t x[3];
                    x[a] = f; x[b] = jb; x[c] = jc;
                    int64_t fi = face_at(g, a, x);
                    double pl, pr_;
                    if (f > 0 && f < n) {
                        int64_t xl[3] = {x[0], x[1], x[2]};
                        xl[a] = f - 1;
                        int64_t L = cell_at(g, xl), R = cell_at(g, x);
                        if (is_cut(flags, L, a, +1)) { U[fi] = Ustar[fi]; continue; }
                        pl = p[L]; pr_ = p[R];
                    } else {
                        int s = f == 0 ? -1 : +1;
                        int bc = bc_of(pr, a, s);
                        int64_t xin[3] = {x[0], x[1], x[2]};
                        xin[a] = f == 0 ? 0 : n - 1;
                        int64_t Pin = cell_at(g, xin);
                        if (bc == OR_BC_PERIODIC) {
                            int64_t xl[3] = {x[0], x[1], x[2]}, xr[3] = {x[0], x[1], x[2]};
                            xl[a] = n - 1; xr[a] = 0;
                            pl = p[cell_at(g, xl)]; pr_ = p[cell_at(g, xr)];
                        } else if (bc == OR_BC_OUTFLOW) {
                            if (s < 0) { pl = -p[Pin]; pr_ = p[Pin]; } else { pl = p[Pin]; pr_ = -p[Pin]; }
                        } else {
                            U[fi] = Ustar[fi];
                            continue;
                        }
                    }
                    U[fi] = Ustar[fi] - dt * (pr_ - pl) / dx;
                }
    }
}

int or_step(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
            int64_t nrec, const int64_t* cellrec, double* u, double* U, double* p, double* Hprev,
            int first_step, double tol, int32_t maxit, int32_t solver, double omega, or_stats* st) {
    const int64_t N = ncells(g);
    const int64_t NF = nfaces_axis(g, 0) + nfaces_axis(g, 1) + nfaces_axis(g, 2);
    double* nut = (double*)calloc((size_t)N, sizeof(double));
    double* H = (double*)malloc((size_t)(3 * N) * sizeof(double));
    double* us = (double*)malloc((size_t)(3 * N) * sizeof(double));
    double* us2 = (double*)malloc((size_t)(3 * N) * sizeof(double));
    double* Us = (double*)malloc((size_t)NF * sizeof(double));
    double* b = (double*)malloc((size_t)N * sizeof(double));
    if (pr->csm_on) or_csm(g, pr, flags, rec, cellrec, u, nut);
    st->mom_iters = 0;
    if (pr->integrator == OR_CRANK_NICOLSON) {
        st->mom_iters = or_predict_cn(g, pr, flags, rec, cellrec, u, U, nut, H, us, pr->mom_tol, pr->mom_maxit);
        if (st->mom_iters < 0) {
            free(nut); free(H); free(us); free(us2); free(Us); free(b);
            st->status = 4;
            return 4;
        }
    } else {
        or_predict(g, pr, flags, rec, cellrec, u, U, nut, Hprev, H, us, first_step);
    }
    memcpy(Hprev, H, (size_t)(3 * N) * sizeof(double));
    st->fsum[0] = st->fsum[1] = st->fsum[2] = 0.0;
    if (pr->forcing_on && nrec > 0) {
        or_forcing(g, pr, flags, rec, nrec, us, us2, st->fsum);
        memcpy(us, us2, (size_t)(3 * N) * sizeof(double));
    }
    or_faces(g, pr, flags, rec, cellrec, us, Us);
    or_rhs(g, pr, Us, b);
    int status = or_solve(g, pr, flags, b, p, tol, maxit, solver, omega, st);
    or_correct(g, pr, flags, us, Us, p, u, U);
    free(nut); free(H); free(us); free(us2); free(Us); free(b);
    return status;
}

/* ------------------------------------------------------------------------------------------------ */
/* Eq. force: per triangle, Shepard (inverse squared distance) averages of p over the cell centres of */
/* the 2x2x2 block around the centroid X, split into the front (n.(x - X) > 0) and back (< 0) sides.  */
/* Pressure pushes on the front side along -n and on the back side along +n.                         */

void or_forces(const or_grid* g, const float* tri, int64_t ntri, const double* p, double out[4]) {
    double F[3] = {0, 0, 0};
    int64_t used = 0;
    for (int64_t t = 0; t < ntri; ++t) {
        double A[3], B[3], C[3];
        if (!tri_load(tri + 9 * t, A, B, C)) continue;
        double e1[3], e2[3], n[3], X[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = B[d] - A[d];
            e2[d] = C[d] - A[d];
            X[d] = (A[d] + B[d] + C[d]) / 3.0;
        }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0.0)) continue;
        double area = 0.5 * len * g->dx * g->dx;
        for (int d = 0; d < 3; ++d) n[d] /= len;
        int64_t base[3];
        for (int d = 0; d < 3; ++d) base[d] = (int64_t)floor(X[d] - 0.5);
        double sw[2] = {0, 0}, sp[2] = {0, 0};
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    int64_t x[3] = {base[0] + di, base[1] + dj, base[2] + dk};
                    if (x[0] < 0 || x[1] < 0 || x[2] < 0 || x[0] >= g->nx || x[1] >= g->ny || x[2] >= g->nz)
                        continue;
                    double r[3], r2 = 0.0, sd = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        r[d] = ((double)x[d] + 0.5) - X[d];
                        r2 += r[d] * r[d];
                        sd += n[d] * r[d];
                    }
                    if (sd == 0.0) continue;
                    if (r2 < 1e-24) r2 = 1e-24;
                    double w = 1.0 / r2;
                    int side = sd > 0.0 ? 0 : 1;           /* 0 front, 1 back */
                    sw[side] += w;
                    sp[side] += w * p[cell_at(g, x)];
                }
        if (sw[0] == 0.0 || sw[1] == 0.0) continue;
        double pf = sp[0] / sw[0], pb = sp[1] / sw[1];
        for (int d = 0; d < 3; ++d) F[d] += area * (pb - pf) * n[d];
        ++used;
    }
    out[0] = F[0];
    out[1] = F[1];
    out[2] = F[2];
    out[3] = (double)used;
}

/* ------------------------------------------------------------------------------------------------ */
/* Surface pressure per triangle side (Eq. force) with the thin-plate filter Z (Eq. force_filter).    */
/* Reading of the garbled filter: a surrounding cell centre x^(k) takes part in the Shepard average    */
/* of surface node X only if X is the first surface that x^(k) sees towards X, i.e. the open segment  */
/* from X to x^(k) crosses no other triangle (then |X - x| + |x^(k) - X^(k)| is one link length with  */
/* X^(k) = X).  Points behind a second surface closer than a cell -- the inner faces of a plate       */
/* thinner than dx, a duplicated skin -- are cancelled.  Each side is averaged on its own; a side     */
/* left without points has no value (NaN) and adds nothing to the force.                            */

/* orient3d(a, b, c, d) = det[b - a; c - a; d - a], each product and sum rounded once, in this order. */
static double orient3(const double a[3], const double b[3], const double c[3], const double d[3]) {
    double u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
    double v0 = c[0] - a[0], v1 = c[1] - a[1], v2 = c[2] - a[2];
    double w0 = d[0] - a[0], w1 = d[1] - a[1], w2 = d[2] - a[2];
    double m0 = v1 * w2 - v2 * w1;
    double m1 = v0 * w2 - v2 * w0;
    double m2 = v0 * w1 - v1 * w0;
    return (u0 * m0 - u1 * m1) + u2 * m2;
}

/* The open segment X-Y crosses triangle ABC: X and Y strictly on opposite sides of its plane and the */
/* line through them inside or on the triangle's edges. */
static int segment_crosses(const double X[3], const double Y[3], const double A[3], const double B[3],
                           const double C[3]) {
    double o1 = orient3(A, B, C, X), o2 = orient3(A, B, C, Y);
    if (!((o1 > 0.0 && o2 < 0.0) || (o1 < 0.0 && o2 > 0.0))) return 0;
    double e0 = orient3(X, Y, A, B), e1 = orient3(X, Y, B, C), e2 = orient3(X, Y, C, A);
    return (e0 >= 0.0 && e1 >= 0.0 && e2 >= 0.0) || (e0 <= 0.0 && e1 <= 0.0 && e2 <= 0.0);
}

void or_surface_pressure(const or_grid* g, const float* tri, int64_t ntri, const double* p, int zfilter,
                         double* pside, double out[4]) {
    double F[3] = {0, 0, 0};
    int64_t sides = 0;
    for (int64_t t = 0; t < ntri; ++t) {
        pside[2 * t] = NAN;
        pside[2 * t + 1] = NAN;
        double A[3], B[3], C[3];
        if (!tri_load(tri + 9 * t, A, B, C)) continue;
        double e1[3], e2[3], n[3], X[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = B[d] - A[d];
            e2[d] = C[d] - A[d];
            X[d] = (A[d] + B[d] + C[d]) / 3.0;
        }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0.0)) continue;
        double area = 0.5 * len * g->dx * g->dx;
        for (int d = 0; d < 3; ++d) n[d] /= len;
        int64_t base[3];
        for (int d = 0; d < 3; ++d) base[d] = (int64_t)floor(X[d] - 0.5);
        double sw[2] = {0, 0}, sp[2] = {0, 0};
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    int64_t x[3] = {base[0] + di, base[1] + dj, base[2] + dk};
                    if (x[0] < 0 || x[1] < 0 || x[2] < 0 || x[0] >= g->nx || x[1] >= g->ny || x[2] >= g->nz)
                        continue;
                    double Y[3], r2 = 0.0, sd = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        Y[d] = (double)x[d] + 0.5;
                        double r = Y[d] - X[d];
                        r2 += r * r;
                        sd += n[d] * r;
                    }
                    if (sd == 0.0) continue;
                    if (zfilter) {
                        int hidden = 0;
                        for (int64_t o = 0; o < ntri && !hidden; ++o) {
                            if (o == t) continue;
                            double P0[3], P1[3], P2[3];
                            if (!tri_load(tri + 9 * o, P0, P1, P2)) continue;
                            /* a triangle whose bounding box misses the segment's cannot cross it */
                            int apart = 0;
                            for (int d = 0; d < 3; ++d) {
                                double smn = fmin(X[d], Y[d]), smx = fmax(X[d], Y[d]);
                                double tmn = fmin(fmin(P0[d], P1[d]), P2[d]), tmx = fmax(fmax(P0[d], P1[d]), P2[d]);
                                if (tmx < smn || tmn > smx) apart = 1;
                            }
                            if (!apart) hidden = segment_crosses(X, Y, P0, P1, P2);
                        }
                        if (hidden) continue;
                    }
                    if (r2 < 1e-24) r2 = 1e-24;
                    double w = 1.0 / r2;
                    int side = sd > 0.0 ? 0 : 1;           /* 0 front, 1 back */
                    sw[side] += w;
                    sp[side] += w * p[cell_at(g, x)];
                }
        for (int sd = 0; sd < 2; ++sd) {
            if (sw[sd] == 0.0) continue;
            double ps = sp[sd] / sw[sd];
            pside[2 * t + sd] = ps;
            /* pressure pushes on the front side along -n, on the back side along +n */
            for (int d = 0; d < 3; ++d) F[d] += (sd == 0 ? -1.0 : 1.0) * area * ps * n[d];
            ++sides;
        }
    }
    out[0] = F[0];
    out[1] = F[1];
    out[2] = F[2];
    out[3] = (double)sides;
}

/* Viscous force on the body (reading; the paper integrates pressure only): the molecular diffusive
 * momentum flux through every cut link, nu (u_P - u_G) / dx times the face area dx^2, with u_G the
 * ghost value of Eq. q_axis -- exactly the flux the momentum equation exchanges with the wall there
 * -- signed as a force on the body.  out[0..2] = force, out[3] = links used. */
void or_viscous_force(const or_grid* g, const or_params* pr, const uint8_t* flags, const or_record* rec,
                      int64_t nrec, const int64_t* cellrec, const double* u, double out[4]) {
    const int64_t N = ncells(g);
    double F[3] = {0, 0, 0};
    for (int64_t q = 0; q < nrec; ++q) {
        const or_record* R = &rec[q];
        const int64_t P = R->cell;
        for (int c = 0; c < 3; ++c) {
            double uG = or_velocity_across(g, pr, flags, rec, cellrec, u, c, P, (int)R->axis, (int)R->side);
            F[c] += pr->nu * (u[c * N + P] - uG) * g->dx;
        }
    }
    out[0] = F[0];
    out[1] = F[1];
    out[2] = F[2];
    out[3] = (double)nrec;
}

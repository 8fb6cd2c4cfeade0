"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: brute-force geometry, closed-form
eigenpairs, exactness on linear fields, conservation identities, printed constants, or the observed
convergence order against the analytic Taylor-Green vortex.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
PER = (0, 0, 0, 0, 0, 0)
SLIPBOX = (3, 3, 3, 3, 3, 3)


def centres(n):
    return np.arange(n) + 0.5


# --------------------------------------------------------------------------------------------------
# Classification (Sec. 2.4.1)

def _links_expected_box(nx, ny, nz, lo, hi):
    """Brute force for an axis-aligned box: a link is cut iff exactly one of its two centres lies
    inside; t is the crossing's position on the centre-to-centre segment."""
    exp = {}
    N = nx * ny * nz
    dims = (nx, ny, nz)
    for a in range(3):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    x = [i, j, k]
                    if x[a] + 1 >= dims[a]:
                        continue
                    y = list(x)
                    y[a] += 1
                    cP = np.array(x) + 0.5
                    cN = np.array(y) + 0.5
                    inP = np.all((cP > lo) & (cP < hi))
                    inN = np.all((cN > lo) & (cN < hi))
                    b, c = (a + 1) % 3, (a + 2) % 3
                    inside_trans = lo[b] < cP[b] < hi[b] and lo[c] < cP[c] < hi[c]
                    ts = []
                    if inside_trans:
                        for plane in (lo[a], hi[a]):
                            t = plane - cP[a]
                            if 0.0 <= t < 1.0:
                                ts.append(t)
                    assert (inP != inN) == (len(ts) % 2 == 1)
                    if ts:
                        exp[a * N + (i + nx * (j + ny * k))] = (min(ts), max(ts))
    return exp


@pytest.mark.parametrize("m", [1, 3])
def test_classify_box_matches_brute_force(m):
    nx, ny, nz = 12, 10, 9
    lo = np.array([2.3, 1.7, 2.9], np.float32).astype(np.float64)
    hi = np.array([8.6, 7.2, 6.05], np.float32).astype(np.float64)
    tri = W.axis_box(lo, hi, m)
    case = oracle.Case(nx, ny, nz)
    fid, tlo, thi = case.classify(tri)
    exp = _links_expected_box(nx, ny, nz, lo, hi)
    assert sorted(exp) == list(fid)
    for f, a, b in zip(fid, tlo, thi):
        assert abs(a - exp[f][0]) < 1e-12 and abs(b - exp[f][1]) < 1e-12
    # flag bits are the two ends of every cut face
    N = nx * ny * nz
    fl = np.zeros(N, np.uint8)
    for f in fid:
        a, c = divmod(int(f), N)
        st = (1, nx, nx * ny)[a]
        fl[c] |= 1 << (2 * a + 1)
        fl[c + st] |= 1 << (2 * a)
    assert np.array_equal(fl, case.flags)


def test_classify_convex_icosphere_halfspace():
    """Convex closed soup: cut(link) <=> inside(P) != inside(N) by half-space tests, and t_lo/t_hi are
    the entry/exit parameters of the segment through the polytope."""
    n = 16
    tri = W.icosphere(2, 5.3, (8.3, 7.9, 8.1)).astype(np.float64)
    A, B, Cv = tri[:, 0], tri[:, 1], tri[:, 2]
    nrm = np.cross(B - A, Cv - A)
    outward = np.einsum("ij,ij->i", nrm, A - np.array([8.3, 7.9, 8.1])) > 0
    nrm[~outward] *= -1
    off = np.einsum("ij,ij->i", nrm, A)
    case = oracle.Case(n, n, n)
    fid, tlo, thi = case.classify(tri.astype(np.float32))
    got = {int(f): (a, b) for f, a, b in zip(fid, tlo, thi)}
    N = n ** 3
    checked = 0
    for a in range(3):
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    x = [i, j, k]
                    if x[a] == n - 1:
                        continue
                    P = np.array(x) + 0.5
                    fidx = a * N + (i + n * (j + n * k))
                    dn = nrm[:, a]
                    v0 = P @ nrm.T - off              # < 0 on the inner side of every face plane
                    if np.any(np.abs(v0) < 1e-7) or np.any(np.abs(v0 + dn) < 1e-7):
                        continue                      # a centre on a face plane: ambiguous, skip
                    checked += 1
                    # slab method: the segment P + t e_a, t in [0, 1), is inside where all v < 0
                    with np.errstate(divide="ignore", invalid="ignore"):
                        tc = -v0 / dn
                    par = dn == 0
                    if np.any(par & (v0 >= 0)):
                        t_in, t_out = np.inf, -np.inf  # parallel to and outside some face
                    else:
                        t_in = np.max(np.where(dn < 0, tc, -np.inf))
                        t_out = np.min(np.where(dn > 0, tc, np.inf))
                    ts = [t for t in (t_in, t_out) if t_in < t_out and 0.0 <= t < 1.0]
                    assert (fidx in got) == bool(ts), (a, x, ts)
                    p_in = bool(np.all(v0 < 0))
                    n_in = bool(np.all(v0 + dn < 0))
                    if len(ts) == 1:
                        assert p_in != n_in
                    if ts:
                        assert abs(got[fidx][0] - min(ts)) < 1e-9
                        assert abs(got[fidx][1] - max(ts)) < 1e-9
    assert checked > 3 * 14 * 16 * 16 * 0.9


def test_classify_matches_moller_trumbore_on_random_soup():
    tri = W.random_soup(3000, (0, 0, 0), (20, 16, 12), 4.0, seed=11)
    case = oracle.Case(20, 16, 12)
    assert case.mt_disagreements(tri) == 0


def test_classify_skips_nonfinite_and_outside():
    tri = W.random_soup(50, (0, 0, 0), (8, 8, 8), 3.0, seed=5)
    bad = tri.copy()
    bad[3, 1, 2] = np.nan
    bad[7, 0, 0] = np.inf
    far = (tri + 1000.0).astype(np.float32)
    case = oracle.Case(8, 8, 8)
    case.classify(np.concatenate([bad, far]))
    assert case.n_skipped == 2
    ref = oracle.Case(8, 8, 8)
    keep = np.ones(50, bool); keep[[3, 7]] = False
    ref.classify(tri[keep])
    assert np.array_equal(case.cut[0], ref.cut[0]) and np.array_equal(case.flags, ref.flags)


def test_coplanar_triangle_gives_no_hit():
    # triangle in the plane y = 2.5 contains grid lines along x and z: W = 0 for them
    tri = np.array([[[0.2, 2.5, 0.3], [7.1, 2.5, 0.4], [0.5, 2.5, 6.6]]], np.float32)
    case = oracle.Case(8, 8, 8)
    fid, _, _ = case.classify(tri)
    assert all(int(f) // 512 == 1 for f in fid)   # only y-links can be cut


# --------------------------------------------------------------------------------------------------
# Ghost values (Eq. q_axis), distribution function (Eq. distribution_function)

def _wall_case(x0, n=12, extra=None):
    """A full plane wall x = x0 across a slip box, optionally a second wall."""
    walls = [x0] + ([] if extra is None else [extra])
    tri = []
    for xw in walls:
        tri.append([[xw, -1.0, -1.0], [xw, 3 * n, -1.0], [xw, -1.0, 3 * n]])
    case = oracle.Case(n, 6, 5, bc=SLIPBOX)
    case.set_geometry(np.array(tri, np.float32))
    return case


@pytest.mark.parametrize("x0", [5.03, 5.2, 5.49, 5.5, 5.51, 5.77, 5.97])
def test_ghost_exact_for_linear_field(x0):
    """For q = beta (x - x0) the wall value is 0 and the ghost must equal the linear extrapolant q(x_N)
    on both sides of the wall (upper and lower branch)."""
    x0 = float(np.float32(x0))
    case = _wall_case(x0)
    nx, ny, nz = 12, 6, 5
    xc = np.arange(nx) + 0.5
    q = np.broadcast_to(0.7 * (xc - x0), (nz, ny, nx))
    u = np.stack([q, 2 * q, -q]).reshape(-1)
    f = int(np.floor(x0 - 0.5))
    for comp, scale in ((0, 0.7), (1, 1.4), (2, -0.7)):
        for (i, side) in ((f, +1), (f + 1, -1)):
            P = i + nx * (2 + ny * 3)
            g = case.velocity_across(u, comp, P, 0, side)
            assert g == pytest.approx(scale * (xc[i] + side - x0), abs=1e-12)
    br = set(case.rec["branch"].tolist())
    assert br <= {0, 1}


def test_ghost_branch_c_when_opposite_is_blocked():
    # cell 4 (centre 4.5): +x wall at 4.9 (d = 0.4 < 0.5) and a -x wall at 4.2, so the opposite
    # neighbour O = cell 3 is behind a wall and the lower branch cannot be used -> branch C
    case = _wall_case(float(np.float32(4.9)), extra=float(np.float32(4.2)))
    r = case.rec
    sel = (r["cell"] % 12 == 4) & (r["side"] == 1)
    assert sel.sum() == 30 and np.all(r["branch"][sel] == 2) and np.all(r["opp"][sel] == -1)
    # branch C is the upper branch evaluated at d = 1/2: ghost = 2 q_IB - q_P
    assert np.all(r["c_ib"][sel] == 2.0) and np.all(r["c_p"][sel] == -1.0)
    assert np.all(r["c_o"][sel] == 0.0)


def test_distribution_weights_match_printed_values():
    gold = GOLD["distribution_function_samples"]
    for d, wf, wg in zip(gold["d"][1:], gold["fluid_side"][1:], gold["ghost_side"][1:]):
        case = _wall_case(float(np.float32(5.5 + d)))
        r = case.rec
        sel = (r["side"] == 1)
        assert np.allclose(r["d"][sel], d, atol=1e-6)
        assert np.allclose(r["w_fluid"][sel], wf, atol=1e-6)
        assert np.allclose(r["w_ghost"][sel], wg, atol=1e-6)
        assert np.allclose(r["w_fluid"] + r["w_ghost"], 1.0 / (1.0 + r["d"]), rtol=1e-14)


def test_setup_regions_and_deadend_bits():
    case = oracle.Case(10, 10, 10)
    case.set_geometry(W.axis_box((3.2, 3.3, 3.4), (6.6, 6.7, 6.8), 1))
    fl = case.flags
    inc = (fl & 63) != 0
    assert np.array_equal(inc, (fl & 64) != 0)
    adj = (fl & 128) != 0
    assert not np.any(adj & inc)
    # every Omega_adj cell touches an Omega_inc cell and vice versa every neighbour of inc is inc|adj
    F = fl.reshape(10, 10, 10)
    I = (F & 64) != 0
    A = (F & 128) != 0
    nb = np.zeros_like(I)
    for ax in range(3):
        for s in (-1, 1):
            sh = np.roll(I, s, axis=ax)
            edge = [slice(None)] * 3
            edge[ax] = 0 if s == 1 else -1
            sh[tuple(edge)] = False
            nb |= sh
    assert np.array_equal(A, nb & ~I)
    assert len(case.rec) == 2 * len(case.cut[0])


# --------------------------------------------------------------------------------------------------
# CSM (Sec. 2.3)

def _interior(nx, ny, nz):
    m = np.zeros((nz, ny, nx), bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m.reshape(-1)


def _linear_field(n, G):
    """u_b = sum_a G[a][b] x_a sampled at cell centres (G[a][b] = du_b/dx_a)."""
    x = centres(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    pos = [X, Y, Z]
    return np.stack([sum(G[a][b] * pos[a] for a in range(3)) for b in range(3)]).reshape(-1)


def test_csm_closed_forms():
    n = 7
    case = oracle.Case(n, n, n, bc=SLIPBOX)
    m = _interior(n, n, n)
    rot = [[0, 1, 0], [-1, 0, 0], [0, 0, 0]]          # u = (-y, x, 0): rigid rotation
    assert np.all(case.csm(_linear_field(n, rot))[m] == 0.0)
    strain = [[1, 0, 0], [0, -1, 0], [0, 0, 0]]       # u = (x, -y, 0): F_CS = -1, C = C1
    nut = case.csm(_linear_field(n, strain))[m]
    assert np.allclose(nut, GOLD["csm_C1"]["value"] * np.sqrt(2.0), rtol=1e-14)
    shear = [[0, 0, 0], [1, 0, 0], [0, 0, 0]]         # u = (y, 0, 0): Q = 0
    assert np.allclose(case.csm(_linear_field(n, shear))[m], 0.0, atol=1e-16)
    # |F_CS| <= 1 bounds nu_t <= C1 dx^2 |S|
    rng = np.random.default_rng(0)
    u = rng.standard_normal(3 * n ** 3)
    nut = case.csm(u)
    assert np.all(nut >= 0.0)
    case2 = oracle.Case(n, n, n, dx=0.5, bc=SLIPBOX)
    nut2 = case2.csm(u)
    assert np.allclose(nut2, nut * 0.25 / 0.5, rtol=1e-12)   # nu_t ~ dx^2 * |S| ~ dx^2 / dx


def test_csm_random_gradient_bound():
    n = 5
    case = oracle.Case(n, n, n, bc=SLIPBOX)
    m = _interior(n, n, n)
    rng = np.random.default_rng(3)
    for _ in range(20):
        G = rng.standard_normal((3, 3))
        nut = case.csm(_linear_field(n, G))[m]
        S = 0.5 * (G + G.T)
        Wt = 0.5 * (G - G.T)
        SS, WW = np.sum(S * S), np.sum(Wt * Wt)
        F = (WW - SS) / (WW + SS)
        assert abs(F) <= 1.0
        assert np.allclose(nut, 0.05 * abs(F) ** 1.5 * np.sqrt(SS), rtol=1e-12)


# --------------------------------------------------------------------------------------------------
# Predictor (Sec. 2.1): conservation and consistency

def test_predictor_conserves_momentum_periodic():
    n = 8
    rng = np.random.default_rng(1)
    case = oracle.Case(n, n, n, nu=0.05, dt=0.1, bc=PER)
    u = rng.standard_normal(3 * n ** 3)
    U = case.faces(u)
    nut = case.csm(u)
    H, _ = case.predict(u, U, nut, np.zeros_like(u), True)
    Hs = H.reshape(3, -1).sum(1)
    assert np.all(np.abs(Hs) < 1e-11 * np.abs(H).sum())


_UIN = np.array([0.8, -0.3, 0.2])
_BC_FIELDS = {
    # face tested, boundary conditions, a linear field satisfying that face's condition, normal axis
    "inflow": ((1, 2, 0, 0, 0, 0), lambda x: _UIN[:, None] + np.outer([0.3, -0.2, 0.45], x[:, 0]), 0),
    "noslip": ((0, 0, 0, 0, 4, 3), lambda x: np.outer([0.3, -0.2, 0.45], x[:, 2]), 2),
    "slip": ((0, 0, 3, 3, 0, 0),
             lambda x: np.stack([np.full(len(x), 0.7), 0.35 * x[:, 1], np.full(len(x), -0.4)]), 1),
}


@pytest.mark.parametrize("face", sorted(_BC_FIELDS))
def test_boundary_ghosts_are_exact_for_linear_fields(face):
    """The outer boundary ghosts (reading; the paper omits them) are linear extrapolations.  They are
    2 u_in - u_P at the inflow, -u_P at a no-slip wall, and at a slip wall the normal component
    mirrored and the tangential ones copied.  So the viscous operator of a linear field that meets the
    face's condition (Dirichlet value u_in at the inflow face, zero at the no-slip face, zero normal
    component and no normal variation of the tangential ones at a slip face) vanishes in the cells
    next to that face.  A plain u_in ghost at the inflow, swapped slip parities or a copied no-slip
    ghost each leave 0.01-0.07 there."""
    bc, field, ax = _BC_FIELDS[face]
    n = (10, 9, 8)
    N = n[0] * n[1] * n[2]
    xc = np.stack([np.arange(N) % n[0], (np.arange(N) // n[0]) % n[1], np.arange(N) // (n[0] * n[1])], 1) + 0.5
    case = oracle.Case(*n, nu=0.05, dt=0.2, bc=bc, u_in=tuple(_UIN), csm_on=0)
    u = field(xc).reshape(-1).copy()
    L = case.momentum_operator(u, np.zeros(case.NF), np.zeros(N)).reshape(3, -1)
    near = xc[:, ax] < n[ax] - 2        # away from the opposite face, whose condition the field breaks
    assert np.abs(L[:, near]).max() < 1e-14
    assert np.abs(L).max() > 1e-3       # the opposite face does see the field (the check is not empty)


def _x_invariant_field(n):
    """A velocity that does not vary along x: smooth periodic modes in y and z."""
    N = n[0] * n[1] * n[2]
    xc = np.stack([np.arange(N) % n[0], (np.arange(N) // n[0]) % n[1], np.arange(N) // (n[0] * n[1])], 1) + 0.5
    ty, tz = 2 * np.pi * xc[:, 1] / n[1], 2 * np.pi * xc[:, 2] / n[2]
    u = np.stack([0.7 + 0.2 * np.sin(ty) + 0.1 * np.cos(tz), -0.3 + 0.15 * np.cos(ty) * np.sin(tz),
                  0.4 + 0.25 * np.sin(tz) - 0.1 * np.cos(2 * ty)])
    return xc, u.reshape(-1).copy()


@pytest.mark.parametrize("xplus,expect_exact", [(2, True), (1, False), (3, False), (4, False)])
def test_outflow_ghost_is_a_zero_normal_gradient(xplus, expect_exact):
    """Reading of the outflow face (the paper leaves the outer boundaries out, Sec. 2.1): the velocity
    ghost across it is the near cell's own value, so the face imposes a zero normal gradient.  For a
    field that does not vary along x, the momentum operator (diffusion plus the transpose SGS term
    with a uniform nu_t; no advection) must then be the same in the cells next to the x+ face as in
    interior cells with the same (y, z), because a zero-gradient face adds no flux.  The same field
    with the x+ face read instead as an inflow (ghost 2 u_in - u_P), a slip wall (normal component
    mirrored) or a no-slip wall (ghost -u_P) differs there by more than 1e-3, so the check tells the
    outflow ghost apart from every other ghost the oracle has."""
    n = (12, 10, 8)
    xc, u = _x_invariant_field(n)
    bc = (1, xplus, 0, 0, 0, 0)
    case = oracle.Case(*n, nu=0.05, dt=0.2, bc=bc, u_in=(0.8, -0.3, 0.2), csm_on=0)
    N = case.N
    L = case.momentum_operator(u, np.zeros(case.NF), np.full(N, 0.07)).reshape(3, n[2], n[1], n[0])
    edge, mid = L[:, :, :, n[0] - 1], L[:, :, :, n[0] // 2]
    scale = np.abs(mid).max()
    assert scale > 1e-3                        # the field has a nonzero operator (the check is not empty)
    gap = np.abs(edge - mid).max()
    if expect_exact:
        assert gap <= 1e-14 * max(scale, 1.0)
        # and the interior column is x-invariant as well (the inflow face is two cells away from it)
        assert np.abs(L[:, :, :, 2:] - mid[..., None]).max() <= 1e-14 * max(scale, 1.0)
    else:
        assert gap > 1e-3


def test_viscous_and_sgs_stress_of_a_linear_field_vanish_at_a_wall():
    """Sec. 2.1 / Eq. SGSstress: for a linear velocity u = c + A x with constant nu and nu_t the stress
    divergence div(nu grad u + nu_t (grad u + grad u^T)) is zero.  With the face velocities set to zero
    (no advection) and u_IB = u(X) on every record, the momentum operator must vanish in every cell
    whose stencil stays inside the box, the cells next to an oblique wall included.  There the ghost
    values of Eq. q_axis are exact for linear fields, and the transpose term on a cut face takes the
    cell's own gradient (reading).  Dropping that term, or flipping its sign, leaves 0.04-0.08."""
    n = (14, 12, 10)
    case = oracle.Case(*n, nu=0.05, dt=0.2, bc=SLIPBOX)
    lo, hi = -20.0, 40.0
    case.set_geometry(np.array([[[5.3, lo, lo], [9.9, hi, lo], [4.1, lo, hi]],
                                [[4.1, lo, hi], [9.9, hi, lo], [8.7, hi, hi]]], np.float32))
    A = np.array([[0.3, 0.5, -0.2], [0.1, -0.1, 0.4], [0.25, -0.3, -0.2]])
    c0 = np.array([0.4, -0.2, 0.1])
    N = case.N
    xc = np.stack([np.arange(N) % n[0], (np.arange(N) // n[0]) % n[1], np.arange(N) // (n[0] * n[1])], 1) + 0.5
    u = (c0[None, :] + xc @ A.T).T.reshape(-1).copy()
    case.rec["uib"][:] = c0[None, :] + record_points(case) @ A.T
    assert np.all(case.rec["branch"] < 2) and len(set(case.rec["axis"])) == 3
    L = case.momentum_operator(u, np.zeros(case.NF), np.full(N, 0.07)).reshape(3, -1)
    inner = np.all((xc > 3) & (xc < np.array(n) - 3), axis=1)
    near = inner & ((case.flags & 63) != 0)
    assert near.sum() >= 40
    assert np.abs(L[:, inner]).max() < 1e-13


def test_predictor_uniform_flow_is_steady():
    n = 6
    case = oracle.Case(n, n, n, nu=0.05, dt=0.1, bc=PER)
    u = np.concatenate([np.full(n ** 3, 0.3), np.full(n ** 3, -0.2), np.full(n ** 3, 0.1)])
    H, us = case.predict(u, case.faces(u), case.csm(u), np.zeros_like(u), True)
    assert np.all(H == 0.0) and np.array_equal(us, u)


def test_predictor_diffusion_of_a_sine_mode():
    """Pure diffusion (U = 0, nu_t = 0) of u_x = sin(2 pi y / n) in a periodic box: the discrete
    Laplacian eigenvalue -(2 - 2 cos(2 pi / n)) nu / dx^2 is exact."""
    n = 16
    case = oracle.Case(n, n, 4, nu=0.3, dt=0.1, bc=PER, csm_on=0)
    y = centres(n)
    ux = np.broadcast_to(np.sin(2 * np.pi * y / n)[None, :, None], (4, n, n))
    u = np.stack([ux, 0 * ux, 0 * ux]).reshape(-1)
    H, _ = case.predict(u, np.zeros(case.NF), np.zeros(case.N), np.zeros_like(u), True)
    lam = -(2 - 2 * np.cos(2 * np.pi / n)) * 0.3
    assert np.allclose(H[:case.N], lam * u[:case.N], atol=1e-14)
    assert np.all(H[case.N:] == 0)


# --------------------------------------------------------------------------------------------------
# Poisson operator and solvers (Eq. poisson)

def _mode(n, kind, k):
    i = centres(n) - 0.5 + 0.5  # (i + 1/2)
    if kind == "per":
        th = 2 * np.pi * k / n
        return np.cos(th * i), -(2 - 2 * np.cos(th))
    if kind == "neu":
        th = np.pi * k / n
        return np.cos(th * i), -(2 - 2 * np.cos(th))
    th = np.pi * (k + 0.5) / n      # Neumann at the low face, p = 0 at the high face
    return np.cos(th * i), -(2 - 2 * np.cos(th))


@pytest.mark.parametrize("bcx,kind", [(0, "per"), (3, "neu"), (2, "dir")])
def test_poisson_operator_eigenpairs(bcx, kind):
    nx, ny, nz = 12, 8, 6
    dx = 0.7
    bc = [bcx, bcx, 3, 3, 0, 0]
    if kind == "dir":
        bc[0] = 1
    case = oracle.Case(nx, ny, nz, dx=dx, bc=tuple(bc))
    mx, lx = _mode(nx, kind, 3)
    my, ly = _mode(ny, "neu", 2)
    mz, lz = _mode(nz, "per", 1)
    p = (mz[:, None, None] * my[None, :, None] * mx[None, None, :]).reshape(-1)
    Ap = case.apply(p)
    lam = (lx + ly + lz) / dx ** 2
    assert np.allclose(Ap, lam * p, atol=1e-12 * np.abs(lam))


def test_poisson_operator_decouples_at_a_cut_wall():
    nx = 10
    case = _wall_case(float(np.float32(4.3)), n=nx)   # cuts the x-link between cells 3 and 4
    # on cells 0..3 the wall is a Neumann face: cos modes of the 4-cell block are eigenvectors
    th = np.pi * 1 / 4
    blk = np.cos(th * (centres(4)))
    p = np.zeros((5, 6, nx))
    p[:, :, :4] = blk
    Ap = case.apply(p.reshape(-1)).reshape(5, 6, nx)
    lam = -(2 - 2 * np.cos(th))
    assert np.allclose(Ap[:, :, :4], lam * p[:, :, :4], atol=1e-13)
    assert np.allclose(Ap[:, :, 4:], 0.0)


@pytest.mark.parametrize("solver", [oracle.BICGSTAB, oracle.CG, oracle.RBSOR])
def test_poisson_solve_recovers_eigenmode(solver):
    nx, ny, nz = 16, 8, 8
    case = oracle.Case(nx, ny, nz, bc=(1, 2, 3, 3, 3, 3))
    mx, lx = _mode(nx, "dir", 1)
    my, ly = _mode(ny, "neu", 1)
    phi = (np.ones(nz)[:, None, None] * my[None, :, None] * mx[None, None, :]).reshape(-1)
    lam = lx + ly
    omega = 1.0 if solver != oracle.RBSOR else 1.7
    p, st = case.solve(phi, tol=1e-11, solver=solver, omega=omega, maxit=20000)
    assert st.status == 0 and st.relres <= 1e-11
    assert np.allclose(p, phi / lam, atol=1e-9 * np.abs(phi / lam).max())


def test_poisson_solution_converges_at_second_order_through_the_boundaries():
    """Eq. poisson against a smooth manufactured pressure that is no eigenfunction of the operator:
    p = cos(pi x / 2)(1 + x^2) (1 + 0.3 cos(pi y / L_y)) on x in [0, 1].  The inflow face x = 0 is
    Neumann, the outflow face x = 1 holds p = 0, and the slip walls in y and z are Neumann.  With
    b = laplacian(p) at the cell centres the discrete solution must approach p at second order."""
    a = np.pi / 2
    errs = []
    for n in (16, 32, 64):
        dx = 1.0 / n
        nx, ny, nz = n, n // 2, 2
        ly = ny * dx
        case = oracle.Case(nx, ny, nz, dx, bc=(1, 2, 3, 3, 3, 3))
        x = np.broadcast_to(((np.arange(nx) + 0.5) * dx)[None, None, :], (nz, ny, nx)).reshape(-1)
        y = np.broadcast_to(((np.arange(ny) + 0.5) * dx)[None, :, None], (nz, ny, nx)).reshape(-1)
        f = np.cos(a * x) * (1 + x * x)
        fxx = -a * a * np.cos(a * x) * (1 + x * x) - 4 * a * x * np.sin(a * x) + 2 * np.cos(a * x)
        gy = 1 + 0.3 * np.cos(np.pi * y / ly)
        gyy = -0.3 * (np.pi / ly) ** 2 * np.cos(np.pi * y / ly)
        p, st = case.solve(fxx * gy + f * gyy, tol=1e-13, maxit=20000)
        assert st.status == 0
        errs.append(np.abs(p - f * gy).max())
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 2.0) < 0.1), (errs, slopes)


# --------------------------------------------------------------------------------------------------
# Whole step: projection identity, mass balance, momentum, Taylor-Green convergence

def _pieces(case, state, tol=1e-12):
    u, U = state["u"], state["U"]
    nut = case.csm(u)
    H, us = case.predict(u, U, nut, state["H"], state["n"] == 0)
    us2, _ = case.forcing(us)
    Us = case.faces(us2)
    b = case.rhs(Us)
    p, st = case.solve(b, state["p"], tol=tol)
    un, Un = case.correct(us2, Us, p)
    return dict(us=us2, Us=Us, b=b, p=p, u=un, U=Un, st=st)


def _div_faces(U, nx, ny, nz, dx):
    Ux, Uy, Uz = oracle.split_faces(U, nx, ny, nz)
    return (np.diff(Ux, axis=2) + np.diff(Uy, axis=1) + np.diff(Uz, axis=0)).reshape(-1) / dx


def test_projection_identity_and_mass_balance():
    cfg = W.get_config("sphere_64x32x32")
    case = oracle.Case(32, 16, 16, 1.0, cfg.nu, cfg.dt, cfg.bc)
    case.set_geometry(W.icosphere(2, 3.1, (10.2, 8.1, 7.9)))
    state = case.initial_state(W.initial_fields(W.Config("t", 32, 16, 16, 0, 0, 0, 0, 0, cfg.bc,
                                                         seed=7)))
    r = _pieces(case, state, tol=1e-6)
    div = _div_faces(r["U"], 32, 16, 16, 1.0)
    res = r["b"] - case.apply(r["p"])
    assert np.allclose(div, cfg.dt * res, atol=1e-12 * np.abs(r["b"]).max() * cfg.dt)
    Ux, Uy, Uz = oracle.split_faces(r["Us"], 32, 16, 16)
    assert abs(Ux[:, :, 0].sum() - Ux[:, :, -1].sum()) < 1e-12 * Ux[:, :, 0].size
    assert np.all(Uy[:, 0] == 0) and np.all(Uy[:, -1] == 0)
    # the cut faces of a stationary wall carry no flux
    fid = case.cut[0]
    N = case.N
    for f in fid[:50]:
        a, c = divmod(int(f), N)
        k, rem = divmod(c, 32 * 16)
        j, i = divmod(rem, 32)
        face = (Ux[k, j, i + 1], Uy[k, j + 1, i], Uz[k + 1, j, i])[a]
        assert face == 0.0


def record_points(case, dx=1.0, lo=0.0):
    """Physical position X of each link record's wall point: the cell centre moved by d along the
    record's axis towards its side."""
    r = case.rec
    P = r["cell"]
    X = np.stack([P % case.nx, (P // case.nx) % case.ny, P // (case.nx * case.ny)], 1) + 0.5
    X[np.arange(len(r)), r["axis"]] += r["side"] * r["d"]
    return lo + X * dx


@pytest.mark.parametrize("integrator", [0, 1])
def test_wall_moving_with_a_uniform_flow_is_invisible(integrator):
    """A wall carried along by a uniform flow (u_IB = u everywhere) must leave the flow exactly uniform:
    every ghost of Eq. q_axis reproduces a constant, the forcing sees u*_X = u_IB, and the cut faces
    pass the wall's own normal velocity, so b = 0 and p stays uniform.  Blocking the cut faces instead
    would stop the flow at the wall."""
    n = (12, 10, 8)
    case = oracle.Case(*n, nu=0.05, dt=0.2, bc=PER, quick=0.1, integrator=integrator)
    lo, hi = -20.0, 40.0
    case.set_geometry(np.array([[[3.3, lo, lo], [11.9, hi, lo], [2.6, lo, hi]],
                                [[2.6, lo, hi], [11.9, hi, lo], [10.8, hi, hi]]], np.float32))
    assert len(case.rec) > 0 and len(set(case.rec["axis"])) == 3
    v = np.array([0.7, -0.2, 0.3])
    case.rec["uib"][:] = v
    u0 = np.broadcast_to(v[:, None], (3, case.N)).copy()
    st = case.initial_state(u0)
    for _ in range(3):
        s = case.step(st, tol=1e-12)
        assert s.status == 0
    assert np.abs(st["u"].reshape(3, -1) - v[:, None]).max() < 1e-12
    assert np.abs(st["p"] - st["p"].mean()).max() < 1e-10
    Ux, Uy, Uz = oracle.split_faces(st["U"], *n)
    assert np.allclose(Ux, v[0], atol=1e-12) and np.allclose(Uy, v[1], atol=1e-12) and np.allclose(Uz, v[2], atol=1e-12)


def test_step_conserves_momentum_periodic():
    n = 12
    u0, _, dx = W.taylor_green(n, 0.0, 100.0, nz=2)
    rng = np.random.default_rng(2)
    u0 = u0 + 0.05 * rng.standard_normal(u0.shape)
    case = oracle.Case(n, n, 2, dx, 0.01, 0.01, PER)
    st = case.initial_state(u0)
    m0 = st["u"].reshape(3, -1).sum(1)
    for _ in range(3):
        case.step(st, tol=1e-12)
    m1 = st["u"].reshape(3, -1).sum(1)
    assert np.allclose(m0, m1, atol=1e-10)


@pytest.mark.slow
def test_taylor_green_second_order_without_ib():
    """Sec. 2.5: without the IB the scheme is second order in space (error ratio ~4 per halving)."""
    re, dt, nsteps = 100.0, 2e-3, 50
    errs = []
    for n in (16, 32, 64):
        u0, _, dx = W.taylor_green(n, 0.0, re)
        case = oracle.Case(n, n, 1, dx, 1.0 / re, dt, PER, csm_on=0, forcing_on=0)
        st = case.initial_state(u0)
        for _ in range(nsteps):
            case.step(st, tol=1e-12)
        ua, _, _ = W.taylor_green(n, nsteps * dt, re)
        e = st["u"].reshape(3, -1)[0] - ua[0].reshape(-1)
        errs.append(np.sqrt(np.mean(e ** 2)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((slopes > 1.8) & (slopes < 2.3)), (errs, slopes)
    # the decay rate of the velocity amplitude matches exp(-2 pi^2 t / Re)
    assert GOLD["taylor_green"]["velocity_decay_rate"] == pytest.approx(2 * np.pi ** 2 / re)


@pytest.mark.slow
@pytest.mark.parametrize("integrator", [0, 1])
@pytest.mark.parametrize("shape", ["circle", "diamond"])
def test_taylor_green_with_an_immersed_body_converges(shape, integrator):
    """The verification of Sec. 2.5: the periodic Taylor-Green vortex (Re = 100) with a circle of radius
    1 or the inscribed square of side sqrt(2), the wall velocity taken from the analytic solution,
    central differences, ghost cells plus forcing; AB2 as in the paper, and the Crank-Nicolson
    predictor of Eq. crank-nicolson.  The paper measures L2 slopes of 1.34-1.37 (about 2
    on its coarse grids) from the first-order axis projection.  Here each halving must cut the L2 error
    by a slope between 1 and 2.3, and the maximum error must fall too.  The diamond's walls pass
    through cell centres (d = 0 and d = 1), the forcing's hardest case."""
    re, dt, nsteps = 100.0, 2e-3, 50
    l2, linf = [], []
    for n in (16, 32, 64):
        u0, _, dx = W.taylor_green(n, 0.0, re)
        case = oracle.Case(n, n, 1, dx, 1.0 / re, dt, PER, csm_on=0, integrator=integrator, mom_tol=1e-12)
        case.set_geometry(W.taylor_green_body(n, 1, shape))
        X = record_points(case, dx, -2.0)
        st = case.initial_state(u0)
        for k in range(nsteps):
            case.rec["uib"][:] = W.taylor_green_velocity(X[:, 0], X[:, 1], (k + 1) * dt, re)
            s = case.step(st, tol=1e-10)
            assert s.status == 0
        ua, _, _ = W.taylor_green(n, nsteps * dt, re)
        e = st["u"].reshape(3, -1)[0] - ua[0].reshape(-1)
        l2.append(np.sqrt(np.mean(e ** 2)))
        linf.append(np.abs(e).max())
    slopes = np.log2(np.array(l2[:-1]) / np.array(l2[1:]))
    assert np.all((slopes >= 1.0) & (slopes <= 2.3)), (l2, slopes)
    assert linf[0] > linf[1] > linf[2], linf


# --------------------------------------------------------------------------------------------------
# Forcing (Eq. forcing_term, discrete_forcing_term, distribution_function) and dead-end filter

def test_forcing_zero_at_wall_velocity_and_linear():
    case = _wall_case(float(np.float32(5.3)))
    N = case.N
    us = np.zeros(3 * N)
    out, fs = case.forcing(us)
    assert np.all(out == 0.0) and np.all(fs == 0.0)
    rng = np.random.default_rng(4)
    us = rng.standard_normal(3 * N)
    o1, f1 = case.forcing(us)
    o2, f2 = case.forcing(2.5 * us)
    assert np.allclose(o2 - 2.5 * us, 2.5 * (o1 - us), atol=1e-12)
    # one wall between cells 4 (centre 4.5, wall at d = 0.8) and 5 (wall at d = 0.2): each cell is
    # pulled towards u_IB = 0 by its own record with the ghost branch (1 - d)/(1 + d) of the printed D
    u = np.zeros(3 * N)
    u[:N] = 1.0
    o, _ = case.forcing(u)
    x = np.arange(N) % 12
    d = float(np.float32(5.3)) - 4.5
    expP = 1.0 - (1 - d) / (1 + d)
    expG = 1.0 - d / (1 + (1 - d))
    assert np.allclose(o[:N][x == 4], expP) and np.allclose(o[:N][x == 5], expG)
    assert np.allclose(o[:N][(x != 4) & (x != 5)], 1.0)
    # a cell crossed by several walls whose weights add up to more than 1 takes their normalised sum:
    # cell (4, 4) boxed by walls at 4.05 and 4.95 in x and y (d = 0.45 on four links, total weight
    # 4 * 0.55 / 1.45 > 1); with u* uniform every wall velocity interpolates to u*, so the normalised
    # force lands the cell exactly on u_IB = 0 (the plain sum would overshoot to -0.52)
    lo, hi = -40.0, 120.0
    walls = [[[4.05, lo, lo], [4.05, hi, lo], [4.05, lo, hi]], [[4.95, lo, lo], [4.95, hi, lo], [4.95, lo, hi]],
             [[lo, 4.05, lo], [lo, 4.05, hi], [hi, 4.05, lo]], [[lo, 4.95, lo], [lo, 4.95, hi], [hi, 4.95, lo]]]
    box = oracle.Case(9, 9, 5, bc=SLIPBOX)
    box.set_geometry(np.array(walls, np.float32))
    P = 4 + 9 * (4 + 9 * 2)
    assert bin(int(box.flags[P]) & 63).count("1") == 4
    assert 4 * 0.55 / 1.45 > 1.0
    u = np.zeros(3 * box.N)
    u[:box.N] = 1.0
    o, _ = box.forcing(u)
    assert abs(o[P]) < 1e-6


def test_forcing_imposes_the_wall_velocity_on_a_cell_the_wall_passes_through():
    """Gibou's imposition, which Eq. distribution_function follows: a wall through the centre of cell
    P (d = 0) gives P the weight 1, so after the forcing u_P equals u_IB whatever the field, while the
    cell across, whose wall point lies a full cell away (d = 1), gets the weight 0."""
    case = _wall_case(4.5)
    N = case.N
    r = case.rec
    x = r["cell"] % 12
    assert np.all(r["d"][x == 4] == 0.0) and np.all(r["d"][x == 5] == 1.0)
    assert np.all(r["w_ghost"][x == 4] == 1.0) and np.all(r["w_ghost"][x == 5] == 0.0)
    v = np.array([0.3, -0.7, 0.25])
    case.rec["uib"][:] = v
    rng = np.random.default_rng(11)
    u = rng.standard_normal(3 * N)
    o, _ = case.forcing(u)
    xc = np.arange(N) % 12
    for c in range(3):
        assert np.allclose(o[c * N:(c + 1) * N][xc == 4], v[c], rtol=0, atol=1e-14)   # u + dt (v - u)/dt
        assert np.array_equal(o[c * N:(c + 1) * N][xc != 4], u[c * N:(c + 1) * N][xc != 4])


def test_deadend_filter_cancels_forcing():
    """Eq. deadend_filter: the forcing is cancelled where at least 5 of the 6 axis links are blocked (at
    most one open direction), and kept where two directions stay open.  Cell (4, 4, 4) of a 9^3 slip box
    is walled in on 4, 5 or 6 sides by full planes."""
    thr = GOLD["deadend_threshold"]["value"]
    n = 9
    lo, hi = -40.0, 120.0     # right triangles whose legs span the whole cross-section
    planes = {
        "x-": [[4.2, lo, lo], [4.2, hi, lo], [4.2, lo, hi]], "x+": [[4.8, lo, lo], [4.8, hi, lo], [4.8, lo, hi]],
        "y-": [[lo, 4.3, lo], [lo, 4.3, hi], [hi, 4.3, lo]], "y+": [[lo, 4.7, lo], [lo, 4.7, hi], [hi, 4.7, lo]],
        "z-": [[lo, lo, 4.2], [hi, lo, 4.2], [lo, hi, 4.2]], "z+": [[lo, lo, 4.8], [hi, lo, 4.8], [lo, hi, 4.8]],
    }
    P = 4 + n * (4 + n * 4)
    for walls in (["x-", "x+", "y-", "y+"], ["x-", "x+", "y-", "y+", "z-"], sorted(planes)):
        tri = np.array([planes[w] for w in walls], np.float32)
        for on in (0, 1):
            case = oracle.Case(n, n, n, bc=SLIPBOX, deadend_on=on)
            case.set_geometry(tri)
            assert bin(int(case.flags[P]) & 63).count("1") == len(walls)
            o, _ = case.forcing(np.ones(3 * case.N))
            forced = o[P] != 1.0
            assert forced == (on == 0 or len(walls) < thr), (walls, on)


# --------------------------------------------------------------------------------------------------
# Invariance to dirty topology (Sec. 3.3)

@pytest.mark.slow
def test_cracks_duplicates_and_a_hidden_shell_leave_the_outside_flow_unchanged():
    """Sec. 3.3: a sphere whose faces do not join (every vertex copy jittered by 0.02 cells), carries
    duplicated faces 0.1 cells off its surface and hides a nested shell gives the same outside flow as
    the clean sphere, because the outermost surface is the same.  Sphere of radius 4 at 64x32x32,
    Re = 100, 20 steps: beyond 1.5 cells from the surface the velocity fields agree to 1 % (relative
    L2), and pointwise to a fifth of the wake's own deviation from the free stream."""
    cfg = W.get_config("sphere_64x32x32")
    clean = cfg.soup()
    rng = np.random.default_rng(21)
    tri = clean.astype(np.float64)
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    dup = rng.choice(len(tri), size=len(tri) // 50, replace=False)
    dirty = np.concatenate([tri, tri[dup] + 0.1 * nrm[dup][:, None, :]])
    dirty = dirty + rng.normal(0.0, 0.02, dirty.shape)
    dirty = np.concatenate([dirty, W.icosphere(3, 2.8, (16.0, 16.0, 16.0), dtype=np.float64)]).astype(np.float32)
    u = {}
    for name, soup in (("clean", clean), ("dirty", dirty)):
        case = oracle.Case.from_config(cfg)
        case.set_geometry(soup)
        st = case.initial_state(W.initial_fields(cfg))
        for _ in range(20):
            assert case.step(st, tol=1e-6).status == 0
        u[name] = st["u"].reshape(3, -1)
    N = cfg.ncell
    c = np.stack([np.arange(N) % 64, (np.arange(N) // 64) % 32, np.arange(N) // (64 * 32)]) + 0.5
    out = np.linalg.norm(c - 16.0, axis=0) > 5.5
    diff = u["dirty"][:, out] - u["clean"][:, out]
    wake = np.abs(u["clean"][0, out] - 1.0).max()
    assert wake > 0.3
    assert np.linalg.norm(diff) < 0.01 * np.linalg.norm(u["clean"][:, out])
    assert np.abs(diff).max() < 0.2 * wake


# --------------------------------------------------------------------------------------------------
# Forces (Eq. force)

def test_forces_constant_pressure_and_archimedes():
    n = 24
    R = 6.2
    c = (12.1, 11.9, 12.05)
    tri = W.icosphere(4, R, c)
    case = oracle.Case(n, n, n)
    x = centres(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    inside = ((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 < R ** 2).reshape(-1)
    out = case.forces(tri, np.full(n ** 3, 3.0))
    assert np.allclose(out[:3], 0.0, atol=1e-10) and out[3] == len(tri)
    p = np.where(inside, 3.0, 3.0 + 0 * X.reshape(-1))
    out = case.forces(tri, p)
    assert np.allclose(out[:3], 0.0, atol=1e-9)
    # p = x outside and a uniform value inside: F = -(volume) e_x (Archimedes), discretisation-limited
    p = np.where(inside, 0.0, X.reshape(-1))
    out = case.forces(tri, p)
    V = 4.0 / 3.0 * np.pi * R ** 3
    assert out[0] == pytest.approx(-V, rel=0.06)
    assert abs(out[1]) < 0.03 * V and abs(out[2]) < 0.03 * V


# --------------------------------------------------------------------------------------------------
# QUICK blending of the advective face value (the hybrid scheme of Sec. 3.1 / 3.3)

@pytest.mark.parametrize("Uval", [1.0, -1.0])
@pytest.mark.parametrize("gamma", [0.0, 0.1, 1.0])
def test_quick_blend_closed_form_on_a_cubic(Uval, gamma):
    """u_x = x^3 advected by a uniform U: the face-flux difference is 3x^2 + 1 for central values and
    3x^2 + 1/4 for QUICK's (6 upwind + 3 downwind - far upwind)/8, so H_x = -U (3x^2 + 1 - 3 gamma / 4)."""
    nx, ny, nz = 14, 4, 4
    case = oracle.Case(nx, ny, nz, nu=0.0, dt=0.1, bc=(3, 3, 0, 0, 0, 0), csm_on=0, quick=gamma)
    xc = np.arange(nx) + 0.5
    ux = np.broadcast_to(xc ** 3, (nz, ny, nx))
    u = np.stack([ux, 0 * ux, 0 * ux]).reshape(-1)
    U = np.zeros(case.NF)
    Ux, _, _ = oracle.split_faces(U, nx, ny, nz)
    Ux[...] = Uval
    H, _ = case.predict(u, U, np.zeros(case.N), np.zeros_like(u), True)
    Hx = H[:case.N].reshape(nz, ny, nx)
    exp = -Uval * (3 * xc ** 2 + 1.0 - 0.75 * gamma)
    assert np.allclose(Hx[:, :, 2:-2], np.broadcast_to(exp[2:-2], (nz, ny, nx - 4)), rtol=1e-12, atol=1e-9)


def test_quick_blend_conserves_momentum_periodic():
    n = 8
    rng = np.random.default_rng(11)
    case = oracle.Case(n, n, n, nu=0.02, dt=0.1, bc=PER, quick=0.1)
    u = rng.standard_normal(3 * n ** 3)
    H, _ = case.predict(u, case.faces(u), case.csm(u), np.zeros_like(u), True)
    assert np.all(np.abs(H.reshape(3, -1).sum(1)) < 1e-11 * np.abs(H).sum())


# --------------------------------------------------------------------------------------------------
# Crank-Nicolson predictor (Eq. crank-nicolson)

def _face_symbol(theta, Uval, gamma):
    """Advected value on face i+1/2 relative to u_i for the mode e^{i theta i}: central average
    blended with QUICK taken from the upwind side."""
    e = np.exp(1j * theta)
    central = 0.5 * (1 + e)
    quick = (6 + 3 * e - 1 / e) / 8 if Uval >= 0 else (6 * e + 3 - e * e) / 8
    return (1 - gamma) * central + gamma * quick


def _fourier_case(gamma, integrator):
    nx, ny, nz = 16, 12, 4
    nu, dt = 0.05, 0.4
    case = oracle.Case(nx, ny, nz, nu=nu, dt=dt, bc=PER, csm_on=0, quick=gamma, integrator=integrator)
    U = np.zeros(case.NF)
    Ux, Uy, _ = oracle.split_faces(U, nx, ny, nz)
    Ux[...] = 0.7
    Uy[...] = -0.45
    tx, ty = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    lam = 0.0
    for th, Uval in ((tx, 0.7), (ty, -0.45)):
        lam += -Uval * _face_symbol(th, Uval, gamma) * (1 - np.exp(-1j * th))
        lam += -nu * (2 - 2 * np.cos(th))
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    phase = tx * i + ty * j + np.zeros((nz, 1, 1))
    return case, U, lam, phase


@pytest.mark.parametrize("gamma", [0.0, 0.1])
def test_crank_nicolson_amplification_of_a_fourier_mode(gamma):
    """Uniform U = (0.7, -0.45, 0), periodic box, nu_t = 0: every mode e^{i(theta_x i + theta_y j)}
    is an eigenvector of L with the eigenvalue lam built from the face-value symbols, so the
    Crank-Nicolson predictor multiplies it by (1 + dt lam / 2) / (1 - dt lam / 2) and the Euler first
    step by 1 + dt lam."""
    case, U, lam, phase = _fourier_case(gamma, 1)
    dt = case.pr.dt
    comps = [np.cos(phase + q) for q in (0.0, 0.9, 2.1)]
    u = np.stack(comps).reshape(-1)
    H, us, it = case.predict_cn(u, U, np.zeros(case.N), tol=1e-14, maxit=200)
    assert it > 0
    g = (1 + 0.5 * dt * lam) / (1 - 0.5 * dt * lam)
    exp = np.stack([np.real(g * np.exp(1j * (phase + q))) for q in (0.0, 0.9, 2.1)]).reshape(-1)
    assert np.allclose(us, exp, rtol=0, atol=1e-11)
    # the Euler first step of the explicit path uses the same operator
    _, ue = case.predict(u, U, np.zeros(case.N), np.zeros_like(u), True)
    exp_e = np.stack([np.real((1 + dt * lam) * np.exp(1j * (phase + q))) for q in (0.0, 0.9, 2.1)]).reshape(-1)
    assert np.allclose(ue, exp_e, rtol=0, atol=1e-12)
    # the scheme is neutral for pure advection and damps with diffusion: |g| < 1 here
    assert abs(g) < 1.0


def test_momentum_operator_is_affine_with_the_homogeneous_part():
    """With a wall (cut links, moving wall velocity) and an inflow face, L(u) - L(0) equals the
    homogeneous operator L_0(u) for any u, and L_0 is linear."""
    case = oracle.Case(14, 10, 9, nu=0.03, dt=0.2, bc=(1, 2, 3, 3, 4, 0), u_in=(1.0, 0.2, -0.1), quick=0.1)
    tri = W.icosphere(2, 2.6, (6.3, 5.1, 4.4))
    case.set_geometry(tri)
    assert len(case.rec) > 0
    case.rec["uib"][:, 0] = 0.3            # a moving wall: the inhomogeneous ghost part is nonzero
    rng = np.random.default_rng(5)
    u = rng.standard_normal(3 * case.N)
    v = rng.standard_normal(3 * case.N)
    U = case.faces(u)
    nut = np.abs(rng.standard_normal(case.N)) * 0.01
    L0 = case.momentum_operator(np.zeros(3 * case.N), U, nut)
    assert np.abs(L0).max() > 1e-3
    Lu = case.momentum_operator(u, U, nut)
    Lh = case.momentum_operator(u, U, nut, hom=True)
    assert np.allclose(Lu - L0, Lh, rtol=0, atol=1e-12)
    Lhv = case.momentum_operator(v, U, nut, hom=True)
    Lhs = case.momentum_operator(2.0 * u - 3.0 * v, U, nut, hom=True)
    assert np.allclose(Lhs, 2.0 * Lh - 3.0 * Lhv, rtol=0, atol=1e-11)


def test_crank_nicolson_solves_its_system_with_a_body():
    """u* - u^n = dt (L(u*) + L(u^n)) / 2 holds to the solve tolerance with cut links and an inflow."""
    case = oracle.Case(14, 10, 9, nu=0.03, dt=0.3, bc=(1, 2, 3, 3, 4, 3), u_in=(1.0, 0.0, 0.0), quick=0.1,
                       integrator=1)
    case.set_geometry(W.icosphere(2, 2.6, (6.3, 5.1, 4.4)))
    rng = np.random.default_rng(6)
    u = np.concatenate([np.ones(case.N), np.zeros(2 * case.N)]) + 0.1 * rng.standard_normal(3 * case.N)
    U = case.faces(u)
    nut = case.csm(u)
    H, us, it = case.predict_cn(u, U, nut, tol=1e-13, maxit=300)
    assert it > 0
    assert np.allclose(H, case.momentum_operator(u, U, nut), rtol=0, atol=0)
    lhs = (us - u) / case.pr.dt
    rhs = 0.5 * (case.momentum_operator(us, U, nut) + H)
    assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(H)


def test_crank_nicolson_uniform_flow_and_momentum():
    n = 8
    case = oracle.Case(n, n, n, nu=0.05, dt=0.3, bc=PER, quick=0.1, integrator=1)
    u = np.concatenate([np.full(n ** 3, 0.3), np.full(n ** 3, -0.2), np.full(n ** 3, 0.1)])
    H, us, it = case.predict_cn(u, case.faces(u), case.csm(u))
    assert it == 0 and np.array_equal(us, u)
    rng = np.random.default_rng(12)
    u = rng.standard_normal(3 * n ** 3)
    H, us, it = case.predict_cn(u, case.faces(u), case.csm(u), tol=1e-13)
    assert it > 0
    d = (us - u).reshape(3, -1).sum(1)
    assert np.all(np.abs(d) < 1e-11 * np.abs(us - u).sum())


@pytest.mark.slow
def test_crank_nicolson_step_converges_in_time():
    """Taylor-Green vortex on a fixed 32x32 grid with Crank-Nicolson steps: halving dt halves the
    difference to a dt/8 run.  The predictor alone is second order (the Fourier pin above), but the
    step corrects with p^{n+1} only (Eq. correction, no pressure in the predictor) and advects with
    U^n, so the whole step is first order in time."""
    n, re, T = 32, 50.0, 0.4
    u0, _, dx = W.taylor_green(n, 0.0, re)
    sols = {}
    for dt in (0.1, 0.05, 0.0125):
        case = oracle.Case(n, n, 1, dx, 1.0 / re, dt, PER, csm_on=0, forcing_on=0, integrator=1,
                           mom_tol=1e-13)
        st = case.initial_state(u0)
        for _ in range(int(round(T / dt))):
            case.step(st, tol=1e-13)
        sols[dt] = st["u"].copy()
    e1 = np.linalg.norm(sols[0.1] - sols[0.0125])
    e2 = np.linalg.norm(sols[0.05] - sols[0.0125])
    ratio = e1 / e2
    assert 1.8 < ratio < 2.6, ratio


# --------------------------------------------------------------------------------------------------
# Surface pressure and the thin-plate filter (Eq. force, Eq. force_filter)

def _square(z, lo=3.1, hi=12.9):
    a, b, c, d = (lo, lo, z), (hi, lo, z), (hi, hi, z), (lo, hi, z)
    return np.array([[a, b, c], [a, c, d]], np.float32)


def test_filter_cancels_the_inner_faces_of_a_thin_plate():
    """Two parallel squares 0.1 cells apart (a plate thinner than a cell): without the filter both
    squares see both sides and the force doubles; with it the inner faces are cancelled and the pair
    carries the force of one square."""
    n = 16
    case = oracle.Case(n, n, n)
    x = centres(n)
    Z = np.meshgrid(x, x, x, indexing="ij")[0].reshape(-1)
    p = 2.0 + 0.5 * Z + np.where(Z > 10.25, 1.5, 0.0)      # a jump across the plate
    one = _square(10.2)
    two = np.concatenate([one, _square(10.3)])
    ps1, F1 = case.surface_pressure(one, p, zfilter=True)
    ps0, F0 = case.surface_pressure(one, p, zfilter=False)
    assert np.array_equal(ps1, ps0) and np.array_equal(F1, F0)          # nothing to hide behind
    assert F1[3] == 4 and abs(F1[2]) > 1.0
    ps2, F2 = case.surface_pressure(two, p, zfilter=True)
    assert np.all(np.isnan(ps2[:2, 0])) and np.all(np.isnan(ps2[2:, 1]))  # inner faces cancelled
    assert np.allclose(ps2[:2, 1], ps1[:, 1]) and not np.any(np.isnan(ps2[2:, 0]))
    assert F2[3] == 4
    assert np.allclose(F2[:3], F1[:3], rtol=0.0, atol=1e-12 * abs(F1[2]) + 0.02 * abs(F1[2]))
    _, F2n = case.surface_pressure(two, p, zfilter=False)
    assert F2n[3] == 8
    assert F2n[2] == pytest.approx(2.0 * F1[2], rel=0.03)


def test_filter_on_a_double_skin_sphere_gives_archimedes_once():
    """A closed sphere wrapped in a second skin 0.1 cells outside (the frame-skin case): with p = x
    outside and 0 inside, the filtered force is close to -V e_x of one body, the unfiltered one about
    twice.  Cell centres that happen to lie inside the 0.1-cell gap still count for both skins (the
    filter cancels only where no point lies between them), hence the looser bound."""
    n = 24
    R = 6.2
    c = (12.1, 11.9, 12.05)
    inner = W.icosphere(3, R, c)
    outer = W.icosphere(3, R + 0.1, c)
    case = oracle.Case(n, n, n)
    x = centres(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    inside = ((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 < (R + 0.05) ** 2).reshape(-1)
    p = np.where(inside, 0.0, X.reshape(-1))
    V = 4.0 / 3.0 * np.pi * R ** 3
    _, Fs = case.surface_pressure(inner, p, zfilter=True)
    assert Fs[0] == pytest.approx(-V, rel=0.08)
    psf, Ff = case.surface_pressure(np.concatenate([inner, outer]), p, zfilter=True)
    assert Ff[0] == pytest.approx(-V, rel=0.15)
    nt = len(inner)
    assert np.isnan(psf[:nt, 0]).mean() > 0.6 and np.isnan(psf[nt:, 1]).mean() > 0.6
    assert not np.isnan(psf[:nt, 1]).any() and not np.isnan(psf[nt:, 0]).any()
    _, Fn = case.surface_pressure(np.concatenate([inner, outer]), p, zfilter=False)
    assert Fn[0] == pytest.approx(-2.0 * V, rel=0.12)


def test_surface_pressure_uniform_and_matches_forces_on_a_clean_body():
    n = 24
    R = 6.2
    c = (12.1, 11.9, 12.05)
    tri = W.icosphere(3, R, c)
    case = oracle.Case(n, n, n)
    ps, F = case.surface_pressure(tri, np.full(n ** 3, 3.0), zfilter=True)
    ok = ~np.isnan(ps)
    assert ok.all() and np.allclose(ps, 3.0, rtol=1e-15, atol=0)
    rng = np.random.default_rng(4)
    p = rng.standard_normal(n ** 3)
    ps, F = case.surface_pressure(tri, p, zfilter=False)
    both = ~np.isnan(ps).any(1)
    ref = case.forces(tri, p)
    if both.all():
        assert np.allclose(F[:3], ref[:3], rtol=1e-12, atol=1e-12)


def test_viscous_force_of_a_sheared_plate():
    """A zero-thickness no-slip plate spanning a periodic box at z = 4.3 with u_x = a |z - 4.3| on both
    sides: the ghost values of Eq. q_axis are exact for the linear profiles, every column has one cut
    link on each side, each carries nu a dx^2, so F_x = 2 nu a (nx ny dx^2) and F_y = F_z = 0; with
    u_x = a (z - 4.3) (the same shear continuing through the plate) the two sides cancel."""
    nx, ny, nz, nu, a = 8, 6, 9, 0.07, 0.3
    case = oracle.Case(nx, ny, nz, nu=nu, dt=0.1, bc=(0, 0, 0, 0, 3, 3))
    zw = 4.3
    tri = np.array([[(-1, -1, zw), (9, -1, zw), (9, 9, zw)], [(-1, -1, zw), (9, 9, zw), (-1, 9, zw)]], np.float32)
    case.set_geometry(tri)
    assert len(case.rec) == 2 * nx * ny
    z = np.arange(nz) + 0.5
    zz = np.broadcast_to(z[:, None, None], (nz, ny, nx)).reshape(-1)
    zwf = float(np.float32(zw))
    u = np.concatenate([a * np.abs(zz - zwf), np.zeros(case.N), np.zeros(case.N)])
    F = case.viscous_force(u)
    assert F[3] == 2 * nx * ny
    assert F[0] == pytest.approx(2 * nu * a * nx * ny, rel=1e-12)
    assert abs(F[1]) < 1e-14 and abs(F[2]) < 1e-14
    u = np.concatenate([a * (zz - zwf), np.zeros(case.N), np.zeros(case.N)])
    F = case.viscous_force(u)
    assert abs(F[0]) < 1e-12

"""The step at the two largest workloads' full sizes, in the configuration the benchmark times, against
the FP64 CPU oracle.

Workloads: the 512x256x256 cube and plate on a no-slip floor, and the 1024x512x384 vehicle-like
assembly (about 2 M dirty triangles, gaps, nested parts, dead-end filter on).  Scheme: FP32 stencils
with FP64 iterative refinement, Crank-Nicolson with 10 % QUICK, CG preconditioned by the connected-part
multigrid with omega 1.6, inner tolerance 1e-5 and residual checks every 8 iterations.  After a few
steps on the GPU:
- every operator of the step, applied by the GPU to its own full-size fields, matches the oracle on a
  z-slab: the oracle runs on the slab plus two planes each side (the stencils reach two cells) and the
  two are compared on the slab's inner planes;
- the pressure residual ||b - A p|| / ||b|| of the GPU's last step, evaluated by the oracle's operator
  on the whole grid, is within the tolerance;
- the projection identity div U^{n+1} = dt (b - A p) holds cell by cell on the whole grid.
And 10 steps on a true-scale crop of the vehicle assembly (under the body's front corner, with
dead-end cells and butted parts) match the oracle's 10 steps.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

FULL = ["cube_plate_512x256x256", "vehicle_1024x512x384"]
QUICK = 0.1
FP32_OP_TOL = 2e-5


@pytest.fixture(scope="module")
def L():
    from paper_2002_06206_gb300 import build
    build.build()
    from paper_2002_06206_gb300 import ibmles
    ibmles.lib()
    return ibmles


def bench_solver(L, g, cfg, geo, tol=None):
    return L.Solver(g, cfg.nu, cfg.dt, cfg.bc, cfg.u_in, precision=L.FP32_REFINE64, solver=L.CG,
                    tol=cfg.tol if tol is None else tol, check_every=8, inner_tol=1e-5, geometry=geo,
                    precond=L.MULTIGRID, mg_sweeps=2, mg_omega=1.6, quick=QUICK, integrator=L.CRANK_NICOLSON)


def rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


@pytest.fixture(scope="module", params=FULL)
def run(L, request):
    cfg = W.get_config(request.param)
    tri = cfg.soup()
    g = L.make_grid(cfg.nx, cfg.ny, cfg.nz, cfg.dx)
    geo = L.Geometry(g, torch.from_numpy(tri).cuda(), deadend_on=cfg.deadend_on)
    solver = bench_solver(L, g, cfg, geo)
    st = solver.fields(W.initial_fields(cfg))
    for _ in range(4):
        s = solver.step(st)
        assert s.status == 0 and s.relres <= cfg.tol
    torch.cuda.synchronize()
    yield cfg, tri, geo, solver, st, s
    solver.close()
    geo.close()
    del st
    torch.cuda.empty_cache()


def cells_slab(x, cfg, lo, nzs, ncomp):
    """z-planes [lo, lo + nzs) of a component-major cell field (device) as float64 (host)."""
    v = x.view(ncomp, cfg.nz, cfg.ny, cfg.nx)[:, lo:lo + nzs]
    return v.cpu().numpy().astype(np.float64).reshape(-1)


def faces_slab(U, cfg, lo, nzs):
    """The faces of z-planes [lo, lo + nzs) of a concatenated face vector (device), as float64 (host)."""
    nx, ny, nz = cfg.nx, cfg.ny, cfg.nz
    nfx, nfy = (nx + 1) * ny * nz, nx * (ny + 1) * nz
    Ux = U[:nfx].view(nz, ny, nx + 1)[lo:lo + nzs]
    Uy = U[nfx:nfx + nfy].view(nz, ny + 1, nx)[lo:lo + nzs]
    Uz = U[nfx + nfy:].view(nz + 1, ny, nx)[lo:lo + nzs + 1]
    return np.concatenate([t.cpu().numpy().astype(np.float64).reshape(-1) for t in (Ux, Uy, Uz)])


def inner(x, cfg, nzs, ncomp, m=2):
    return x.reshape(ncomp, nzs, cfg.ny, cfg.nx)[:, m:nzs - m]


def inner_faces(Uf, cfg, nzs, m=2, outflow=True):
    """Inner-plane faces of a slab face vector; the outflow face column (shifted by a whole-domain flux
    sum) is left out when `outflow` is False."""
    Ux, Uy, Uz = oracle.split_faces(Uf, cfg.nx, cfg.ny, nzs)
    Ux = Ux[m:nzs - m, :, :] if outflow else Ux[m:nzs - m, :, :cfg.nx]
    return np.concatenate([Ux.reshape(-1), Uy[m:nzs - m].reshape(-1), Uz[m:nzs - m + 1].reshape(-1)])


def slab_case(cfg, tri, lo, nzs):
    t = tri.copy()
    t[..., 2] -= np.float32(lo)
    case = oracle.Case(cfg.nx, cfg.ny, nzs, cfg.dx, cfg.nu, cfg.dt, cfg.bc, cfg.u_in, cfg.csm_on, cfg.forcing_on,
                       cfg.deadend_on, QUICK, 1)
    case.set_geometry(t)
    return case


def test_full_size_operators_match_the_oracle_on_a_slab(L, run):
    cfg, tri, geo, solver, st, _ = run
    N, NF = cfg.ncell, solver.NF
    P = 8
    # a slab through the bodies: the plate of the cube-and-plate workload, the middle of the assembly
    k0 = 60 if cfg.nz == 256 else 92
    lo, nzs = k0 - 2, P + 4
    case = slab_case(cfg, tri, lo, nzs)
    fl = geo.flags.view(cfg.nz, cfg.ny, cfg.nx)[lo:lo + nzs].cpu().numpy()
    fin = case.flags.reshape(nzs, cfg.ny, cfg.nx)
    # the slab's own classification agrees with the full grid's away from the slab's ends
    assert np.array_equal(fl[2:-2], fin[2:-2])
    assert np.count_nonzero(fl[2:-2] & 63) > 1000
    f32 = torch.float32
    u, U, p = st["u"], st["U"], st["p"]
    # GPU: the step's operators on its own full-size fields
    nut = torch.empty(N, dtype=f32, device="cuda")
    solver.csm(u, nut)
    H = torch.empty(3 * N, dtype=f32, device="cuda")
    us = torch.empty(3 * N, dtype=f32, device="cuda")
    solver.predict_cn(u, U, nut, H, us)
    usf = us.clone()
    solver.forcing(usf)
    Us = torch.empty(NF, dtype=f32, device="cuda")
    solver.faces(usf, Us)
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    solver.rhs(Us, b)
    un = torch.empty(3 * N, dtype=f32, device="cuda")
    Un = torch.empty(NF, dtype=f32, device="cuda")
    solver.correct(usf, Us, p, un, Un)
    torch.cuda.synchronize()
    # oracle on the slab, from the GPU's inputs
    u_s = cells_slab(u, cfg, lo, nzs, 3)
    nut_ref = case.csm(u_s)
    assert rel(inner(cells_slab(nut, cfg, lo, nzs, 1), cfg, nzs, 1), inner(nut_ref, cfg, nzs, 1)) <= FP32_OP_TOL
    U_s = faces_slab(U, cfg, lo, nzs)
    nut_s = cells_slab(nut, cfg, lo, nzs, 1)
    H_ref = case.momentum_operator(u_s, U_s, nut_s)
    Hg, Hr = inner(cells_slab(H, cfg, lo, nzs, 3), cfg, nzs, 3), inner(H_ref, cfg, nzs, 3)
    scale = np.linalg.norm(np.abs(U_s).max() * inner(u_s, cfg, nzs, 3)) + np.linalg.norm(Hr)
    assert np.linalg.norm(Hg - Hr) <= FP32_OP_TOL * scale
    us_s = cells_slab(us, cfg, lo, nzs, 3)
    usf_ref, _ = case.forcing(us_s)
    assert rel(inner(cells_slab(usf, cfg, lo, nzs, 3), cfg, nzs, 3), inner(usf_ref, cfg, nzs, 3)) <= FP32_OP_TOL
    usf_s = cells_slab(usf, cfg, lo, nzs, 3)
    Us_ref = case.faces(usf_s)
    Us_s = faces_slab(Us, cfg, lo, nzs)
    assert rel(inner_faces(Us_s, cfg, nzs, outflow=False), inner_faces(Us_ref, cfg, nzs, outflow=False)) <= FP32_OP_TOL
    b_ref = case.rhs(Us_s)
    assert rel(inner(cells_slab(b, cfg, lo, nzs, 1), cfg, nzs, 1), inner(b_ref, cfg, nzs, 1)) <= FP32_OP_TOL
    p_s = cells_slab(p, cfg, lo, nzs, 1)
    un_ref, Un_ref = case.correct(usf_s, Us_s, p_s)
    assert rel(inner(cells_slab(un, cfg, lo, nzs, 3), cfg, nzs, 3), inner(un_ref, cfg, nzs, 3)) <= FP32_OP_TOL
    assert rel(inner_faces(faces_slab(Un, cfg, lo, nzs), cfg, nzs), inner_faces(Un_ref, cfg, nzs)) <= FP32_OP_TOL
    Ap = torch.empty(N, dtype=torch.float64, device="cuda")
    solver.apply(p, Ap)
    assert rel(inner(cells_slab(Ap, cfg, lo, nzs, 1), cfg, nzs, 1), inner(case.apply(p_s), cfg, nzs, 1)) <= 1e-12


def test_full_size_residual_and_projection_identity(L, run):
    cfg, tri, geo, solver, st, s = run
    N = cfg.ncell
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    solver.last_rhs(b)
    bh, ph = b.cpu().numpy(), st["p"].cpu().numpy()
    ref = oracle.Case(cfg.nx, cfg.ny, cfg.nz, cfg.dx, cfg.nu, cfg.dt, cfg.bc, cfg.u_in, cfg.csm_on, cfg.forcing_on,
                      cfg.deadend_on, QUICK, 1)
    ref.set_geometry(tri)
    assert np.array_equal(ref.flags, geo.flags.cpu().numpy())
    res = bh - ref.apply(ph)
    relres = np.linalg.norm(res) / np.linalg.norm(bh)
    assert relres <= cfg.tol * 1.0001 and abs(relres - s.relres) <= 1e-3 * cfg.tol
    del ph
    Ux, Uy, Uz = oracle.split_faces(st["U"].cpu().numpy(), cfg.nx, cfg.ny, cfg.nz)
    umax = max(np.abs(Ux).max(), np.abs(Uy).max(), np.abs(Uz).max())
    div = (np.diff(Ux, axis=2).astype(np.float64) + np.diff(Uy, axis=1) + np.diff(Uz, axis=0)).reshape(-1)
    # FP32 faces: the identity holds to the rounding of the stored face values
    assert np.abs(div - cfg.dt * res).max() <= 1e-5 * umax


def vehicle_crop():
    """A 48x32x24 window of the vehicle assembly at its own resolution, under the front corner of the
    body (z from 13, next to the parts that hang below it): butted parts with sub-cell gaps and four
    dead-end cells."""
    cfg = W.get_config("vehicle_1024x512x384")
    tri = cfg.soup()
    lo = np.array([192, 363, 13], np.float32)
    n = np.array([48, 32, 24])
    sel = np.all((tri.max(1) >= lo - 1) & (tri.min(1) <= lo + n + 1), axis=1)
    return cfg, (tri[sel] - lo).astype(np.float32), n


def test_ten_steps_on_a_vehicle_crop_match_the_oracle(L):
    cfg, tri, (nx, ny, nz) = vehicle_crop()
    g = L.make_grid(int(nx), int(ny), int(nz))
    geo = L.Geometry(g, torch.from_numpy(tri).cuda(), deadend_on=1)
    ref = oracle.Case(int(nx), int(ny), int(nz), 1.0, cfg.nu, cfg.dt, cfg.bc, cfg.u_in, 1, 1, 1, QUICK, 1)
    ref.pr.mom_tol = 1e-10
    ref.set_geometry(tri)
    assert np.array_equal(geo.flags.cpu().numpy(), ref.flags)
    cut = sum(((ref.flags >> q) & 1).astype(int) for q in range(6))
    assert (cut >= 5).sum() >= 4                     # the dead-end filter has cells to act on
    solver = bench_solver(L, g, W.Config("crop", int(nx), int(ny), int(nz), cfg.nu, cfg.dt, 10, 1e-6, 1, cfg.bc),
                          geo)
    u0 = W.initial_fields(W.Config("crop", int(nx), int(ny), int(nz), 0, 0, 0, 0, 0, cfg.bc, seed=4))
    st = solver.fields(u0)
    ost = ref.initial_state(u0)
    for _ in range(10):
        s = solver.step(st)
        assert s.status == 0 and s.relres <= 1e-6
        ref.step(ost, tol=1e-6)
    torch.cuda.synchronize()
    assert rel(st["u"].cpu().numpy(), ost["u"]) <= 1e-4
    assert rel(st["U"].cpu().numpy(), ost["U"]) <= 1e-4
    solver.close()

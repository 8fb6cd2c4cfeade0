"""The multigrid preconditioner of the pressure solve on the GPU.

- Its coarse unknowns are the connected parts of the 2^l-cell blocks: the number of unknowns of every
  level equals the number of connected components of the fine cells' link graph cut into those blocks,
  counted here by brute force on the oracle's flags.
- The fused fine-grid passes (TMA-staged, z-marching kernels that do the four half-sweeps before the
  coarse correction plus the restriction in one pass, and the four after it plus (r, z) in another)
  give the V-cycle of the separate passes: one V-cycle applied to the same vector agrees to FP32
  rounding, on grids with ragged tiles, several z-chunks and an odd plane count; and whole solves reach
  the tolerance with the same iteration counts.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

CHANNEL = (1, 2, 3, 3, 3, 3)
GROUND = (1, 2, 3, 3, 4, 3)


@pytest.fixture(scope="module")
def L():
    from paper_2002_06206_gb300 import build
    build.build()
    from paper_2002_06206_gb300 import ibmles
    ibmles.lib()
    return ibmles


def soup_for(nx, ny, nz, seed):
    """A dirty sphere, a zero-thickness plate and loose triangles, sized to the grid."""
    r = 0.22 * min(nx, ny, nz)
    c = (0.3 * nx + 0.37, 0.5 * ny - 0.21, 0.5 * nz + 0.13)
    return np.concatenate([W.dirty_sphere(seed=seed, radius=r, center=c, subdiv=3),
                           W.fan_disk((0.62 * nx + 0.3, 0.45 * ny, 0.5 * nz), 0.3 * min(ny, nz), 0, 48),
                           W.random_soup(120, (2, 2, 2), (nx - 2, ny - 2, nz - 2), 3.0, seed=seed)]).astype(np.float32)


def components_in_blocks(flags, n, level):
    """Connected components of the fine link graph (uncut links inside the domain) after removing every
    link that leaves a 2^level block."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    nx, ny, nz = n
    N = nx * ny * nz
    f = flags.reshape(nz, ny, nx)
    idx = np.arange(N).reshape(nz, ny, nx)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rows, cols = [], []
    for a, bit in ((2, 2), (1, 8), (0, 32)):                  # +x, +y, +z links (axis of the array)
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[a] = slice(0, -1)
        sl1[a] = slice(1, None)
        sl0, sl1 = tuple(sl0), tuple(sl1)
        coord = (K, J, I)[a]
        ok = ((f[sl0] & bit) == 0) & ((coord[sl0] >> level) == (coord[sl1] >> level))
        rows.append(idx[sl0][ok])
        cols.append(idx[sl1][ok])
    r, c = np.concatenate(rows), np.concatenate(cols)
    G = coo_matrix((np.ones(len(r)), (r, c)), shape=(N, N))
    return connected_components(G, directed=False)[0]


@pytest.mark.parametrize("shape,bc", [((112, 50, 37), CHANNEL), ((96, 40, 33), GROUND)])
def test_coarse_unknowns_are_the_connected_parts_of_each_block(L, shape, bc):
    nx, ny, nz = shape
    tri = soup_for(nx, ny, nz, 5)
    g = L.make_grid(nx, ny, nz)
    geo = L.Geometry(g, torch.from_numpy(tri).cuda())
    ref = oracle.Case(nx, ny, nz, bc=bc)
    ref.classify(tri)
    assert np.array_equal(geo.flags.cpu().numpy() & 63, ref.flags & 63)
    solver = L.Solver(g, 0.01, 0.2, bc, precision=L.FP32_REFINE64, tol=1e-6, geometry=geo, precond=L.MULTIGRID)
    nlev, _, M = solver.mg_info()
    assert nlev >= 3
    for lev in range(1, nlev):
        expect = components_in_blocks(ref.flags, shape, lev)
        assert M[lev] == expect, (lev, M[lev], expect)
    # walls split blocks: more unknowns than whole blocks on level 1
    assert M[1] > ((nx + 1) // 2) * ((ny + 1) // 2) * ((nz + 1) // 2)
    solver.close()


@pytest.mark.parametrize("shape,bc", [((112, 50, 37), CHANNEL), ((128, 64, 96), GROUND), ((256, 128, 128), CHANNEL)])
def test_fused_fine_passes_give_the_vcycle_of_separate_passes(L, shape, bc):
    nx, ny, nz = shape
    tri = soup_for(nx, ny, nz, 7)
    g = L.make_grid(nx, ny, nz)
    geo = L.Geometry(g, torch.from_numpy(tri).cuda())
    solvers = [L.Solver(g, 0.01, 0.2, bc, precision=L.FP32_REFINE64, tol=1e-6, geometry=geo, precond=L.MULTIGRID,
                        mg_omega=1.8, mg_passes=passes) for passes in (0, 1)]
    assert solvers[0].mg_info()[1] and not solvers[1].mg_info()[1]
    rng = np.random.default_rng(3)
    N = nx * ny * nz
    r = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).cuda()
    z = [torch.empty(N, dtype=torch.float32, device="cuda") for _ in range(2)]
    for s, zz in zip(solvers, z):
        s.precond(r, zz)
    torch.cuda.synchronize()
    za, zb = z[0].cpu().numpy().astype(np.float64), z[1].cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(za))
    assert np.linalg.norm(za - zb) <= 1e-5 * np.linalg.norm(zb)
    # whole solves: b in the range of A (sealed pockets need zero-sum right-hand sides)
    ref = oracle.Case(nx, ny, nz, bc=bc)
    ref.set_geometry(tri)
    b = ref.apply(rng.standard_normal(N))
    its = []
    for s in solvers:
        p = torch.zeros(N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.from_numpy(b).cuda(), p, 1e-6)
        res = np.linalg.norm(b - ref.apply(p.cpu().numpy())) / np.linalg.norm(b)
        assert st.status == 0 and res <= 1e-6 * 1.0001
        its.append(st.iters)
    assert abs(its[0] - its[1]) <= 1 + its[1] // 10, its
    for s in solvers:
        s.close()

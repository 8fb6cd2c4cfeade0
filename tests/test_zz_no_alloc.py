"""ibm_classify_noalloc: classification for callers that cannot call cudaMalloc (for example code
running under a framework that owns every device allocation through its own pool).  It must give
exactly what ibm_classify gives with a caller workspace, on consecutive calls that share the
library's fixed scratch, and reject inputs whose scratch need exceeds it.  This file is named so that
pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def L():
    from paper_2002_06206_gb300 import build
    build.build()
    from paper_2002_06206_gb300 import ibmles
    ibmles.lib()
    return ibmles


def _noalloc(L, grid, tri, cap):
    N = grid.nx * grid.ny * grid.nz
    flags = torch.full((N,), 0xAB, dtype=torch.uint8, device="cuda")
    fid = torch.full((cap,), -7, dtype=torch.int64, device="cuda")
    tlo = torch.full((cap,), np.nan, dtype=torch.float64, device="cuda")
    thi = torch.full((cap,), np.nan, dtype=torch.float64, device="cuda")
    gp = L.GeomParams(1e-9, 0.0, 0, 0)
    n_cut, n_tests = C.c_int64(), C.c_int64()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.lib().ibm_classify_noalloc(C.byref(grid), C.c_void_p(tri.data_ptr()), tri.shape[0], C.byref(gp),
                                      C.c_void_p(flags.data_ptr()), C.c_void_p(fid.data_ptr()),
                                      C.c_void_p(tlo.data_ptr()), C.c_void_p(thi.data_ptr()), cap, C.byref(n_cut),
                                      C.byref(n_tests), s)
    assert rc == L.OK, L.lib().ibm_last_error()
    n = n_cut.value
    return flags.cpu().numpy(), fid[:n].cpu().numpy(), tlo[:n].cpu().numpy(), thi[:n].cpu().numpy(), n_tests.value


def test_noalloc_classification_matches_workspace_version_twice(L):
    cases = [(64, 32, 32, W.icosphere(3, 4.0, (16.0, 16.0, 16.0))),
             (96, 48, 48, W.dirty_sphere(seed=2, radius=6.0, center=(24.0, 24.0, 24.0), subdiv=4))]
    for nx, ny, nz, soup in cases:         # two calls in a row on the shared scratch
        g = L.make_grid(nx, ny, nz)
        tri = torch.from_numpy(soup).cuda()
        ref = L.Geometry(g, tri)           # ibm_classify with its own workspace
        flags, fid, tlo, thi, nt = _noalloc(L, g, tri, cap=4 * len(soup) + 1024)
        assert np.array_equal(flags, (ref.flags.cpu().numpy() & 63))
        assert np.array_equal(fid, ref.face_id.cpu().numpy())
        assert np.array_equal(tlo, ref.t_lo.cpu().numpy())
        assert np.array_equal(thi, ref.t_hi.cpu().numpy())
        assert nt == ref.n_tests and len(fid) == ref.n_cut > 0


def test_noalloc_rejects_inputs_beyond_its_scratch(L):
    g = L.make_grid(256, 128, 128)
    gp = L.GeomParams(1e-9, 0.0, 0, 0)
    n = C.c_int64()
    rc = L.lib().ibm_classify_noalloc(C.byref(g), None, 10, C.byref(gp), None, None, None, None, 0, C.byref(n),
                                      None, None)
    assert rc == L.E_INVALID
    assert b"scratch" in L.lib().ibm_last_error()

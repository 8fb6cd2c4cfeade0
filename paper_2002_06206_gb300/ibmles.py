"""Thin Python binding of the C ABI in include/ibmles.h (argument marshalling only).

Device memory and streams come from PyTorch: every tensor passed here must be a contiguous CUDA tensor
of the dtype the call documents; its data_ptr() goes straight to the library.  Every computation runs
in the library's CUDA kernels -- there is no fallback: if libibmles.so is missing or fails to load,
importing this module's entry points raises.
"""
import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libibmles.so")

OK, E_INVALID, E_NOMEM, E_CUDA, E_NOCONV, E_NONFINITE, E_CAPACITY = range(7)
PERIODIC, INFLOW, OUTFLOW, SLIP, NOSLIP = range(5)
FP64, FP32_REFINE64 = 0, 1
CG, BICGSTAB, RBSOR = 0, 1, 2
NO_PRECOND, MULTIGRID = 0, 1
ADAMS_BASHFORTH, CRANK_NICOLSON = 0, 1


class IbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("ibmles error %d: %s" % (code, msg))
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("reserved", C.c_int32),
                ("dx", C.c_double)]


class GeomParams(C.Structure):
    _fields_ = [("eps_edge", C.c_double), ("eps_det", C.c_double), ("deadend_on", C.c_int32),
                ("reserved", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("nu", C.c_double), ("dt", C.c_double), ("u_in", C.c_double * 3), ("bc", C.c_int32 * 6),
                ("csm_on", C.c_int32), ("forcing_on", C.c_int32), ("precision", C.c_int32),
                ("solver", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("check_every", C.c_int32), ("inner_tol", C.c_double), ("sor_omega", C.c_double),
                ("precond", C.c_int32), ("mg_sweeps", C.c_int32), ("mg_omega", C.c_double),
                ("quick", C.c_double), ("integrator", C.c_int32), ("mom_max_iter", C.c_int32),
                ("mom_tol", C.c_double), ("mg_passes", C.c_int32), ("reserved", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("outer", C.c_int32), ("status", C.c_int32), ("guess_used", C.c_int32),
                ("relres", C.c_double), ("bnorm", C.c_double), ("fsum", C.c_double * 3),
                ("relres0", C.c_double), ("relres_guess", C.c_double), ("mom_iters", C.c_int32),
                ("reserved", C.c_int32)]

    def as_dict(self):
        return {"iters": self.iters, "outer": self.outer, "status": self.status, "relres": self.relres,
                "bnorm": self.bnorm, "fsum": list(self.fsum), "guess_used": self.guess_used,
                "relres0": self.relres0, "relres_guess": self.relres_guess, "mom_iters": self.mom_iters}


_lib = None

SIGNATURES = {
    "ibm_classify_workspace_bytes": (C.c_size_t, [C.c_void_p, C.c_int64]),
    "ibm_classify": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_size_t, C.c_void_p]),
    "ibm_classify_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ibm_setup": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_int64, C.c_void_p, C.c_void_p]),
    "ibm_geom_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ibm_geom_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ibm_set_boundary_velocity": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ibm_geom_destroy": (None, [C.c_void_p]),
    "les_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "les_destroy": (None, [C.c_void_p]),
    "les_init_faces": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "les_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                           C.c_void_p, C.c_void_p]),
    "les_csm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "les_predict_cn": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "les_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_int32, C.c_void_p]),
    "les_forcing": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "les_faces": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "les_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "les_correct": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p]),
    "poisson_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "poisson_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_int32,
                                C.c_void_p, C.c_void_p]),
    "forces": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "les_num_faces": (C.c_int64, [C.c_void_p]),
    "poisson_precond": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ibm_probe_fma_rate": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p]),
    "les_mg_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "les_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "les_profile_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "les_kernel_launches": (C.c_int64, [C.c_void_p]),
    "ibm_net_num_params": (C.c_int, []),
    "ibm_net_create": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ibm_net_destroy": (None, [C.c_void_p]),
    "ibm_net_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ibm_net_get_grads": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ibm_net_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "ibm_net_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_float, C.c_void_p, C.c_void_p]),
    "ibm_net_target": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                 C.c_void_p]),
    "les_attach_guess": (C.c_int, [C.c_void_p, C.c_void_p]),
    "les_last_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ibm_surface_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "ibm_surface_destroy": (None, [C.c_void_p]),
    "ibm_surface_bin_entries": (C.c_int64, [C.c_void_p]),
    "ibm_surface_pressure": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ibm_last_error": (C.c_char_p, []),
}


def lib():
    """Load libibmles.so (built by build.py); raises if it is missing -- there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libibmles.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(SIGNATURES)


def _check(rc):
    if rc != OK:
        raise IbmError(rc, lib().ibm_last_error().decode())
    return rc


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def make_grid(nx, ny, nz, dx=1.0):
    return Grid(nx, ny, nz, 0, dx)


def fma_rate(precision=FP64, stream=None):
    """Measured FMA rate of the current GPU, TFLOP/s."""
    out = C.c_double()
    _check(lib().ibm_probe_fma_rate(precision, C.byref(out), _stream(stream)))
    return out.value


def num_faces(nx, ny, nz):
    return (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1)


class Surface:
    """Triangle bins for the surface pressure with the thin-plate filter (ibm_surface_*).  Keeps a
    reference to the soup tensor, which must stay unchanged."""

    def __init__(self, grid, tri, stream=None):
        self.tri = tri
        h = C.c_void_p()
        _check(lib().ibm_surface_create(C.byref(grid), _ptr(tri, torch.float32, "tri"), tri.shape[0],
                                        _stream(stream), C.byref(h)))
        self.handle = h
        self.ntri = tri.shape[0]

    def bin_entries(self):
        return int(lib().ibm_surface_bin_entries(self.handle))

    def pressure(self, p, zfilter=True, pside=None, stream=None):
        """Returns (pside[ntri, 2] device tensor, [Fx, Fy, Fz, sides])."""
        if pside is None:
            pside = torch.empty((self.ntri, 2), dtype=torch.float64, device=p.device)
        out = (C.c_double * 4)()
        _check(lib().ibm_surface_pressure(self.handle, _ptr(p, torch.float64, "p"), int(bool(zfilter)),
                                          _ptr(pside, torch.float64, "pside"), out, _stream(stream)))
        return pside, list(out)

    def close(self):
        if getattr(self, "handle", None):
            lib().ibm_surface_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Geometry:
    """Classified triangle soup + link records (ibm_classify + ibm_setup) on the current device."""

    def __init__(self, grid, tri, eps_edge=1e-9, eps_det=0.0, deadend_on=0, stream=None, cap=None):
        self.grid = grid
        self.N = grid.nx * grid.ny * grid.nz
        self.gp = GeomParams(eps_edge, eps_det, deadend_on, 0)
        dev = torch.device("cuda", torch.cuda.current_device())
        tri = tri.to(dev, torch.float32).contiguous().view(-1, 3, 3) if isinstance(tri, torch.Tensor) \
            else torch.as_tensor(tri, dtype=torch.float32).to(dev).contiguous().view(-1, 3, 3)
        self.tri = tri
        self.flags = torch.empty(self.N, dtype=torch.uint8, device=dev)
        ws = lib().ibm_classify_workspace_bytes(C.byref(grid), tri.shape[0])
        self.workspace = torch.empty(max(int(ws), 1), dtype=torch.uint8, device=dev)
        cap = cap if cap is not None else max(1024, 2 * int(tri.shape[0]) + 1024)
        s = _stream(stream)
        while True:
            self.face_id = torch.empty(cap, dtype=torch.int64, device=dev)
            self.t_lo = torch.empty(cap, dtype=torch.float64, device=dev)
            self.t_hi = torch.empty(cap, dtype=torch.float64, device=dev)
            n_cut = C.c_int64(0)
            n_tests = C.c_int64(0)
            rc = lib().ibm_classify(C.byref(grid), _ptr(tri), tri.shape[0], C.byref(self.gp), _ptr(self.flags),
                                    _ptr(self.face_id), _ptr(self.t_lo), _ptr(self.t_hi), cap, C.byref(n_cut),
                                    C.byref(n_tests), _ptr(self.workspace), self.workspace.numel(), s)
            if rc == E_CAPACITY:
                cap = int(n_cut.value)
                continue
            _check(rc)
            break
        self.n_cut = int(n_cut.value)
        self.n_tests = int(n_tests.value)
        self.workspace = None           # 48 bytes per cell, needed by the classification only
        self.face_id = self.face_id[:self.n_cut]
        self.t_lo = self.t_lo[:self.n_cut]
        self.t_hi = self.t_hi[:self.n_cut]
        h = C.c_void_p()
        _check(lib().ibm_setup(C.byref(grid), C.byref(self.gp), _ptr(self.flags), _ptr(self.face_id),
                               _ptr(self.t_lo), _ptr(self.t_hi), self.n_cut, C.byref(h), s))
        self.handle = h
        nr, ni = C.c_int64(), C.c_int64()
        _check(lib().ibm_geom_info(h, C.byref(nr), C.byref(ni)))
        self.n_rec, self.n_inc = int(nr.value), int(ni.value)

    def export(self, stream=None):
        dev = self.flags.device
        idx = torch.empty((max(self.n_rec, 1), 6), dtype=torch.int64, device=dev)
        coef = torch.empty((max(self.n_rec, 1), 6), dtype=torch.float64, device=dev)
        cellrec = torch.empty(self.N, dtype=torch.int64, device=dev)
        _check(lib().ibm_geom_export(self.handle, _ptr(idx), _ptr(coef), _ptr(cellrec), _stream(stream)))
        return idx[:self.n_rec], coef[:self.n_rec], cellrec

    def set_boundary_velocity(self, uib=None, stream=None):
        p = None if uib is None else _ptr(uib, torch.float64, "uib")
        _check(lib().ibm_set_boundary_velocity(self.handle, p, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            lib().ibm_geom_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """One LES state (les_create): holds the workspace; fields stay caller-owned torch tensors."""

    def __init__(self, grid, nu, dt, bc, u_in=(1.0, 0.0, 0.0), precision=FP64, solver=CG, tol=1e-6,
                 max_iter=100000, check_every=16, inner_tol=1e-4, sor_omega=1.9, csm_on=1, forcing_on=1,
                 geometry=None, precond=NO_PRECOND, mg_sweeps=2, mg_omega=1.6, quick=0.0,
                 integrator=ADAMS_BASHFORTH, mom_tol=0.0, mom_max_iter=0, mg_passes=0):
        self.grid = grid
        self.N = grid.nx * grid.ny * grid.nz
        self.NF = num_faces(grid.nx, grid.ny, grid.nz)
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        self.params = Params(nu, dt, (C.c_double * 3)(*u_in), (C.c_int32 * 6)(*bc), csm_on, forcing_on,
                             precision, solver, tol, max_iter, check_every, inner_tol, sor_omega, precond,
                             mg_sweeps, mg_omega, quick, integrator, mom_max_iter, mom_tol, mg_passes, 0)
        self.geometry = geometry
        h = C.c_void_p()
        _check(lib().les_create(C.byref(grid), C.byref(self.params),
                                geometry.handle if geometry is not None else None, C.byref(h)))
        self.handle = h

    def fields(self, u0):
        """Allocate the state tensors (u, U, p, H) on the device from a cell velocity u0[3, N]."""
        dev = torch.device("cuda", torch.cuda.current_device())
        u = torch.as_tensor(u0).to(dev, self.dtype).reshape(-1).contiguous().clone()
        U = torch.empty(self.NF, dtype=self.dtype, device=dev)
        self.init_faces(u, U)
        p = torch.zeros(self.N, dtype=torch.float64, device=dev)
        H = torch.zeros(3 * self.N, dtype=self.dtype, device=dev)
        return {"u": u, "U": U, "p": p, "H": H, "n": 0}

    def init_faces(self, u, U, stream=None):
        _check(lib().les_init_faces(self.handle, _ptr(u, self.dtype, "u"), _ptr(U, self.dtype, "U"), _stream(stream)))

    def step(self, st, stream=None):
        stats = Stats()
        _check(lib().les_step(self.handle, _ptr(st["u"], self.dtype, "u"), _ptr(st["U"], self.dtype, "U"),
                              _ptr(st["p"], torch.float64, "p"), _ptr(st["H"], self.dtype, "H"),
                              int(st["n"] == 0), C.byref(stats), _stream(stream)))
        st["n"] += 1
        return stats

    def step_raw(self, u, U, p, H, first, stream=None, stats=None):
        return lib().les_step(self.handle, _ptr(u), _ptr(U), _ptr(p), _ptr(H), int(first),
                              None if stats is None else C.byref(stats), _stream(stream))

    def csm(self, u, nut, stream=None):
        _check(lib().les_csm(self.handle, _ptr(u, self.dtype, "u"), _ptr(nut, self.dtype, "nut"), _stream(stream)))

    def predict(self, u, U, nut, Hprev, H, ustar, first, stream=None):
        _check(lib().les_predict(self.handle, _ptr(u, self.dtype), _ptr(U, self.dtype), _ptr(nut, self.dtype),
                                 _ptr(Hprev, self.dtype), _ptr(H, self.dtype), _ptr(ustar, self.dtype), int(first),
                                 _stream(stream)))

    def predict_cn(self, u, U, nut, H, ustar, stream=None):
        it = C.c_int32()
        _check(lib().les_predict_cn(self.handle, _ptr(u, self.dtype), _ptr(U, self.dtype), _ptr(nut, self.dtype),
                                    _ptr(H, self.dtype), _ptr(ustar, self.dtype), C.byref(it), _stream(stream)))
        return it.value

    def forcing(self, ustar, stream=None):
        fs = (C.c_double * 3)()
        _check(lib().les_forcing(self.handle, _ptr(ustar, self.dtype), fs, _stream(stream)))
        return list(fs)

    def faces(self, ustar, Ustar, stream=None):
        _check(lib().les_faces(self.handle, _ptr(ustar, self.dtype), _ptr(Ustar, self.dtype), _stream(stream)))

    def rhs(self, Ustar, b, stream=None):
        _check(lib().les_rhs(self.handle, _ptr(Ustar, self.dtype), _ptr(b, torch.float64), _stream(stream)))

    def correct(self, ustar, Ustar, p, u, U, stream=None):
        _check(lib().les_correct(self.handle, _ptr(ustar, self.dtype), _ptr(Ustar, self.dtype),
                                 _ptr(p, torch.float64), _ptr(u, self.dtype), _ptr(U, self.dtype), _stream(stream)))

    def apply(self, p, Ap, stream=None):
        _check(lib().poisson_apply(self.handle, _ptr(p, torch.float64), _ptr(Ap, torch.float64), _stream(stream)))

    def solve(self, b, p, tol, max_it=100000, solver=CG, stream=None, check=True):
        stats = Stats()
        rc = lib().poisson_solve(self.handle, _ptr(b, torch.float64), _ptr(p, torch.float64), tol, max_it, solver,
                                 C.byref(stats), _stream(stream))
        if check:
            _check(rc)
        return stats if check else (rc, stats)

    def forces(self, tri, p, u=None, stream=None):
        """[0:3] pressure force, [3] triangles used, [4:7] viscous force, [7] links used,
        [8:11] momentum-forcing estimate of the last step, [11] 0."""
        out = (C.c_double * 12)()
        _check(lib().forces(self.handle, _ptr(tri, torch.float32), tri.shape[0], _ptr(p, torch.float64),
                            None if u is None else _ptr(u, self.dtype, "u"), out, _stream(stream)))
        return list(out)

    def precond(self, r, z, stream=None):
        """z = one multigrid V-cycle applied to r (working precision)."""
        _check(lib().poisson_precond(self.handle, _ptr(r, self.dtype, "r"), _ptr(z, self.dtype, "z"), _stream(stream)))

    def mg_info(self):
        """(levels, fused fine passes, unknowns per level)."""
        out = (C.c_int64 * 18)()
        _check(lib().les_mg_info(self.handle, out, 18))
        return int(out[0]), bool(out[1]), [int(out[2 + l]) for l in range(min(int(out[0]), 16))]

    PROFILE_SLOTS = ("csm", "predict", "forcing", "faces", "rhs", "residual", "cg_dir_spmv", "cg_update",
                     "correct", "sor", "mg_fine", "mg_transfer", "mg_coarse", "momentum")

    def profile(self, on):
        _check(lib().les_profile(self.handle, int(on)))

    def profile_read(self):
        ms = (C.c_double * len(self.PROFILE_SLOTS))()
        n = (C.c_int64 * len(self.PROFILE_SLOTS))()
        _check(lib().les_profile_read(self.handle, ms, n))
        return {k: (ms[q], n[q]) for q, k in enumerate(self.PROFILE_SLOTS)}

    def kernel_launches(self):
        return int(lib().les_kernel_launches(self.handle))

    def attach_guess(self, net):
        _check(lib().les_attach_guess(self.handle, net.handle if net is not None else None))
        self.net = net

    def last_rhs(self, b, stream=None):
        _check(lib().les_last_rhs(self.handle, _ptr(b, torch.float64), _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            lib().les_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """Learned initial guess of the pressure solve (ibm_net_*): creation, forward, training steps."""

    def __init__(self, params=None):
        import numpy as np
        self.n_params = int(lib().ibm_net_num_params())
        h = None
        if params is not None:
            arr = np.ascontiguousarray(params, dtype=np.float32)
            assert arr.size == self.n_params
            h = arr.ctypes.data_as(C.c_void_p)
        handle = C.c_void_p()
        _check(lib().ibm_net_create(h, C.byref(handle)))
        self.handle = handle

    def params(self):
        import numpy as np
        out = np.zeros(self.n_params, np.float32)
        _check(lib().ibm_net_get_params(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def grads(self):
        import numpy as np
        out = np.zeros(self.n_params, np.float32)
        _check(lib().ibm_net_get_grads(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def forward(self, grid, b, p, pprev, flags=None, stream=None):
        N = grid.nx * grid.ny * grid.nz
        out = torch.empty(N, dtype=torch.float32, device=b.device)
        s = C.c_double()
        _check(lib().ibm_net_forward(self.handle, C.byref(grid), _ptr(b, torch.float64), _ptr(p, torch.float64),
                                     _ptr(pprev, torch.float64), _ptr(flags, torch.uint8) if flags is not None else None,
                                     _ptr(out, torch.float32), C.byref(s), _stream(stream)))
        return out, s.value

    def target(self, grid, pnext, p, pprev, s, stream=None):
        """(p^{n+1} - 2 p^n + p^{n-1}) / s in FP32, formed on the device (ibm_net_target)."""
        N = grid.nx * grid.ny * grid.nz
        out = torch.empty(N, dtype=torch.float32, device=p.device)
        _check(lib().ibm_net_target(C.byref(grid), _ptr(pnext, torch.float64), _ptr(p, torch.float64),
                                    _ptr(pprev, torch.float64), C.c_double(s), _ptr(out, torch.float32),
                                    _stream(stream)))
        return out

    def train_step(self, grid, b, p, pprev, target, lr, flags=None, stream=None):
        loss = C.c_double()
        _check(lib().ibm_net_train_step(self.handle, C.byref(grid), _ptr(b, torch.float64), _ptr(p, torch.float64),
                                        _ptr(pprev, torch.float64),
                                        _ptr(flags, torch.uint8) if flags is not None else None,
                                        _ptr(target, torch.float32), C.c_float(lr), C.byref(loss), _stream(stream)))
        return loss.value

    def close(self):
        if getattr(self, "handle", None):
            lib().ibm_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

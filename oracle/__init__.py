"""Python front end of the FP64 CPU oracle (ibm_oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain definition of the method that the CUDA
library is checked against, and the timed CPU baseline.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this module; the product package never does.

Arrays follow the oracle's layout: cell fields u[3, nz, ny, nx] (component-major, x fastest), faces
as one concatenated vector Ux | Uy | Uz, soups float32 [ntri, 3, 3] in grid units.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BICGSTAB, CG, RBSOR = 0, 1, 2

RECORD_DTYPE = np.dtype([
    ("cell", np.int64), ("far", np.int64), ("opp", np.int64), ("axis", np.int64),
    ("side", np.int64), ("branch", np.int64), ("d", np.float64), ("c_ib", np.float64),
    ("c_p", np.float64), ("c_o", np.float64), ("w_fluid", np.float64), ("w_ghost", np.float64),
    ("uib", np.float64, (3,)),
])


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("pad_", C.c_int32),
                ("dx", C.c_double)]


class Params(C.Structure):
    _fields_ = [("nu", C.c_double), ("dt", C.c_double), ("u_in", C.c_double * 3),
                ("bc", C.c_int32 * 6), ("csm_on", C.c_int32), ("forcing_on", C.c_int32),
                ("deadend_on", C.c_int32), ("integrator", C.c_int32), ("quick", C.c_double),
                ("mom_tol", C.c_double), ("mom_maxit", C.c_int32), ("pad_", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("relres", C.c_double),
                ("bnorm", C.c_double), ("fsum", C.c_double * 3), ("mom_iters", C.c_int32),
                ("pad_", C.c_int32)]


def build(force=False):
    """Compile the oracle with gcc (no FMA contraction: the predicate must be reproducible)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ibm_oracle.h"))):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        i64 = C.c_int64
        L.or_classify.restype = i64
        L.or_classify.argtypes = [P, P, i64, C.c_double, C.c_double, P, P, P, P, i64, P, P]
        L.or_mt_disagreements.restype = i64
        L.or_mt_disagreements.argtypes = [P, P, i64, C.c_double, C.c_double]
        L.or_setup.restype = i64
        L.or_setup.argtypes = [P, P, P, P, P, i64, P, P, P, P]
        L.or_velocity_across.restype = C.c_double
        L.or_velocity_across.argtypes = [P, P, P, P, P, P, C.c_int, i64, C.c_int, C.c_int]
        L.or_csm.argtypes = [P, P, P, P, P, P, P]
        L.or_predict.argtypes = [P, P, P, P, P, P, P, P, P, P, P, C.c_int]
        L.or_momentum_operator.argtypes = [P, P, P, P, P, P, P, P, C.c_int, P]
        L.or_predict_cn.restype = C.c_int
        L.or_predict_cn.argtypes = [P, P, P, P, P, P, P, P, P, P, C.c_double, C.c_int32]
        L.or_forcing.argtypes = [P, P, P, P, i64, P, P, P]
        L.or_faces.argtypes = [P, P, P, P, P, P, P]
        L.or_rhs.argtypes = [P, P, P, P]
        L.or_apply.argtypes = [P, P, P, P, P]
        L.or_solve.restype = C.c_int
        L.or_solve.argtypes = [P, P, P, P, P, C.c_double, C.c_int32, C.c_int32, C.c_double, P]
        L.or_correct.argtypes = [P, P, P, P, P, P, P, P]
        L.or_step.restype = C.c_int
        L.or_step.argtypes = [P, P, P, P, i64, P, P, P, P, P, C.c_int, C.c_double, C.c_int32,
                              C.c_int32, C.c_double, P]
        L.or_forces.argtypes = [P, P, i64, P, P]
        L.or_surface_pressure.argtypes = [P, P, i64, P, C.c_int, P, P]
        L.or_viscous_force.argtypes = [P, P, P, P, i64, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _chk(a, dtype):
    assert a.dtype == dtype and a.flags.c_contiguous, (a.dtype, dtype)
    return a


def nfaces(nx, ny, nz):
    return (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1)


def split_faces(U, nx, ny, nz):
    n0 = (nx + 1) * ny * nz
    n1 = nx * (ny + 1) * nz
    return (U[:n0].reshape(nz, ny, nx + 1), U[n0:n0 + n1].reshape(nz, ny + 1, nx),
            U[n0 + n1:].reshape(nz + 1, ny, nx))


class Case:
    """Grid + physics parameters + (optionally) a classified geometry, all held by the oracle."""

    def __init__(self, nx, ny, nz, dx=1.0, nu=0.0, dt=1.0, bc=(0, 0, 0, 0, 0, 0),
                 u_in=(1.0, 0.0, 0.0), csm_on=1, forcing_on=1, deadend_on=0, quick=0.0,
                 integrator=0, mom_tol=1e-12, mom_maxit=1000):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz
        self.NF = nfaces(nx, ny, nz)
        self.g = Grid(nx, ny, nz, 0, dx)
        self.pr = Params(nu, dt, (C.c_double * 3)(*u_in), (C.c_int32 * 6)(*bc), csm_on,
                         forcing_on, deadend_on, integrator, quick, mom_tol, mom_maxit, 0)
        self.flags = np.zeros(self.N, np.uint8)
        self.rec = np.zeros(0, RECORD_DTYPE)
        self.cellrec = np.full(self.N, -1, np.int64)
        self.inc = np.zeros(0, np.int64)
        self.cut = (np.zeros(0, np.int64), np.zeros(0), np.zeros(0))

    @classmethod
    def from_config(cls, cfg):
        return cls(cfg.nx, cfg.ny, cfg.nz, cfg.dx, cfg.nu, cfg.dt, cfg.bc, cfg.u_in, cfg.csm_on,
                   cfg.forcing_on, cfg.deadend_on, cfg.quick, cfg.integrator)

    # -- geometry ------------------------------------------------------------------------------
    def classify(self, tri, eps_edge=1e-9, eps_det=0.0):
        tri = np.ascontiguousarray(tri, np.float32)
        L = lib()
        cap = 1 << 16
        while True:
            fid = np.zeros(cap, np.int64)
            tlo = np.zeros(cap)
            thi = np.zeros(cap)
            sk = np.zeros(1, np.int64)
            nt = np.zeros(1, np.int64)
            n = L.or_classify(C.byref(self.g), _p(tri), len(tri), eps_edge, eps_det, _p(self.flags),
                              _p(fid), _p(tlo), _p(thi), cap, _p(sk), _p(nt))
            if n < 0:
                raise MemoryError("oracle classification")
            if n <= cap:
                break
            cap = int(n)
        self.cut = (fid[:n].copy(), tlo[:n].copy(), thi[:n].copy())
        self.n_skipped = int(sk[0])
        self.n_tests = int(nt[0])
        return self.cut

    def setup(self):
        fid, tlo, thi = self.cut
        n = len(fid)
        self.rec = np.zeros(2 * n, RECORD_DTYPE)
        inc = np.zeros(self.N, np.int64)
        ninc = np.zeros(1, np.int64)
        k = lib().or_setup(C.byref(self.g), _p(self.flags), _p(fid), _p(tlo), _p(thi), n,
                           _p(self.rec), _p(self.cellrec), _p(inc), _p(ninc))
        if k < 0:
            raise RuntimeError("oracle setup: cut face missing from the list")
        self.rec = self.rec[:k]
        self.inc = inc[:int(ninc[0])].copy()
        return self.rec

    def set_geometry(self, tri, eps_edge=1e-9, eps_det=0.0):
        self.classify(tri, eps_edge, eps_det)
        return self.setup()

    # -- operators -----------------------------------------------------------------------------
    def _args(self):
        return C.byref(self.g), C.byref(self.pr), _p(self.flags), _p(self.rec), _p(self.cellrec)

    def velocity_across(self, u, comp, P, axis, side):
        u = _chk(np.ascontiguousarray(u, np.float64), np.float64)
        return lib().or_velocity_across(*self._args(), _p(u), comp, int(P), axis, side)

    def csm(self, u):
        u = np.ascontiguousarray(u, np.float64)
        nut = np.zeros(self.N)
        lib().or_csm(*self._args(), _p(u), _p(nut))
        return nut

    def predict(self, u, U, nut, Hprev, first_step):
        u = np.ascontiguousarray(u, np.float64)
        U = np.ascontiguousarray(U, np.float64)
        nut = np.ascontiguousarray(nut, np.float64)
        Hprev = np.ascontiguousarray(Hprev, np.float64)
        H = np.zeros(3 * self.N)
        us = np.zeros(3 * self.N)
        lib().or_predict(*self._args(), _p(u), _p(U), _p(nut), _p(Hprev), _p(H), _p(us),
                         int(first_step))
        return H, us

    def momentum_operator(self, u, U, nut, hom=False):
        """L(u) (per unit volume) with U and nu_t fixed; hom drops the wall and inflow velocities."""
        u = np.ascontiguousarray(u, np.float64)
        U = np.ascontiguousarray(U, np.float64)
        nut = np.ascontiguousarray(nut, np.float64)
        out = np.zeros(3 * self.N)
        lib().or_momentum_operator(*self._args(), _p(u), _p(U), _p(nut), int(bool(hom)), _p(out))
        return out

    def predict_cn(self, u, U, nut, tol=1e-12, maxit=1000):
        """Crank-Nicolson predictor; returns (H = L(u^n), u*, BiCGStab iterations or -1)."""
        u = np.ascontiguousarray(u, np.float64)
        U = np.ascontiguousarray(U, np.float64)
        nut = np.ascontiguousarray(nut, np.float64)
        H = np.zeros(3 * self.N)
        us = np.zeros(3 * self.N)
        it = lib().or_predict_cn(*self._args(), _p(u), _p(U), _p(nut), _p(H), _p(us), tol, maxit)
        return H, us, it

    def forcing(self, ustar):
        ustar = np.ascontiguousarray(ustar, np.float64)
        out = np.zeros(3 * self.N)
        fs = np.zeros(3)
        lib().or_forcing(C.byref(self.g), C.byref(self.pr), _p(self.flags), _p(self.rec),
                         len(self.rec), _p(ustar), _p(out), _p(fs))
        return out, fs

    def faces(self, ustar):
        ustar = np.ascontiguousarray(ustar, np.float64)
        U = np.zeros(self.NF)
        lib().or_faces(C.byref(self.g), C.byref(self.pr), _p(self.flags), _p(self.rec), _p(self.cellrec),
                       _p(ustar), _p(U))
        return U

    def rhs(self, Ustar):
        Ustar = np.ascontiguousarray(Ustar, np.float64)
        b = np.zeros(self.N)
        lib().or_rhs(C.byref(self.g), C.byref(self.pr), _p(Ustar), _p(b))
        return b

    def apply(self, p):
        p = np.ascontiguousarray(p, np.float64)
        Ap = np.zeros(self.N)
        lib().or_apply(C.byref(self.g), C.byref(self.pr), _p(self.flags), _p(p), _p(Ap))
        return Ap

    def solve(self, b, p0=None, tol=1e-10, maxit=100000, solver=BICGSTAB, omega=1.0):
        b = np.ascontiguousarray(b, np.float64)
        p = np.zeros(self.N) if p0 is None else np.array(p0, np.float64).reshape(-1).copy()
        st = Stats()
        lib().or_solve(C.byref(self.g), C.byref(self.pr), _p(self.flags), _p(b), _p(p), tol,
                       maxit, solver, omega, C.byref(st))
        return p, st

    def correct(self, ustar, Ustar, p):
        ustar = np.ascontiguousarray(ustar, np.float64)
        Ustar = np.ascontiguousarray(Ustar, np.float64)
        p = np.ascontiguousarray(p, np.float64)
        u = np.zeros(3 * self.N)
        U = np.zeros(self.NF)
        lib().or_correct(C.byref(self.g), C.byref(self.pr), _p(self.flags), _p(ustar), _p(Ustar),
                         _p(p), _p(u), _p(U))
        return u, U

    def step(self, state, tol=1e-10, maxit=100000, solver=BICGSTAB, omega=1.0):
        """Advance `state` (dict with u, U, p, H, n) by one fractional step in place."""
        st = Stats()
        for k in ("u", "U", "p", "H"):
            assert state[k].dtype == np.float64 and state[k].flags.c_contiguous
        status = lib().or_step(*self._args()[:4], len(self.rec), _p(self.cellrec),
                               _p(state["u"]), _p(state["U"]), _p(state["p"]), _p(state["H"]),
                               int(state["n"] == 0), tol, maxit, solver, omega, C.byref(st))
        state["n"] += 1
        return st

    def initial_state(self, u0):
        """State at n = 0: cell velocity u0, face velocity from the face rule, p = 0, H = 0."""
        u = np.ascontiguousarray(u0, np.float64).reshape(-1).copy()
        return {"u": u, "U": self.faces(u), "p": np.zeros(self.N), "H": np.zeros(3 * self.N), "n": 0}

    def forces(self, tri, p):
        tri = np.ascontiguousarray(tri, np.float32)
        p = np.ascontiguousarray(p, np.float64)
        out = np.zeros(4)
        lib().or_forces(C.byref(self.g), _p(tri), len(tri), _p(p), _p(out))
        return out

    def viscous_force(self, u):
        """Viscous force on the body from the cut links: [Fx, Fy, Fz, links]."""
        u = np.ascontiguousarray(u, np.float64)
        out = np.zeros(4)
        lib().or_viscous_force(C.byref(self.g), C.byref(self.pr), _p(self.flags), _p(self.rec), len(self.rec),
                               _p(self.cellrec), _p(u), _p(out))
        return out

    def surface_pressure(self, tri, p, zfilter=True):
        """Per-triangle (front, back) Shepard pressures (NaN where a side has no point) and the force
        summed over the sides that have a value; zfilter applies the thin-plate filter."""
        tri = np.ascontiguousarray(tri, np.float32)
        p = np.ascontiguousarray(p, np.float64)
        pside = np.zeros((len(tri), 2))
        out = np.zeros(4)
        lib().or_surface_pressure(C.byref(self.g), _p(tri), len(tri), _p(p), int(bool(zfilter)), _p(pside),
                                  _p(out))
        return pside, out

    def mt_disagreements(self, tri, eps_edge=1e-9, eps_det=0.0):
        tri = np.ascontiguousarray(tri, np.float32)
        return int(lib().or_mt_disagreements(C.byref(self.g), _p(tri), len(tri), eps_edge, eps_det))

"""Throughput of the immersed-boundary LES step on one GB300 (or N independent replicas).

A step is one fractional time step of the whole hot path (CSM eddy viscosity, Crank-Nicolson predictor
with 10 % QUICK and its momentum BiCGStab, IB forcing, face velocities, RHS, pressure solve to
||b - A p|| / ||b|| <= 1e-6 by multigrid-preconditioned CG, correction), FP32 stencils with FP64
iterative refinement of the pressure.  The headline workload is the largest one that fits one GPU:
the 1024 x 512 x 384 (201 M cells) vehicle-like assembly of ~2 M dirty triangles on a no-slip floor,
with the dead-end filter on.  The same line carries the 512 x 256 x 256 cube-and-plate workload
(plain and with the learned initial guess in the same window; the guess is trained on solver
snapshots of the 256 x 128 x 128 dirty sphere), the pure-FP64 path (64 x 32 x 32 sphere, 50 steps to
1e-10, and the cube-and-plate), and the oracle timed on the host cores.
Metric: Mcell-steps/s = cells * steps / seconds.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica on its own GPU (the step has no data exchange on one
grid; see the design notes), timing is max over ranks, and value is the whole-job total.
`--impl reference` times the FP64 CPU oracle instead (rank 0 only), on a bounded sample.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOAD = "vehicle_1024x512x384"
SECONDARY = "cube_plate_512x256x256"
TRAIN_WORKLOAD = "dirty_sphere_256x128x128"
FP64_SMALL = "sphere_64x32x32"
METRIC = "Mcell-steps/s at Poisson rel. residual 1e-6, learned+mixed vs plain, %HBM roof"
UNIT = "Mcell-steps/s"
FALLBACK_HBM = 6800.0
# CG iterations per step charged to the oracle's sample step (about the GPU's measured mean of
# multigrid-preconditioned CG on the vehicle workload; the sample runs exactly this many)
I_REF_DEFAULT = 18


def bytes_per_cell(s, integrator="cn", sweeps=2, fused=False):
    """Algorithmic bytes per cell of each timed kernel group (s = bytes of a working-precision value):
    every array a pass needs is read once and every array it produces is written once."""
    if fused:
        # two launches per V-cycle: pre-smoothing + restriction reads r and the flags and writes z and
        # b_1 (level 1 ~ N/8 values); post-smoothing + (r, z) reads r, z and the flags and writes z
        mg_fine = ((2 * s + 1 + s / 8.0) + (3 * s + 1)) / 2.0
        mg_transfer = 2 * s + 1 + (s + 4) / 8.0          # prolongation: z, flags, x_1, offsets -> z
    else:
        # fine-grid red-black passes of one V-cycle: the first reads r and the flags and writes z (z = 0
        # before it); every other pass reads r, z and the flags and writes z (both colours share lines)
        n_pass = 4 * sweeps
        mg_fine = ((2 * s + 1) + (n_pass - 1) * (3 * s + 1)) / n_pass
        # restriction (r, z, flags -> b_1) and prolongation (z, flags, x_1 -> z), level 1 ~ N/8 values
        mg_transfer = 2 * s + 1 + (s + 4) / 8.0
    return {
        "csm": 4 * s + 1,                 # u (3) + flags -> nu_t
        # AB2: u, U, nu_t, Hprev, flags -> H, u*;  CN: u, U, nu_t, flags -> H, r, r_hat, delta
        "predict": (16 * s + 1) if integrator == "ab2" else (19 * s + 1),
        "faces": 6 * s + 1,               # u*, flags -> U*
        "rhs": 3 * s + 8,                 # U* -> b (fp64)
        "residual": 8 + 8 + 1 + s,        # b, x (fp64), flags -> r
        "cg_dir_spmv": 4 * s + 1,         # z, p_old, flags -> p, q
        "cg_update": 6 * s,               # x, p, r, q -> x, r
        "correct": 12 * s + 9,            # u*, U*, p (fp64), flags -> u, U
        "mg_fine": mg_fine,
        "mg_transfer": mg_transfer,
    }


# the kernel behind each single-kernel group (FP32 path with nx a multiple of 4)
GROUP_KERNEL = {"csm": "k_csm", "predict": "k_cn_begin (tiled + general)", "faces": "k_faces",
                "rhs": "k_rhs", "residual": "k_residual", "cg_dir_spmv": "k_cg_dir_spmv_x4",
                "cg_update": "k_cg_update", "correct": "k_correct_cells + k_correct_faces",
                "mg_fine": "k_mg_smooth0_x4", "mg_transfer": "k_mg_restrict0_x4 + k_mg_prolong0_x4"}
GROUP_KERNEL_FUSED = {"mg_fine": "k_mg_pre_fused + k_mg_post_fused", "mg_transfer": "k_mg_prolong0_x4"}


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def src_hash(files=None):
    """Hash of the CUDA sources (all of them, or the named files of csrc/)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2002_06206_gb300", "csrc")
    for f in sorted(files if files is not None else os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key, workload=WORKLOAD):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this workload and the
    sources that define that kernel (the files listed with it) are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        with open(path) as f:
            d = json.load(f)
        k = d["kernels"].get(kernel_key)
        if not k or k.get("source_hash") != src_hash(k["files"]):
            return None
        if k.get("workload", workload) != workload:
            return None
        return k.get("dram_bytes_per_launch_full_size")
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = os.path.join("/tmp", "bench_clocks_%d_%d.csv" % (os.getpid(), int(time.time() * 1e3)))

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 8:
                    continue
                try:
                    rows.append((float(p[0]), float(p[1]), float(p[2]), p[3], p[4], p[5], p[6], p[7]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([r[0] for r in rows])
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[q] for r in rows for q in range(4) if r[4 + q].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][1]), "samples": len(rows),
                "power_w_max": float(max(r[2] for r in rows)), "reasons": reasons}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_config(name, args, precision="fp32"):
    """The static description of a workload (the same dict in both arms of the benchmark)."""
    cfg = W.get_config(name)
    return {"workload": name, "cells": cfg.ncell, "grid": [cfg.nx, cfg.ny, cfg.nz],
            "precision": "fp32 stencils and cg, fp64 residual refinement" if precision == "fp32" else "fp64",
            "solver": "cg + connected-part multigrid V-cycle" if args.precond == "mg" else "cg",
            "tol": cfg.tol if precision == "fp32" else 1e-10,
            "integrator": "crank-nicolson" if args.integrator == "cn" else "adams-bashforth-2",
            "quick": args.quick, "mg_sweeps": args.mg_sweeps, "mg_omega": args.mg_omega,
            "deadend_filter": bool(cfg.deadend_on), "parallelism": "single",
            "l2": "state far larger than L2 (tens of GB vs 126 MB); no flush needed"
            if cfg.ncell >= 33554432 else "state larger than L2 (~0.4 GB vs 126 MB)"}


# ------------------------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on bounded samples of the same workload

def slab_shape(cfg):
    """Planes and rows of the oracle's sample of a workload: the largest workload takes one plane and the
    middle quarter of the rows (through the bodies), so that a sample step lasts a few seconds; the others
    take two whole planes."""
    if cfg.ncell > 50_000_000:
        return 1, cfg.ny // 4
    return 2, cfg.ny


def _slab_case(cfg, planes, k0, quick, rows=None):
    import oracle
    rows = cfg.ny if rows is None else rows
    j0 = (cfg.ny - rows) // 2
    tri = cfg.soup().copy()
    tri[..., 2] -= k0
    tri[..., 1] -= j0
    case = oracle.Case(cfg.nx, rows, planes, cfg.dx, cfg.nu, cfg.dt, cfg.bc, cfg.u_in, cfg.csm_on,
                       cfg.forcing_on, cfg.deadend_on, quick)
    case.set_geometry(tri)
    u = W.initial_fields(W.Config("slab", cfg.nx, rows, planes, 0, 0, 0, 0, 0, cfg.bc, seed=cfg.seed)).reshape(-1)
    return case, u


def slab_k0(cfg, planes):
    """First plane of the sample slab: through the bodies (a quarter of the height on a floor, the
    middle otherwise)."""
    if cfg.bc[4] == 4:                          # no-slip floor
        return max(0, min(cfg.nz - planes, cfg.nz // 4 - planes // 2))
    return cfg.nz // 2 - planes // 2


class OracleSample:
    """An oracle step on a z-slab of a workload (`planes` planes): CSM, the Crank-Nicolson predictor with
    its momentum BiCGStab (or AB2), forcing, faces, RHS, exactly `iters` CG iterations of the pressure
    solve, correction -- the per-cell work of a full step.  The slab is classified once; every step()
    starts from the same initial field and times the step alone."""

    def __init__(self, name, iters, planes, k0=None, integrator="cn", quick=0.1, mom_tol=1e-6, rows=None):
        cfg = W.get_config(name)
        self.k0 = slab_k0(cfg, planes) if k0 is None else k0
        self.case, self.u = _slab_case(cfg, planes, self.k0, quick, rows)
        self.iters, self.integrator, self.mom_tol, self.planes = int(iters), integrator, mom_tol, planes

    def step(self):
        import oracle
        case, u = self.case, self.u
        U = case.faces(u)
        t0 = time.perf_counter()
        nut = case.csm(u)
        if self.integrator == "cn":
            H, us, _ = case.predict_cn(u, U, nut, tol=self.mom_tol)
        else:
            H, us = case.predict(u, U, nut, np.zeros_like(u), True)
        us2, _ = case.forcing(us)
        Us = case.faces(us2)
        b = case.rhs(Us)
        p, st = case.solve(b, None, tol=1e-30, maxit=self.iters, solver=oracle.CG)
        case.correct(us2, Us, p)
        t1 = time.perf_counter()
        return {"cells": case.N, "seconds": t1 - t0, "k0": self.k0, "planes": self.planes, "cg_iters": st.iters}


def oracle_sample_step(name, iters, planes, k0=None, integrator="cn", quick=0.1, mom_tol=1e-6, rows=None):
    return OracleSample(name, iters, planes, k0, integrator, quick, mom_tol, rows).step()


def _sample_worker(args):
    name, iters, planes, k0, integrator, quick, rows = args
    return oracle_sample_step(name, iters, planes, k0, integrator, quick, rows=rows)


def oracle_full_run(name):
    """The whole small workload on the oracle, as the workload defines it (every step to its tolerance
    with the oracle's BiCGStab); returns (cells, steps, seconds)."""
    import oracle
    cfg = W.get_config(name)
    case = oracle.Case.from_config(cfg)
    case.set_geometry(cfg.soup())
    st = case.initial_state(W.initial_fields(cfg))
    t0 = time.perf_counter()
    for _ in range(cfg.steps):
        case.step(st, tol=cfg.tol)
    return cfg.ncell, cfg.steps, time.perf_counter() - t0


def _full_run_worker(name):
    return oracle_full_run(name)


def _sample_desc(name, planes, iters, integrator, rows=None):
    cfg = W.get_config(name)
    rows = cfg.ny if rows is None else rows
    return ("oracle (FP64, plain C) step on a %dx%dx%d slab of %s (the middle %d of %d rows, %d plane%s through "
            "the bodies): csm, %s predictor, forcing, faces, rhs, %d CG iterations (about the GPU's "
            "multigrid-preconditioned count per step), correction; value = slab cells / seconds of that step"
            % (cfg.nx, rows, planes, name, rows, cfg.ny, planes, "" if planes == 1 else "s",
               "Crank-Nicolson (momentum BiCGStab to 1e-6)" if integrator == "cn" else "AB2", iters))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    I = int(os.environ.get("IBM_REF_ITERS", I_REF_DEFAULT))
    planes, rows = slab_shape(W.get_config(args.workload))
    sample = OracleSample(args.workload, I, planes, integrator=args.integrator, quick=args.quick, rows=rows)
    for _ in range(args.warmup):
        sample.step()
    samples = [sample.step() for _ in range(args.steps)]
    secs = float(sum(s["seconds"] for s in samples))
    cells = samples[0]["cells"]
    value = cells * args.steps / secs / 1e6
    cores = 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": _sample_desc(args.workload, planes, I, args.integrator, rows),
                             "host_cores": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# GPU measurements

def time_classify(L, torch, name=WORKLOAD, repeats=5):
    """ibm_classify on the vehicle-like assembly (separate from the step): median of `repeats` runs,
    in predicate tests per second; the soup and buffers are resident on the device."""
    import ctypes as C
    cfg = W.get_config(name)
    tri = torch.from_numpy(cfg.soup()).cuda()
    g = L.make_grid(cfg.nx, cfg.ny, cfg.nz, cfg.dx)
    lib = L.lib()
    N = cfg.ncell
    ws = torch.empty(lib.ibm_classify_workspace_bytes(C.byref(g), tri.shape[0]), dtype=torch.uint8, device="cuda")
    flags = torch.empty(N, dtype=torch.uint8, device="cuda")
    cap = 4 * tri.shape[0] + 1024
    fid = torch.empty(cap, dtype=torch.int64, device="cuda")
    tlo = torch.empty(cap, dtype=torch.float64, device="cuda")
    thi = torch.empty(cap, dtype=torch.float64, device="cuda")
    gp = L.GeomParams(1e-9, 0.0, cfg.deadend_on, 0)
    stream = torch.cuda.current_stream()
    times, ncut, ntests = [], C.c_int64(), C.c_int64()
    for _ in range(repeats + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = lib.ibm_classify(C.byref(g), C.c_void_p(tri.data_ptr()), tri.shape[0], C.byref(gp),
                              C.c_void_p(flags.data_ptr()), C.c_void_p(fid.data_ptr()), C.c_void_p(tlo.data_ptr()),
                              C.c_void_p(thi.data_ptr()), cap, C.byref(ncut), C.byref(ntests),
                              C.c_void_p(ws.data_ptr()), ws.numel(), C.c_void_p(stream.cuda_stream))
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            return {"workload": name, "error": lib.ibm_last_error().decode()}
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times[1:]))
    return {"workload": name, "triangles": int(tri.shape[0]), "cells": N, "ms": ms,
            "predicate_tests": int(ntests.value), "mtests_per_s": ntests.value / (ms * 1e-3) / 1e6,
            "links_per_s": 3 * N / (ms * 1e-3), "cut_faces": int(ncut.value),
            "note": "median of %d after one warm-up; includes the per-face table fill, compaction and the "
                    "host read of the cut count" % repeats}


def net_init(seed=0, scale=0.05):
    """Initial parameters of the guess network (layout of include/ibmles.h)."""
    rng = np.random.default_rng(seed)
    w = [rng.standard_normal(8 * 27 * 8), rng.standard_normal(8 * 27 * 8), rng.standard_normal(27 * 8)]
    return np.concatenate([x * scale for x in w] + [np.zeros(17)]).astype(np.float32)


def make_solver(L, torch, name, args, precision=None, geo=None, own_scheme=False):
    """Solver of a workload with the benchmark's scheme (Crank-Nicolson, QUICK blend), or with the
    workload's own integrator and blend (own_scheme)."""
    cfg = W.get_config(name)
    integ = cfg.integrator if own_scheme else (1 if args.integrator == "cn" else 0)
    quick = cfg.quick if own_scheme else args.quick
    g = L.make_grid(cfg.nx, cfg.ny, cfg.nz, cfg.dx)
    if geo is None:
        geo = L.Geometry(g, torch.from_numpy(cfg.soup()).cuda(), deadend_on=cfg.deadend_on)
    prec = cfg.precision if precision is None else precision
    solver = L.Solver(g, cfg.nu, cfg.dt, cfg.bc, cfg.u_in, precision=prec, solver=L.CG,
                      tol=cfg.tol if prec != L.FP64 else (cfg.tol if name == FP64_SMALL else 1e-10),
                      max_iter=2000, check_every=args.check_every, inner_tol=args.inner_tol,
                      csm_on=cfg.csm_on, forcing_on=cfg.forcing_on, geometry=geo,
                      precond=L.MULTIGRID if args.precond == "mg" else L.NO_PRECOND,
                      quick=quick, integrator=L.CRANK_NICOLSON if integ == 1 else L.ADAMS_BASHFORTH,
                      mg_sweeps=args.mg_sweeps, mg_omega=args.mg_omega)
    return cfg, g, geo, solver


def checked_step(L, solver, st, tol):
    s = solver.step(st)
    if s.status != 0 or not (s.relres <= tol):
        raise RuntimeError("step failed: status %d, relres %.3e" % (s.status, s.relres))
    return s


def timed_steps(L, torch, solver, st, steps, tol, stream, clocks=None):
    """K steps between CUDA events on the launching stream, inputs resident in HBM."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    stats = []
    n0 = solver.kernel_launches()
    e0.record(stream)
    for _ in range(steps):
        stats.append(checked_step(L, solver, st, tol).as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), stats, solver.kernel_launches() - n0


def solve_summary(stats):
    return {"inner_iters_per_step": float(np.mean([s["iters"] for s in stats])),
            "refinements_per_step": float(np.mean([s["outer"] for s in stats])),
            "momentum_bicgstab_iters_per_step": float(np.mean([s["mom_iters"] for s in stats])),
            "max_relres": float(max(s["relres"] for s in stats))}


def kernel_groups(solver, torch, st, steps, N, s_bytes, args, tol, peak):
    """The same number of steps again with per-kernel CUDA events recorded on the launching stream
    (graphs off while the profiler is on): per group achieved GB/s = algorithmic bytes per launch /
    mean launch time."""
    solver.profile(1)
    torch.cuda.synchronize()
    iters = 0
    for _ in range(steps):
        s = solver.step(st)
        if s.status != 0:
            raise RuntimeError("profiled step failed: status %d" % s.status)
        iters += s.iters
    torch.cuda.synchronize()
    prof = solver.profile_read()
    solver.profile(0)
    levels, fused, _ = solver.mg_info()
    bpc = bytes_per_cell(s_bytes, args.integrator, args.mg_sweeps, fused)
    # The Krylov kernels are launched check_every iterations at a time and return at once when the
    # solve has converged, so their launch counts include such empty launches: the per-iteration groups
    # are averaged over the iterations the solves actually ran (the empty launches' few microseconds
    # stay in the totals).
    per_iter = {"cg_dir_spmv": 1, "cg_update": 1}
    if levels > 0:
        per_iter["mg_fine"] = 2 if fused else 4 * args.mg_sweeps
        per_iter["mg_transfer"] = 1 if fused else 2
    groups = {}
    for k, (ms_k, n_k) in prof.items():
        if n_k <= 0 or k not in bpc:
            continue
        n_eff = min(n_k, per_iter[k] * iters) if k in per_iter and iters > 0 else n_k
        gbs = bpc[k] * N / (ms_k / n_eff * 1e-3) / 1e9
        groups[k] = {"launches": n_eff, "launches_incl_empty": n_k, "avg_launch_ms": ms_k / n_eff,
                     "bytes_per_launch": bpc[k] * N, "achieved_gbs": gbs, "frac": gbs / peak}
    return prof, groups


def measure(L, torch, name, args, world, stream, precision=None, steps=None, warmup=None, profile=True,
            e2e_steps=0, clocks=False, own_scheme=False):
    """Warm-up, then K timed steps; optionally the per-kernel profile pass and the end-to-end pass."""
    cfg, g, geo, solver = make_solver(L, torch, name, args, precision, own_scheme=own_scheme)
    tol = solver.params.tol
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    st = solver.fields(W.initial_fields(cfg))
    for _ in range(warmup):
        checked_step(L, solver, st, tol)
    torch.cuda.synchronize()
    barrier(world)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    gpu_id = "GPU-" + str(props.uuid) if getattr(props, "uuid", None) else str(torch.cuda.current_device())
    clk = None
    if clocks:
        with Clocks(gpu_id) as c:
            ms, stats, launches = timed_steps(L, torch, solver, st, steps, tol, stream)
        clk = c.summary()
    else:
        ms, stats, launches = timed_steps(L, torch, solver, st, steps, tol, stream)
    barrier(world)
    ms = max_over_ranks(ms, world)
    N = cfg.ncell
    out = {"workload": name, "cells": N, "value": N * steps * world / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
           "steps": steps, "warmup": warmup, "timed_steps": [warmup + 1, warmup + steps], "gpu_launches": launches,
           "solve": solve_summary(stats), "clocks": clk}
    s_bytes = 8 if solver.params.precision == L.FP64 else 4
    out["precision"] = "fp32" if s_bytes == 4 else "fp64"
    if profile:
        peak, peak_kind = read_peaks()
        prof, groups = kernel_groups(solver, torch, st, steps, N, s_bytes, args, tol, peak)
        everything = {k: v for k, v in prof.items() if v[1] > 0}
        tot = sum(x[0] for x in everything.values())
        out["shares"] = {k: round(v[0] / tot, 4) for k, v in everything.items()}
        out["groups"] = groups
        out["peak"] = (peak, peak_kind)
        out["mg"] = dict(zip(("levels", "fused_fine_passes", "unknowns"), solver.mg_info()))
        if args.integrator == "cn" and prof["momentum"][1] > 0:
            # momentum BiCGStab per step: M iterations of (68 s + 2) bytes per cell (p update, two operator
            # passes, s update, x/r update over the stacked 3N vector)
            M = out["solve"]["momentum_bicgstab_iters_per_step"]
            mb = M * (68 * s_bytes + 2) * N
            mms = prof["momentum"][0] / steps
            groups["momentum_per_step"] = {"launches": steps, "avg_launch_ms": mms, "bytes_per_launch": mb,
                                           "achieved_gbs": mb / (mms * 1e-3) / 1e9,
                                           "frac": mb / (mms * 1e-3) / 1e9 / peak}
    if e2e_steps:
        # end to end through the public entry point with host buffers: H2D of the step's state from
        # pinned memory, the step, D2H of its result, every step; each step's status is checked.  The
        # state is u, U and p (p^n is the pressure solve's initial guess); H = L(u^n) is an input only
        # of the Adams-Bashforth step (Crank-Nicolson recomputes it), so it travels only then.
        ke = min(steps, e2e_steps)
        keys = ("u", "U", "p", "H") if solver.params.integrator == L.ADAMS_BASHFORTH else ("u", "U", "p")
        host = {k: st[k].cpu().pin_memory() for k in keys}
        dev = {k: torch.empty_like(st[k]) for k in ("u", "U", "p", "H")}
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        stats = L.Stats()
        torch.cuda.synchronize()
        barrier(world)
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for q in range(ke):
            for k in host:
                dev[k].copy_(host[k], non_blocking=True)
            rc = solver.step_raw(dev["u"], dev["U"], dev["p"], dev["H"], False, stats=stats)
            if rc != 0 or not (stats.relres <= tol):
                raise RuntimeError("end-to-end step failed: rc %d, relres %.3e" % (rc, stats.relres))
            for k in host:
                host[k].copy_(dev[k], non_blocking=True)
        e3.record(stream)
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(e2.elapsed_time(e3), world)
        out["e2e"] = {"value": N * ke * world / (ms_e2e * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": h2d, "steps": ke}
        del host, dev
    out["_solver"], out["_state"], out["_geo"] = solver, st, geo
    return out


def release(m):
    for k in ("_solver", "_state", "_geo"):
        obj = m.pop(k, None)
        if k == "_solver" and obj is not None:
            obj.close()
        del obj


def train_guess(L, torch, args):
    """Snapshots (b, p^n, p^{n-1}, p^{n+1}) of the solver's own steps on the dirty sphere, then Adam
    steps on the GPU with the library's forward and backward kernels."""
    cfg, g, geo, solver = make_solver(L, torch, TRAIN_WORKLOAD, args)
    st = solver.fields(W.initial_fields(cfg))
    for _ in range(args.learn_spinup):
        checked_step(L, solver, st, cfg.tol)
    N = cfg.ncell
    snaps = []
    p_prev = st["p"].clone()
    t0 = time.time()
    for n in range(args.learn_snapshots + 1):
        p_n = st["p"].clone()
        checked_step(L, solver, st, cfg.tol)
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        solver.last_rhs(b)
        if n >= 1:
            snaps.append((b, p_n, p_prev, st["p"].clone()))
        p_prev = p_n
    torch.cuda.synchronize()
    t_collect = time.time() - t0
    net = L.Net(net_init())
    losses = []
    t0 = time.time()
    for epoch in range(args.learn_epochs):
        for (b, p_n, p_p, p_next) in snaps:
            _, sc = net.forward(g, b, p_n, p_p, geo.flags)
            target = net.target(g, p_next, p_n, p_p, sc)
            losses.append(net.train_step(g, b, p_n, p_p, target, args.learn_lr, geo.flags))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    solver.close()
    del snaps, st, geo
    torch.cuda.empty_cache()
    return net, {"workload": TRAIN_WORKLOAD, "snapshots": args.learn_snapshots, "epochs": args.learn_epochs,
                 "lr": args.learn_lr, "loss_first": losses[0], "loss_last": losses[-1],
                 "collect_s": t_collect, "train_s": t_train}


def learned_vs_plain(L, torch, m, net, train, args, world, stream):
    """K steps without a guess, K steps with the bare extrapolation 2 p^n - p^{n-1} (the guess of a
    network with zero parameters) and K steps with the trained guess: consecutive windows from the same
    solver state, so the gain of the network itself is the difference of the last two."""
    solver, st = m["_solver"], m["_state"]
    tol = solver.params.tol
    N = m["cells"]

    def window(guess):
        solver.attach_guess(guess)
        if guess is not None:
            checked_step(L, solver, st, tol)                 # the guess needs p^{n-1}
        ms, stats, _ = timed_steps(L, torch, solver, st, args.steps, tol, stream)
        solver.attach_guess(None)
        ms = max_over_ranks(ms, world)
        ratios = [s["relres_guess"] / s["relres0"] for s in stats if s["relres0"] > 0]
        out = {"value": N * args.steps * world / (ms * 1e-3) / 1e6, "ms_per_step": ms / args.steps,
               "solve": solve_summary(stats)}
        if guess is not None:
            out["guess_used_fraction"] = float(np.mean([s["guess_used"] for s in stats]))
            out["median_initial_residual_ratio"] = float(np.median(ratios)) if ratios else None
        return out

    plain = window(None)
    zero = L.Net(np.zeros(net.n_params, np.float32))
    extrap = window(zero)
    zero.close()
    learned = window(net)
    learned.update({"workload": m["workload"], "plain_same_window": plain, "extrapolation_same_window": extrap,
                    "speedup": plain["ms_per_step"] / learned["ms_per_step"],
                    "speedup_over_extrapolation": extrap["ms_per_step"] / learned["ms_per_step"], "train": train,
                    "note": "three consecutive windows from the same solver state: no guess, the bare extrapolation "
                            "2 p^n - p^{n-1} (a network with zero parameters), the trained guess; initial residual "
                            "ratios are the guess's over p^n's; the network is trained on snapshots of a different "
                            "workload (%s)" % TRAIN_WORKLOAD})
    return learned


def roofline_of(m, workload):
    """Roofline object of the dominant single-kernel group of a measured workload."""
    groups = {k: v for k, v in m["groups"].items() if k != "momentum_per_step"}
    dom = max(groups, key=lambda k: groups[k]["launches"] * groups[k]["avg_launch_ms"])
    g = groups[dom]
    peak, kind = m["peak"]
    names = dict(GROUP_KERNEL, **(GROUP_KERNEL_FUSED if m.get("mg", {}).get("fused_fine_passes") else {}))
    # the whole step against HBM: the groups' algorithmic bytes per step (the coarse multigrid levels and
    # the forcing have no byte model and are left out), and the plain-CG byte model of the method,
    # 119 + 41 I + 41 R bytes per cell in FP32 + refinement, 235 + 81 I in FP64 (I inner iterations,
    # R refinements per step)
    alg = sum(v["bytes_per_launch"] * v["launches"] for v in m["groups"].values()) / m["steps"]
    sv = m["solve"]
    fp32 = m.get("precision", "fp32") == "fp32"
    model = (119 + 41 * sv["inner_iters_per_step"] + 41 * sv["refinements_per_step"] if fp32
             else 235 + 81 * sv["inner_iters_per_step"]) * m["cells"]
    sec = m["ms_per_step"] * 1e-3
    step = {"algorithmic_bytes_per_step": alg, "achieved": alg / sec / 1e9, "frac": alg / sec / 1e9 / peak,
            "cg_model_bytes_per_step": model, "cg_model_frac": model / sec / 1e9 / peak,
            "note": "whole step: all groups' algorithmic bytes / the timed step; cg_model is the plain-CG "
                    "byte model (no preconditioner, explicit momentum) at the measured iteration counts"}
    return {"bound": "hbm", "kernel": dom, "kernel_name": names.get(dom, dom), "mg": m.get("mg"),
            "achieved": g["achieved_gbs"], "peak": peak, "unit": "GB/s", "frac": g["achieved_gbs"] / peak,
            "traffic": ncu_traffic(dom, workload), "algorithmic_bytes_per_launch": g["bytes_per_launch"],
            "avg_launch_ms": g["avg_launch_ms"], "peak_source": kind, "step": step, "shares": m["shares"],
            "groups": m["groups"],
            "note": "kernel times from a second pass of the same number of steps with per-kernel events on the "
                    "launching stream (graphs off); frac is of the measured copy peak"}


def cpu_baseline(args, iters, pool_result):
    """Oracle timings on the host cores: one thread and all cores on slab steps of the headline workload
    (each process its own slab), and the small workload run in full on one thread."""
    import multiprocessing as mp
    name = args.workload
    cfg = W.get_config(name)
    planes, rows = slab_shape(cfg)
    one = oracle_sample_step(name, iters, planes, integrator=args.integrator, quick=args.quick, rows=rows)
    ncores = os.cpu_count() or 1
    k0s = [int(v) for v in np.linspace(0, cfg.nz // 2 - planes, ncores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(ncores) as pool:
        t0 = time.perf_counter()
        res = pool.map(_sample_worker, [(name, iters, planes, k, args.integrator, args.quick, rows) for k in k0s])
        wall = time.perf_counter() - t0
    all_cells = sum(r["cells"] for r in res)
    # the slab-steps' own compute time (processes start and classify before they time)
    slowest = max(r["seconds"] for r in res)
    full = pool_result.get() if pool_result is not None else None
    out = {"value": one["cells"] / one["seconds"] / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": _sample_desc(name, planes, iters, args.integrator, rows),
           "host_cores": ncores,
           "all_cores": {"value": all_cells / slowest / 1e6, "cores": ncores, "wall_s_incl_setup": wall,
                         "note": "%d processes, each one slab step of the same workload at a different height, "
                                 "timed concurrently; value = total slab cells / slowest process's step time"
                                 % ncores}}
    if full is not None:
        cells, steps, secs = full
        out["full_run"] = {"workload": FP64_SMALL, "cells": cells, "steps": steps, "seconds": secs,
                           "value": cells * steps / secs / 1e6, "cores": 1,
                           "note": "the whole 50-step FP64 workload to 1e-10 (oracle BiCGStab), one thread"}
    return out


def run_ours(args):
    import multiprocessing as mp
    rank, world, local = dist_env()
    # the oracle's full run of the small workload goes in a spawned process started before any GPU call,
    # on one host core while the GPU is measured
    full_pool = None
    full_res = None
    if rank == 0 and not args.no_cpu_baseline:
        full_pool = mp.get_context("spawn").Pool(1)
        full_res = full_pool.apply_async(_full_run_worker, (FP64_SMALL,))
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    from paper_2002_06206_gb300 import build
    build.build()
    from paper_2002_06206_gb300 import ibmles as L
    stream = torch.cuda.current_stream()

    # ---- the learned initial guess, trained once on dirty-sphere snapshots (not timed)
    net, train = (None, None)
    if not args.no_learned:
        net, train = train_guess(L, torch, args)

    # ---- headline: the largest workload, FP32 + FP64 refinement; then, from the same state, the plain
    # step against the extrapolated and the learned starts
    head = measure(L, torch, args.workload, args, world, stream, profile=True, e2e_steps=args.e2e_steps, clocks=True)
    roof = roofline_of(head, args.workload)
    head_learned = learned_vs_plain(L, torch, head, net, train, args, world, stream) if net is not None else None
    release(head)
    torch.cuda.empty_cache()
    classify = None if args.no_classify else time_classify(L, torch, args.workload)

    # ---- the cube-and-plate workload: plain, then learned vs plain in the same window
    second = None
    if not args.no_secondary:
        sm = measure(L, torch, SECONDARY, args, world, stream, steps=args.steps, warmup=args.warmup, profile=True)
        second = {k: sm[k] for k in ("workload", "cells", "value", "ms_per_step", "steps", "timed_steps", "solve")}
        second["roofline"] = {k: v for k, v in roofline_of(sm, SECONDARY).items() if k not in ("shares",)}
        if net is not None:
            second["learned"] = learned_vs_plain(L, torch, sm, net, train, args, world, stream)
        release(sm)
        torch.cuda.empty_cache()
    if net is not None:
        net.close()

    # ---- the pure-FP64 path
    fp64 = None
    if not args.no_fp64:
        fp64 = {}
        small = W.get_config(FP64_SMALL)
        f1 = measure(L, torch, FP64_SMALL, args, world, stream, precision=L.FP64, steps=small.steps, warmup=0,
                     profile=False, own_scheme=True)
        fp64[FP64_SMALL] = {k: f1[k] for k in ("cells", "value", "ms_per_step", "steps", "solve")}
        fp64[FP64_SMALL]["note"] = ("the whole 50-step workload from its initial field with its own scheme (AB2, "
                                    "central advection), tol 1e-10; L2-resident, as the oracle's full run")
        release(f1)
        f3 = measure(L, torch, SECONDARY, args, world, stream, precision=L.FP64, steps=max(args.steps // 2, 5),
                     warmup=args.warmup, profile=True)
        fp64[SECONDARY] = {k: f3[k] for k in ("cells", "value", "ms_per_step", "steps", "solve")}
        fp64[SECONDARY]["roofline"] = {k: v for k, v in roofline_of(f3, SECONDARY).items() if k not in ("shares",)}
        release(f3)
        torch.cuda.empty_cache()
        # the arithmetic roofs beside the HBM roof: measured FMA rates (2 flops per FMA)
        fp64["fma_tflops"] = {"fp64": L.fma_rate(L.FP64, stream), "fp32": L.fma_rate(L.FP32_REFINE64, stream),
                              "note": "independent FMA chains on every SM, best of three launches"}

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(args, int(round(head["solve"]["inner_iters_per_step"])), full_res)
            full_pool.close()
            full_pool.join()
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args.workload, args), parallelism="replicas" if world > 1 else "single"),
            "solve": head["solve"], "timed_steps": head["timed_steps"],
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": head.get("e2e"),
            "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"],
            "classify": classify,
            "secondary": second,
            "learned": head_learned,
            "fp64": fp64,
        }
        print(json.dumps(line), flush=True)
    elif full_pool is not None:
        full_pool.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=30)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--check-every", type=int, default=8)
    ap.add_argument("--precond", default="mg", choices=["mg", "none"])
    ap.add_argument("--integrator", default="cn", choices=["cn", "ab2"],
                    help="Crank-Nicolson (the paper's production integrator) or Adams-Bashforth 2")
    ap.add_argument("--quick", type=float, default=0.1, help="QUICK fraction of the advected face value")
    ap.add_argument("--mg-sweeps", type=int, default=2, help="red-black sweeps before and after each coarse correction")
    ap.add_argument("--mg-omega", type=float, default=1.6, help="multigrid coarse-correction factor")
    ap.add_argument("--inner-tol", type=float, default=1e-5,
                    help="FP32 inner solve: residual reduction per FP64 refinement")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-classify", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the cube-and-plate line (and the learned guess)")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--learn-spinup", type=int, default=30)
    ap.add_argument("--learn-snapshots", type=int, default=24)
    ap.add_argument("--learn-epochs", type=int, default=8)
    ap.add_argument("--learn-lr", type=float, default=2e-3)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

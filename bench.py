"""Throughput of the immersed-boundary LES step on one GB300 (or N independent replicas).

A step is one fractional time step of the whole hot path (CSM eddy viscosity, Crank-Nicolson predictor
with 10 % QUICK and its momentum BiCGStab, IB forcing, face velocities, RHS, pressure solve to
||b - A p|| / ||b|| <= 1e-6, correction) on the dirty sphere workload: 256 x 128 x 128 cells (4.19 M),
a 40.6k-triangle dirty icosphere soup, FP32 stencils with FP64 iterative refinement of the pressure.
The default warm-up of 400 steps puts the timed window at steps 401-500 of the run.
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

WORKLOAD = "dirty_sphere_256x128x128"
METRIC = "Mcell-steps/s at Poisson rel. residual 1e-6, learned+mixed vs plain, %HBM roof"
UNIT = "Mcell-steps/s"
FALLBACK_HBM = 6800.0
# CG iterations per step the oracle is charged in its extrapolated step (about the GPU's measured
# mean of multigrid-preconditioned CG on this workload)
I_REF_DEFAULT = 20

# algorithmic bytes per cell of each timed kernel group (s = bytes of a working-precision value)
def bytes_per_cell(s, integrator="cn"):
    return {
        "csm": 4 * s + 1,                 # u (3) + flags -> nu_t
        # AB2: u, U, nu_t, Hprev, flags -> H, u*;  CN: u, U, nu_t, flags -> H, r, r_hat, delta
        "predict": (16 * s + 1) if integrator == "ab2" else (19 * s + 1),
        "faces": 6 * s + 1,               # u*, flags -> U*
        "rhs": 3 * s + 8,                 # U* -> b (fp64)
        "residual": 8 + 8 + 1 + s,        # b, x (fp64), flags -> r
        "cg_dir_spmv": 4 * s + 1,         # r, p_old, flags -> p, q
        "cg_update": 6 * s,               # x, p, r, q -> x, r
        "correct": 12 * s + 9,            # u*, U*, p (fp64), flags -> u, U
        "mg_fine": 2 * s + 1,             # one red-black colour pass: z (all), r and z (one colour), flags
    }


# the kernel behind each single-kernel group (FP32 path with nx a multiple of 4)
GROUP_KERNEL = {"csm": "k_csm", "predict": "k_cn_begin (tiled + general)", "faces": "k_faces",
                "rhs": "k_rhs", "residual": "k_residual", "cg_dir_spmv": "k_cg_dir_spmv_x4",
                "cg_update": "k_cg_update", "correct": "k_correct_cells + k_correct_faces",
                "mg_fine": "k_mg_smooth0_x4"}


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


def ncu_traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if the sources that define that kernel
    (the files listed with it) are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        with open(path) as f:
            d = json.load(f)
        k = d["kernels"].get(kernel_key)
        if not k or k.get("source_hash") != src_hash(k["files"]):
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
        self.path = os.path.join("/tmp", "bench_clocks_%d_%d.csv" % (os.getpid(), int(time.time())))

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


# ------------------------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample of the same workload

def oracle_sample(cfg, iters_per_step, n_iter_sample=5, planes=8, integrator="cn", quick=0.1, mom_tol=1e-6):
    """Time the FP64 oracle on a z-slab of the workload (the `planes` planes through the body's centre,
    same soup, same per-cell work) -- one pass of every non-Poisson operator (the Crank-Nicolson
    predictor with its momentum BiCGStab, or the AB2 predictor) plus n_iter_sample CG iterations -- and
    scale to one full-size step: t = (N / N_slab) * (t_ops + I * t_iter)."""
    import oracle
    k0 = cfg.nz // 2 - planes // 2
    tri = cfg.soup().copy()
    tri[..., 2] -= k0
    case = oracle.Case(cfg.nx, cfg.ny, planes, cfg.dx, cfg.nu, cfg.dt, cfg.bc, cfg.u_in, cfg.csm_on,
                       cfg.forcing_on, cfg.deadend_on, quick)
    case.set_geometry(tri)
    u = W.initial_fields(W.Config("slab", cfg.nx, cfg.ny, planes, 0, 0, 0, 0, 0, cfg.bc, seed=cfg.seed)).reshape(-1)
    U = case.faces(u)
    t0 = time.perf_counter()
    nut = case.csm(u)
    if integrator == "cn":
        H, us, mom_it = case.predict_cn(u, U, nut, tol=mom_tol)
    else:
        H, us = case.predict(u, U, nut, np.zeros_like(u), True)
    us2, _ = case.forcing(us)
    Us = case.faces(us2)
    b = case.rhs(Us)
    t1 = time.perf_counter()
    p, st = case.solve(b, None, tol=1e-30, maxit=n_iter_sample, solver=oracle.CG)
    t2 = time.perf_counter()
    case.correct(us2, Us, p)
    t3 = time.perf_counter()
    t_ops = (t1 - t0) + (t3 - t2)
    t_iter = (t2 - t1) / max(st.iters, 1)
    scale = cfg.ncell / case.N
    t_step = scale * (t_ops + iters_per_step * t_iter)
    sample = ("oracle (FP64, 1 thread) on the %dx%dx%d slab through the body centre: one pass of csm, %s "
              "predictor, forcing, faces, rhs, correct plus %d CG iterations; full step = (N/N_slab) * "
              "(t_ops + I * t_iter) with I = %.1f CG iterations per step"
              % (cfg.nx, cfg.ny, planes, "Crank-Nicolson (momentum BiCGStab to %g)" % mom_tol if integrator == "cn"
                 else "AB2", st.iters, iters_per_step))
    return {"t_step_s": t_step, "t_ops_s": t_ops * scale, "t_iter_s": t_iter * scale, "sample": sample,
            "wall_s": t3 - t0}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg = W.get_config(args.workload)
    I = float(os.environ.get("IBM_REF_ITERS", I_REF_DEFAULT))
    kw = dict(integrator=args.integrator, quick=args.quick)
    # The oracle has nothing to warm up; one sample on an 8-plane slab stands for the W warm-up steps
    # and sizes the K timed samples so that the whole run stays within about two minutes.
    first = oracle_sample(cfg, I, planes=8, **kw)
    budget_s = 120.0
    planes = int(max(2, min(8, 8 * (budget_s / max(args.steps, 1)) / max(first["wall_s"], 1e-3))))
    times = []
    for _ in range(args.steps):
        times.append(oracle_sample(cfg, I, planes=planes, **kw))
    t_step = float(np.mean([t["t_step_s"] for t in times]))
    value = cfg.ncell / t_step / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "cells": cfg.ncell,
                       "integrator": "crank-nicolson" if args.integrator == "cn" else "adams-bashforth-2",
                       "quick": args.quick, "slab_planes": planes},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": times[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------

def time_classify(L, torch, name="vehicle_1024x512x384", repeats=5):
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


def timed_steps(torch, solver, st, steps, stream):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    stats = []
    e0.record(stream)
    for _ in range(steps):
        stats.append(solver.step(st).as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), stats


def run_learned(args, L, torch, solver, st, geo, cfg, world):
    """Learned initial guess: snapshots (b, p^n, p^{n-1}, p^{n+1}) from the solver's own steps, Adam
    training on the GPU with the library's kernels, then K steps without and K steps with the guess
    from the same point of the run."""
    N = cfg.ncell
    g = L.make_grid(cfg.nx, cfg.ny, cfg.nz, cfg.dx)
    stream = torch.cuda.current_stream()
    snaps = []
    p_prev = st["p"].clone()
    t0 = time.time()
    for n in range(args.learn_snapshots + 2):
        p_n = st["p"].clone()
        solver.step(st)
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        solver.last_rhs(b)
        if n >= 2:
            snaps.append((b, p_n, p_prev, st["p"].clone()))
        p_prev = p_n
    torch.cuda.synchronize()
    t_collect = time.time() - t0
    net = L.Net(net_init())
    t0 = time.time()
    losses = []
    for epoch in range(args.learn_epochs):
        for (b, p_n, p_p, p_next) in snaps:
            _, sc = net.forward(g, b, p_n, p_p, geo.flags)
            target = ((p_next - 2.0 * p_n + p_p) / sc).to(torch.float32)
            losses.append(net.train_step(g, b, p_n, p_p, target, args.learn_lr, geo.flags))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del snaps
    torch.cuda.empty_cache()
    ms_plain, st_plain = timed_steps(torch, solver, st, args.steps, stream)
    solver.attach_guess(net)
    solver.step(st)                       # the guess needs p^{n-1}
    ms_learn, st_learn = timed_steps(torch, solver, st, args.steps, stream)
    solver.attach_guess(None)
    ms_plain = max_over_ranks(ms_plain, world)
    ms_learn = max_over_ranks(ms_learn, world)
    ratios = [s["relres_guess"] / s["relres0"] for s in st_learn if s["relres0"] > 0]
    net.close()
    return {
        "value": N * args.steps * world / (ms_learn * 1e-3) / 1e6,
        "ms_per_step": ms_learn / args.steps,
        "plain_same_window": {"value": N * args.steps * world / (ms_plain * 1e-3) / 1e6,
                              "ms_per_step": ms_plain / args.steps,
                              "inner_iters_per_step": float(np.mean([s["iters"] for s in st_plain])),
                              "refinements_per_step": float(np.mean([s["outer"] for s in st_plain]))},
        "inner_iters_per_step": float(np.mean([s["iters"] for s in st_learn])),
        "refinements_per_step": float(np.mean([s["outer"] for s in st_learn])),
        "guess_used_fraction": float(np.mean([s["guess_used"] for s in st_learn])),
        "median_initial_residual_ratio": float(np.median(ratios)) if ratios else None,
        "max_relres": float(max(s["relres"] for s in st_learn)),
        "train": {"snapshots": args.learn_snapshots, "epochs": args.learn_epochs, "lr": args.learn_lr,
                  "loss_first": losses[0], "loss_last": losses[-1], "collect_s": t_collect, "train_s": t_train},
        "note": "plain and learned windows are consecutive, after the training snapshots; same solver state",
    }


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    from paper_2002_06206_gb300 import build
    build.build()
    from paper_2002_06206_gb300 import ibmles as L

    cfg = W.get_config(args.workload)
    tri = cfg.soup()
    g = L.make_grid(cfg.nx, cfg.ny, cfg.nz, cfg.dx)
    geo = L.Geometry(g, torch.from_numpy(tri).cuda(), deadend_on=cfg.deadend_on)
    precond = L.MULTIGRID if args.precond == "mg" else L.NO_PRECOND
    integ = L.CRANK_NICOLSON if args.integrator == "cn" else L.ADAMS_BASHFORTH
    solver = L.Solver(g, cfg.nu, cfg.dt, cfg.bc, cfg.u_in, precision=cfg.precision, solver=L.CG, tol=cfg.tol,
                      max_iter=100000, check_every=args.check_every, inner_tol=args.inner_tol,
                      csm_on=cfg.csm_on, forcing_on=cfg.forcing_on, geometry=geo, precond=precond,
                      quick=args.quick, integrator=integ, mg_sweeps=args.mg_sweeps,
                      mg_omega=args.mg_omega)
    st = solver.fields(W.initial_fields(cfg))
    for _ in range(args.warmup):
        solver.step(st)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    props = torch.cuda.get_device_properties(local)
    gpu_id = "GPU-" + str(props.uuid) if getattr(props, "uuid", None) else str(local)

    # ---- timed region: K steps, inputs resident in HBM, the library's fast path (CUDA graphs on)
    iters, outers, relres, moms = [], [], [], []
    solver.profile(0)
    n_launch0 = solver.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(gpu_id) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            s = solver.step(st)
            iters.append(s.iters)
            outers.append(s.outer)
            relres.append(s.relres)
            moms.append(s.mom_iters)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = solver.kernel_launches() - n_launch0
    barrier(world)
    ms_max = max_over_ranks(ms, world)
    clocks = clk.summary()

    # ---- the same number of steps again with per-kernel CUDA events on the launching stream (the
    # profiler records around every kernel group, so graphs are not used here): kernel durations
    solver.profile(1)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        solver.step(st)
    torch.cuda.synchronize()
    prof = solver.profile_read()
    solver.profile(0)

    # ---- end to end through the public API with host buffers: H2D of the step's inputs from pinned
    # memory, the step, D2H of its result, every step
    ke = min(args.steps, args.e2e_steps)
    host = {k: st[k].cpu().pin_memory() for k in ("u", "U", "p", "H")}
    dev = {k: torch.empty_like(st[k]) for k in host}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = h2d
    torch.cuda.synchronize()
    barrier(world)
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    n0 = st["n"]
    for q in range(ke):
        for k in host:
            dev[k].copy_(host[k], non_blocking=True)
        solver.step_raw(dev["u"], dev["U"], dev["p"], dev["H"], False)
        for k in host:
            host[k].copy_(dev[k], non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3), world)
    del n0

    N = cfg.ncell
    value = N * args.steps * world / (ms_max * 1e-3) / 1e6
    e2e_value = N * ke * world / (ms_e2e * 1e-3) / 1e6

    # ---- roofline of the dominant kernel group
    s_bytes = 8 if cfg.precision == L.FP64 else 4
    bpc = bytes_per_cell(s_bytes, args.integrator)
    timed = {k: v for k, v in prof.items() if v[1] > 0 and k in bpc}
    everything = {k: v for k, v in prof.items() if v[1] > 0}
    M = float(np.mean(moms))
    peak, peak_kind = read_peaks()
    # every group with a byte model: achieved = algorithmic bytes per launch / mean launch time
    groups = {}
    for k, (ms_k, n_k) in timed.items():
        gbs = bpc[k] * N / (ms_k / n_k * 1e-3) / 1e9
        groups[k] = {"launches": n_k, "avg_launch_ms": ms_k / n_k, "bytes_per_launch": bpc[k] * N,
                     "achieved_gbs": gbs, "frac": gbs / peak}
    if args.integrator == "cn" and prof["momentum"][1] > 0:
        # the momentum BiCGStab per step (several kernel kinds): M iterations of p update (r, p, v ->
        # p), two operator passes (input, U, nu_t, flags -> output, one dot operand), s update
        # (r, v -> s), x/r update (x, p, s, t, r_hat -> x, r): (68 s + 2) bytes per cell per iteration
        mb = M * (68 * s_bytes + 2) * N
        mms = prof["momentum"][0] / args.steps
        groups["momentum_per_step"] = {"launches": args.steps, "avg_launch_ms": mms, "bytes_per_launch": mb,
                                       "achieved_gbs": mb / (mms * 1e-3) / 1e9,
                                       "frac": mb / (mms * 1e-3) / 1e9 / peak}
    # the dominant single kernel (one kernel kind per launch of the group)
    dom = max(timed, key=lambda k: timed[k][0])
    avg_ms = timed[dom][0] / timed[dom][1]
    algo_bytes = bpc[dom] * N
    achieved = algo_bytes / (avg_ms * 1e-3) / 1e9
    shares = {k: round(v[0] / sum(x[0] for x in everything.values()), 4) for k, v in everything.items()}

    learned = run_learned(args, L, torch, solver, st, geo, cfg, world) if args.learned else None
    classify = None if args.no_classify else time_classify(L, torch)

    line = None
    if rank == 0:
        I = float(np.mean(iters))
        cpu = oracle_sample(cfg, I, integrator=args.integrator, quick=args.quick) if not args.no_cpu_baseline else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "cells": N, "grid": [cfg.nx, cfg.ny, cfg.nz],
                       "triangles": int(len(tri)), "precision": "fp32 stencils and cg, fp64 residual refinement",
                       "solver": "cg + multigrid V-cycle" if precond else "cg", "tol": cfg.tol,
                       "integrator": "crank-nicolson" if args.integrator == "cn" else "adams-bashforth-2",
                       "quick": args.quick, "mg_sweeps": args.mg_sweeps if precond else None,
                       "mg_omega": args.mg_omega if precond else None,
                       "momentum_bicgstab_iters_per_step": M,
                       "timed_steps": [args.warmup + 1, args.warmup + args.steps],
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (~0.4 GB of state per step vs 126 MB L2)",
                       "inner_iters_per_step": I, "refinements_per_step": float(np.mean(outers)),
                       "max_relres": float(np.max(relres))},
            "roofline": {"bound": "hbm", "kernel": dom, "kernel_name": GROUP_KERNEL.get(dom, dom),
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": ncu_traffic(dom),
                         "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_ms": avg_ms,
                         "peak_source": peak_kind, "shares": shares, "groups": groups,
                         "note": "kernel times from a second pass of the same number of steps with per-kernel "
                                 "events (graphs off); shares are of event-timed kernel time"},
            "cpu_baseline": None if cpu is None else {
                "value": N / cpu["t_step_s"] / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": cpu["sample"]},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": ke},
            "gpu_launches": launches,
            "clocks": clocks,
            "classify": classify,
            "learned": learned,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=400)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--check-every", type=int, default=8)
    ap.add_argument("--precond", default="mg", choices=["mg", "none"])
    ap.add_argument("--integrator", default="cn", choices=["cn", "ab2"],
                    help="Crank-Nicolson (the paper's production integrator) or Adams-Bashforth 2")
    ap.add_argument("--quick", type=float, default=0.1, help="QUICK fraction of the advected face value")
    ap.add_argument("--mg-sweeps", type=int, default=2, help="red-black sweeps before and after each coarse correction")
    ap.add_argument("--mg-omega", type=float, default=1.8, help="multigrid coarse-correction factor")
    ap.add_argument("--inner-tol", type=float, default=1e-4)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-classify", action="store_true")
    ap.add_argument("--learned", action="store_true", help="also time the learned initial guess")
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

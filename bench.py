"""Benchmark of the connectivity-aware multigrid solver on GB300.

One step = the whole hot path for one synthetic mesh: assemble M and L of every
level (A = M + t L), project the right-hand sides (vertex x, y, z), solve
(M + t L) x = rhs with mixed-precision V-cycles to relative residual 1e-6 for
all three right-hand sides, and evaluate the solution at the mesh vertices
(one implicit mean-curvature-flow update, Section 5.3).  The hierarchy is built
once before timing.  Default workload: (3,5) torus-knot tube of radius 0.02,
4M triangles, depth 10, t = 1e-4.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead, on a
bounded stretch of the same mesh placed on the same grid.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

import meshgen   # seeded synthetic inputs (no method arithmetic)

METRIC = "unknowns×V-cycles/s; ms to 1e-6 rel. residual, mixed/learned vs plain FP64"
UNIT = "unknowns*V-cycles/s"
WORKLOAD = "knot35_4m_d10"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_over_ranks(ms, units, ws, device):
    """Replicas on ws ranks: every rank times its own copy of the workload, so the job's time
    is the slowest rank's and its units are the sum over ranks (weak scaling).  With one rank
    its own numbers are returned; otherwise a process group must be initialised."""
    if ws == 1:
        return float(ms), float(units)
    import torch
    import torch.distributed as dist
    mx = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    sm = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.item(), sm.item()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- the FP64 CPU oracle on a bounded sample of the workload ----
# The oracle (plain C, one thread) would take hours to build the hierarchy of the whole
# 4M-triangle mesh, so it runs on stretches of the same mesh: the first (or the i-th)
# `ntri` triangles, a contiguous piece of the tube, embedded in the whole mesh's grid cube
# so that its functions, stencils and levels are those of the workload.  The metric is
# unknowns x V-cycles / s, which a stretch measures like the whole.
SAMPLE_TRIS = 80_000
SAMPLE_CYCLES = 400


def oracle_stretch(V, F, ntri, index=0):
    """Triangles [index * ntri, (index + 1) * ntri) of F with their vertices, renumbered."""
    Fp = F[index * ntri:(index + 1) * ntri]
    used = np.unique(Fp)
    remap = np.full(V.shape[0], -1, dtype=np.int64)
    remap[used] = np.arange(used.size)
    return np.ascontiguousarray(V[used]), np.ascontiguousarray(remap[Fp], dtype=np.int32)


def _oracle_cycles(job):
    """One oracle sample: build the stretch's hierarchy, then time `cycles` FP64 V-cycles on
    the x/y/z right-hand sides.  Runs in this process or in a spawned worker (no CUDA)."""
    Vp, Fp, depth, min_depth, emb, t, cycles, barrier = job
    import oracle
    h = oracle.Hierarchy(Vp, Fp, depth, min_depth=min_depth, embedding=emb)
    rhs = h.project_rhs(Vp)
    h.vcycles(t, rhs, cycles=1)
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    h.vcycles(t, rhs, cycles=cycles)
    dt = time.perf_counter() - t0
    return h.ndof(depth), dt


_POOL_BARRIER = None


def _pool_init(barrier):
    global _POOL_BARRIER
    _POOL_BARRIER = barrier


def _pool_job(job):
    return _oracle_cycles(job[:-1] + (_POOL_BARRIER,))


def oracle_baseline(V, F, depth, min_depth, t, cores, ntri=SAMPLE_TRIS, cycles=SAMPLE_CYCLES):
    """Oracle throughput in unknowns x V-cycles / s on `cores` host cores: one stretch per core,
    each in its own spawned process (the oracle is single-threaded); the cycles of all of them
    start together behind a barrier, and the job's time is the slowest one's."""
    import multiprocessing as mp
    import oracle
    emb = oracle.embedding_of(V)
    nstretch = max(1, F.shape[0] // ntri)
    jobs = [oracle_stretch(V, F, ntri, i % nstretch) + (depth, min_depth, emb, t, cycles, None) for i in range(cores)]
    if cores == 1:
        n, dt = _oracle_cycles(jobs[0])
        return n * 3 * cycles / dt, dt, [n]
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    with ctx.Pool(cores, initializer=_pool_init, initargs=(barrier,)) as pool:
        res = pool.map(_pool_job, jobs)
    units = sum(n * 3 * cycles for n, _ in res)
    wall = max(dt for _, dt in res)
    return units / wall, wall, [n for n, _ in res]


def solve_bytes(h, sweeps, nrhs):
    """Algorithmic bytes of one mixed V-cycle step and of the fixed part of a solve.

    Per level d above the coarsest (FP32 values, R = 4 lanes of 4 bytes per row):
      smoothing sweep or residual: nnz*(4 value + 4 column) + n*(4 row pointer + 4 diagonal
        + 3*R*4 right-hand side / x read / x or r written);
      restriction into d-1: children entries*4 + n*R*4 read + n_{d-1}*(4 + 2*R*4);
      prolongation: n*(1 + parents*4 + parents*R*4 + 2*R*4), about 3.4 parents per row.
    Coarsest: the dense inverse (n0^2*4) and 2*n0*R*4.
    Finest FP64 outer step: conversion n*R*(8+4+4), update n*R*(8+4+8), FP64 residual
      nnz*(8+4) + n*(4 + 3*R*8), norms n*R*8.
    """
    import paper_1505_03615_gb300 as L
    R = 4 if nrhs > 2 else nrhs
    d0, D = L.lbmg_levels(h)
    cyc = 0.0
    for d in range(d0 + 1, D + 1):
        n, nnz, _ = L.lbmg_level_info(h, d)
        nc = L.lbmg_level_info(h, d - 1)[0]
        sweep = nnz * 8 + n * (8 + 3 * R * 4)
        cyc += (sweeps + 1) * sweep
        cyc += 3.4 * n * 4 + n * R * 4 + nc * (4 + 2 * R * 4)
        cyc += n * (1 + 3.4 * 4 + 3.4 * R * 4 + 2 * R * 4)
    n0 = L.lbmg_level_info(h, d0)[0]
    cyc += n0 * n0 * 4 + 2 * n0 * R * 4
    n, nnz, _ = L.lbmg_level_info(h, D)
    outer = n * R * 16 + n * R * 20 + nnz * 12 + n * (4 + 3 * R * 8) + n * R * 8
    return cyc + outer, nnz * 12 + n * (4 + 3 * R * 8) + 2 * n * R * 8


def reference_main(args):
    """Reference arm: the FP64 CPU oracle as it stands (one core), on a stretch of the same
    mesh on the same grid; each step is SAMPLE_CYCLES / 4 V-cycles on the x/y/z right-hand sides."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import meshgen
    import oracle
    V, F, depth, t, f, tol, _ = meshgen.config_mesh(args.workload)
    Vp, Fp = oracle_stretch(V, F, SAMPLE_TRIS)
    h = oracle.Hierarchy(Vp, Fp, depth, min_depth=args.oracle_min_depth, embedding=oracle.embedding_of(V))
    rhs = h.project_rhs(Vp)
    n = h.ndof(depth)
    cyc = SAMPLE_CYCLES // 4
    for _ in range(args.warmup):
        h.vcycles(t, rhs, cycles=1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        h.vcycles(t, rhs, cycles=cyc)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n * rhs.shape[1] * cyc * args.steps / total
    sample = (f"{cyc} FP64 lexicographic-GS V-cycles x 3 right-hand sides per step on the first {Fp.shape[0]} "
              f"triangles of the {args.workload} mesh, on its grid (depth {depth}, n={n}), one host core")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "triangles": int(Fp.shape[0]), "depth": depth, "t": t,
                   "sample_of": int(F.shape[0])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# training meshes of the learned correction: small stand-ins shaped like the plain-method
# sphere (depth 5), the (2,3) torus-knot tube (depth 7) and the two nearly touching sheets
# (depth 7); the residual histories of plain V-cycles on them are the training data
LEARNED_TRAIN = [
    ("icosphere(3), depth 5, t=1e-3", lambda: meshgen.icosphere(3, 1.0, 1e-3, 1), 5, 1e-3),
    ("(2,3) knot tube r=0.04 400x40, depth 7, t=1e-4", lambda: meshgen.torus_knot_tube(2, 3, 1.0, 0.04, 400, 40, 1e-6, 2),
     7, 1e-4),
    ("double sheet 60, depth 7, t=1e-3", lambda: meshgen.double_sheet(60, 0.05, 6, 0.5, 1e-6, 4), 7, 1e-3),
]
LEARNED_HISTORY = (0, 1, 2, 4, 8, 14, 22, 29)


def learned_train(L, dev, steps, lr, batch=4, block=5, seed=0):
    """The learned correction's network, trained on the GPU (setup, untimed).  Data: residual
    histories of plain FP64 V-cycles from zero on two right-hand sides per training mesh (the
    projected vertex coordinates and a random vertex function; 30 cycles kept).  Adam steps on
    the mean gradient of `batch` samples, drawn from the cycles in LEARNED_HISTORY of one mesh,
    `block` steps per visit of a random mesh (the optimiser state travels between the meshes'
    handles); the learning rate drops to lr/3 after half the steps and to lr/10 after three
    quarters.  Returns (parameters, loss history, seconds)."""
    import torch
    rng = np.random.default_rng(seed + 100)
    handles = []
    t0 = time.perf_counter()
    try:
        data = np.random.default_rng(seed)
        for _, make, depth, t in LEARNED_TRAIN:
            V, F = make()
            h = L.lbmg_build_hierarchy(V, F, depth)
            handles.append(h)
            L.lbmg_assemble(h, t)
            n = L.lbmg_level_info(h, depth)[0]
            for f in (V, data.uniform(-1, 1, size=V.shape)):
                rhs = torch.zeros((n, 3), dtype=torch.float64, device=dev)
                L.lbmg_project_rhs(h, torch.tensor(np.ascontiguousarray(f), device=dev), rhs)
                L.lbmg_learned_collect(h, rhs, 0, 30)
        P = L.lbmg_learned_nparams()
        init = np.random.default_rng(seed)
        W1 = np.zeros((32, 64))
        W1[:30] = init.normal(0, 0.05, size=(30, 64))
        p = np.concatenate([W1.ravel(), np.zeros(64), init.normal(0, 0.05, size=64), np.zeros(1)])
        state = np.concatenate([p, np.zeros(2 * P + 1)])
        hist = []
        done = 0
        while done < steps:
            frac = done / steps
            lr_now = lr if frac < 0.5 else (lr / 3 if frac < 0.75 else lr / 10)
            k = rng.integers(len(handles))
            L.lbmg_learned_state(handles[k], state)
            picks = (rng.choice(LEARNED_HISTORY, size=(block, batch)) +
                     30 * rng.integers(0, 2, size=(block, batch)))
            hist += list(L.lbmg_learned_train(handles[k], picks, lr_now))
            state = L.lbmg_learned_state(handles[k])
            done += block
        return state[:P], np.array(hist), time.perf_counter() - t0
    finally:
        for h in handles:
            L.lbmg_destroy(h)


def learned_compare(L, h, step, nsteps, params, hist, train_s, args):
    """The workload's own step with the learned correction in front of every cycle (trained
    params), and with the untrained one (zero network: the plain Jacobi start), nsteps each."""
    import torch
    out = {"trained_on": [m[0] for m in LEARNED_TRAIN], "train_steps": int(len(hist)), "batch": 4,
           "lr": args.learned_lr,
           "train_s": train_s, "loss_first50": float(np.mean(hist[:50])), "loss_last50": float(np.mean(hist[-50:])),
           "loss": "mean log(||r after||^2 / ||r before||^2) of one learned iteration",
           "solve": "mixed V(2,2) defect correction, one graph launch per solve"}
    try:
        for name, prm, k in (("learned", params, nsteps), ("jacobi_start", np.zeros_like(params), max(1, min(3, nsteps)))):
            L.lbmg_learned_params(h, prm)
            L.lbmg_learned_enable(h, True)
            step()
            torch.cuda.synchronize()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record()
            cyc, fb = 0, 0
            for _ in range(k):
                st = step()
                cyc += st.cycles
                fb = max(fb, st.learned_fallback)
            g1.record()
            torch.cuda.synchronize()
            out[name] = {"ms_to_tol": g0.elapsed_time(g1) / k, "cycles_per_step": cyc / k, "fallback": fb, "steps": k}
    finally:
        L.lbmg_learned_enable(h, False)
    return out


BATCH = "batch64"
CUBES = "cube_mindepth"


def _dof_perm(c, mt, oc, om, nt):
    """oracle index of every library function: both identify a function by its grid corner and
    the smallest triangle of its component"""
    def keys(cc, mm):
        cc = cc.astype(np.int64)
        return ((cc[:, 0] * 8192 + cc[:, 1]) * 8192 + cc[:, 2]) * (nt + 1) + mm.astype(np.int64)
    kl, ko = keys(c, mt), keys(oc, om)
    order = np.argsort(ko)
    perm = order[np.minimum(np.searchsorted(ko[order], kl), len(ko) - 1)]
    if not np.array_equal(ko[perm], kl):
        raise RuntimeError("library and oracle functions differ")
    return perm


def cube_main(args):
    """The minimum-depth experiment of Section 5.2 on the 6x6x6 grid of unit cubes one unit apart
    (depth 5, screening weight alpha = 0.01, i.e. A = M + L / alpha): one W-cycle with ten
    Gauss-Seidel sweeps per level from a U[0, 1] start, right-hand side 0, the coarsest level
    relaxed, for every minimum depth 0..5 in the split and the unsplit space.  Prints the
    residual alpha ||A x_1|| / ||x_0|| of the GPU and of the oracle (the same coloured cycle) and
    the GPU time of the cycle."""
    import torch

    import meshgen
    import oracle
    import paper_1505_03615_gb300 as L
    dev = torch.device("cuda", 0)
    alpha = 0.01
    t = 1.0 / alpha
    V, F = meshgen.cube_grid(6, 1.0, 1.0, 2)
    rows = []
    for split in (True, False):
        for m in range(6):
            h = L.lbmg_build_hierarchy(V, F, 5, min_depth=m, split=int(split), cycle=1, coarse_smooth=1, nu1=10,
                                       nu2=10)
            try:
                L.lbmg_assemble(h, t)
                n = L.lbmg_level_info(h, 5)[0]
                x0 = meshgen.random_start(n, 1)
                zero = torch.zeros((n, 1), dtype=torch.float64, device=dev)
                x = torch.tensor(x0, device=dev)
                L.lbmg_vcycles(h, zero, x, 1, L.LBMG_FP64)   # warm-up (graph capture)
                x = torch.tensor(x0, device=dev)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                L.lbmg_vcycles(h, zero, x, 1, L.LBMG_FP64)
                e1.record()
                torch.cuda.synchronize()
                r = torch.zeros_like(x)
                L.lbmg_residual(h, 5, zero, x, r)
                gpu = alpha * float(torch.linalg.norm(r)) / float(np.linalg.norm(x0))
                o = oracle.Hierarchy(V, F, 5, min_depth=m, split=split)
                c, mt = L.lbmg_get_dofs(h, 5)
                oc, om = o.dofs(5)
                perm = _dof_perm(c, mt, oc, om, F.shape[0])
                xo0 = np.zeros_like(x0)
                xo0[perm] = x0
                Mo, Lo = o.matrices(5)
                xo = o.cycles(t, np.zeros_like(x0), xo0, cycles=1, nu1=10, nu2=10, gamma=2, coloured=True,
                              coarse_smooth=True)
                orc = alpha * float(np.linalg.norm((Mo + t * Lo) @ xo)) / float(np.linalg.norm(x0))
                rows.append({"split": split, "min_depth": m, "residual_gpu": gpu, "residual_oracle": orc,
                             "functions_per_level": [L.lbmg_level_info(h, d)[0] for d in range(m, 6)],
                             "w_cycle_ms": e0.elapsed_time(e1)})
            finally:
                L.lbmg_destroy(h)
    print(json.dumps({"workload": CUBES, "triangles": int(F.shape[0]), "depth": 5, "alpha": alpha,
                      "cycle": "one W(10,10), coarsest level relaxed, right-hand side 0, start U[0,1]",
                      "residual": "alpha ||A x1|| / ||x0||", "rows": rows}), flush=True)



def batch_main(args):
    """64 seeded meshes of uneven size (10k-300k triangles; tori, ellipsoids, torus knots;
    depth 7-9) in one hierarchy, x/y/z right-hand sides, t = 1e-4, mixed precision to 1e-6
    per mesh in one persistent launch per solve.  A step is assemble + project + solve +
    vertex evaluation of the whole batch; the value counts every mesh's unknowns."""
    import torch

    import meshgen
    import paper_1505_03615_gb300 as L

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    meshes = meshgen.batch_mix(64)
    t, tol, nrhs = 1e-4, 1e-6, 3
    t_build = time.perf_counter()
    hb = L.lbmg_build_batch(meshes)
    t_build = time.perf_counter() - t_build
    ninst = L.lbmg_instances(hb)
    nu = sum(L.lbmg_instance_info(hb, i)[2] for i in range(ninst))
    f = np.concatenate([V for V, _, _ in meshes], axis=0)
    nv = f.shape[0]
    f_dev = torch.tensor(f, dtype=torch.float64, device=dev)
    rhs = torch.zeros((nu, nrhs), dtype=torch.float64, device=dev)
    x = torch.zeros_like(rhs)
    u = torch.zeros((nv, nrhs), dtype=torch.float64, device=dev)

    def step(precision=L.LBMG_MIXED, f_in=f_dev, u_out=u):
        L.lbmg_assemble(hb, t)
        L.lbmg_project_rhs(hb, f_in, rhs)
        x.zero_()
        solve = L.lbmg_solve_pcg if args.solver == "pcg" else L.lbmg_solve
        code, st = solve(hb, rhs, x, tol, args.max_cycles, precision)
        if code not in (L.LBMG_OK, L.LBMG_NOT_CONVERGED):
            raise RuntimeError(f"batch solve failed with status {code}")
        L.lbmg_eval_vertices(hb, x, u_out)
        return st

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.25)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    cycles, rel, solve_ms, nconv = 0, 0.0, 0.0, ninst
    for _ in range(args.steps):
        st = step()
        cycles += st.cycles
        solve_ms += st.ms_total
        inst = L.lbmg_instance_residuals(hb, nrhs)
        rel = max(rel, float(inst.max()))
        nconv = min(nconv, int((inst.max(axis=1) <= tol).sum()))
    e1.record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms, all_cycles = reduce_over_ranks(e0.elapsed_time(e1), cycles, ws, dev)
    value = nu * nrhs * all_cycles / (ms / 1e3)
    # end to end with pinned host buffers
    f_pin = torch.tensor(f, dtype=torch.float64).pin_memory()
    u_pin = torch.zeros((nv, nrhs), dtype=torch.float64).pin_memory()
    step(f_in=f_pin.numpy(), u_out=u_pin.numpy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_cycles = 0
    for _ in range(args.steps):
        e2e_cycles += step(f_in=f_pin.numpy(), u_out=u_pin.numpy()).cycles
    torch.cuda.synchronize()
    e2e_ms, e2e_all = reduce_over_ranks(1e3 * (time.perf_counter() - t0), e2e_cycles, ws, dev)
    e2e_value = nu * nrhs * e2e_all / (e2e_ms / 1e3)
    # plain FP64 on the same batch
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step(L.LBMG_FP64)
    torch.cuda.synchronize()
    g0.record()
    fp64_cycles = step(L.LBMG_FP64).cycles
    g1.record()
    torch.cuda.synchronize()
    fp64_ms = g0.elapsed_time(g1)
    peak, peak_kind = _peaks()
    opts = L.lbmg_default_options()
    cyc_bytes, fixed_bytes = solve_bytes(hb, opts.nu1 + opts.nu2, nrhs)
    launch_bytes = cyc_bytes * (cycles / args.steps) + fixed_bytes
    avg_ms = solve_ms / args.steps
    achieved = launch_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    a_cnt, p_cnt, per_cycle, fixed = L.lbmg_launch_counts(hb, L.LBMG_MIXED)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 relax / f64 assembly, residual with f64 values as f32 pairs", "data": "synthetic",
            "config": {"workload": BATCH, "meshes": ninst, "triangles": int(sum(F.shape[0] for _, F, _ in meshes)),
                       "depths": sorted({int(d) for _, _, d in meshes}), "dofs_finest_total": nu, "nrhs": nrhs,
                       "t": t, "tol": tol, "precision": "mixed",
                       "solve": ("V-cycle-preconditioned CG, per-mesh step lengths, graph per iteration"
                                 if args.solver == "pcg" else "V-cycles, persistent (one launch per solve)"),
                       "l2": "inputs larger than L2 (assembly streams several GB per step)",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "ms_to_tol_mixed": ms / args.steps, "ms_to_tol_fp64": fp64_ms, "cycles_per_step": cycles / args.steps,
            "fp64_cycles_per_step": fp64_cycles, "max_rel_residual_per_mesh": rel,
            "meshes_converged": nconv, "max_cycles": args.max_cycles,
            "setup_s": {"hierarchy_build_and_upload": t_build},
            "solver": args.solver,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": ("whole mixed batch solve, algorithmic bytes of its V-cycles "
                                                     "and FP64 steps over its device time"),
                         "peak_kind": peak_kind, "bytes_per_launch": launch_bytes, "avg_launch_ms": avg_ms},
            "cpu_baseline": None,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(nv * nrhs * 8),
                    "d2h_bytes_per_step": int(nv * nrhs * 8)},
            "gpu_launches": int(args.steps * (a_cnt + p_cnt + 4 + 1)), "clocks": clk,
        }), flush=True)
    L.lbmg_destroy(hb)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lbmg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-min-depth", type=int, default=1,
                    help="coarsest depth of the oracle's V-cycle on its sample (the library's on the default workload)")
    ap.add_argument("--persistent", action="store_true", help="one cooperative launch per solve")
    ap.add_argument("--gpu-clip", action="store_true",
                    help="cut the triangles into finest-voxel pieces on the GPU during the hierarchy build")
    ap.add_argument("--no-graphs", action="store_true", help="launch each cycle's kernels directly (profilers)")
    ap.add_argument("--only-timed", action="store_true", help="stop after the timed steps (profiling runs)")
    ap.add_argument("--learned-zero", action="store_true",
                    help="with --only-timed: time the solve with the learned correction of the zero network (the "
                         "Jacobi start; the same kernels and cost as a trained one) instead of plain cycles")
    ap.add_argument("--no-pdl", action="store_true", help="plain stream order between the cycle's kernels")
    ap.add_argument("--no-tune", action="store_true", help="default launch shapes (no autotuning at setup)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned correction (trained on three small meshes as setup, then timed on the "
                         "workload's own step)")
    ap.add_argument("--learned-steps", type=int, default=800, help="Adam steps of the learned network")
    ap.add_argument("--learned-lr", type=float, default=1e-2)
    ap.add_argument("--solver", default="vcycle", choices=["vcycle", "pcg"],
                    help="V-cycle iteration (the paper's solver, default) or V-cycle-preconditioned CG")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="named synthetic workload (meshgen.CONFIGS); the default is the metric's own configuration")
    ap.add_argument("--tune-cache", default=None,
                    help="tuning cache file: loaded before tuning (matching levels are not timed), saved after")
    ap.add_argument("--cycle", default="v", choices=["v", "w"], help="V-cycle (default) or W-cycle")
    ap.add_argument("--cmcf-steps", type=int, default=3, help="flow steps timed after the main measurement")
    ap.add_argument("--nu", type=int, default=2, help="smoothing sweeps before and after the coarse correction")
    ap.add_argument("--force-shape", default=None,
                    help="TPR,TPB: after tuning, set the finest level's mixed-precision sweep and residual launch "
                         "shape (profiling runs)")
    ap.add_argument("--max-cycles", type=int, default=2000,
                    help="cap on V-cycles per solve (profiling runs cap it to keep launch lists short)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_main(args)
    if args.workload == BATCH:
        return batch_main(args)
    if args.workload == CUBES:
        return cube_main(args)

    import torch

    import meshgen
    import paper_1505_03615_gb300 as L

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    workload = args.workload
    V, F, depth, t, f, tol, _ = meshgen.config_mesh(workload)
    f = f.reshape(V.shape[0], -1)
    nv = V.shape[0]
    t_build = time.perf_counter()
    h = L.lbmg_build_hierarchy(V, F, depth, persistent=int(args.persistent), use_graphs=int(not args.no_graphs),
                               gpu_clip=int(args.gpu_clip),
                               pdl=int(not args.no_pdl), cycle=int(args.cycle == "w"), nu1=args.nu, nu2=args.nu)
    t_build = time.perf_counter() - t_build
    d0, D = L.lbmg_levels(h)
    n, nnz, nfrag = L.lbmg_level_info(h, D)
    nrhs = f.shape[1]
    # setup, like the hierarchy build: launch shapes tuned once per mesh on its own matrices
    L.lbmg_assemble(h, t)
    torch.cuda.synchronize()
    t_tune = time.perf_counter()
    if not args.no_tune:
        if args.tune_cache and os.path.exists(args.tune_cache):
            L.lbmg_tune_cache_load(args.tune_cache)
        for prec in (L.LBMG_MIXED, L.LBMG_FP64):
            L.lbmg_autotune(h, nrhs, prec, reps=4)
        if args.tune_cache:
            L.lbmg_tune_cache_save(args.tune_cache)
    torch.cuda.synchronize()
    t_tune = time.perf_counter() - t_tune
    if args.force_shape:
        tpr, tpb = (int(v) for v in args.force_shape.split(","))
        for kind in (0, 1):
            L.lbmg_set_launch_shape(h, D, L.LBMG_MIXED, kind, tpr, tpb)
    shapes = {str(d): L.lbmg_launch_shape(h, d, L.LBMG_MIXED) for d in range(d0 + 1, D + 1)}
    tuned_us = {str(d): [round(1e3 * v, 2) for v in L.lbmg_tuned_times(h, d, L.LBMG_MIXED)] for d in range(d0 + 1, D + 1)}
    f_dev = torch.tensor(f, dtype=torch.float64, device=dev)
    rhs = torch.zeros((n, nrhs), dtype=torch.float64, device=dev)
    x = torch.zeros_like(rhs)
    u = torch.zeros((nv, nrhs), dtype=torch.float64, device=dev)
    max_cycles = args.max_cycles

    if args.learned_zero:
        if not args.only_timed:
            raise SystemExit("--learned-zero is a profiling switch: use it with --only-timed")
        L.lbmg_learned_params(h, np.zeros(L.lbmg_learned_nparams()))
        L.lbmg_learned_enable(h, True)

    def step(precision=L.LBMG_MIXED):
        L.lbmg_assemble(h, t)
        L.lbmg_project_rhs(h, f_dev, rhs)
        x.zero_()
        solve = L.lbmg_solve_pcg if args.solver == "pcg" else L.lbmg_solve
        code, st = solve(h, rhs, x, tol, max_cycles, precision)
        if code != L.LBMG_OK and not (code == L.LBMG_NOT_CONVERGED and args.max_cycles < 2000):
            raise RuntimeError(f"solve did not converge: {st.rel_residual[:3]}")
        L.lbmg_eval_vertices(h, x, u)
        return st

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.25)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    cycles, smooth_ms, solve_ms, rel = 0, 0.0, 0.0, 0.0
    for _ in range(args.steps):
        st = step()
        cycles += st.cycles
        smooth_ms += st.ms_fine_smooth
        solve_ms += st.ms_total
        rel = max(rel, max(st.rel_residual[:nrhs]))
    e1.record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_max, all_cycles = reduce_over_ranks(e0.elapsed_time(e1), cycles, ws, dev)
    value = n * nrhs * all_cycles / (ms_max / 1e3)
    ms_per_step = ms_max / args.steps
    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms_per_step,
                              "cycles_per_step": cycles / args.steps, "note": "timed steps only"}), flush=True)
        L.lbmg_destroy(h)
        return

    # end to end through the C ABI with host buffers (pinned): H2D of the vertex data,
    # D2H of the evaluated vertex positions, inside the timed region
    f_pin = torch.tensor(f, dtype=torch.float64).pin_memory()
    u_pin = torch.zeros((nv, nrhs), dtype=torch.float64).pin_memory()
    f_np, u_np = f_pin.numpy(), u_pin.numpy()

    def step_e2e():
        L.lbmg_assemble(h, t)
        L.lbmg_project_rhs(h, f_np, rhs)
        x.zero_()
        solve = L.lbmg_solve_pcg if args.solver == "pcg" else L.lbmg_solve
        code, st = solve(h, rhs, x, tol, max_cycles, L.LBMG_MIXED)
        L.lbmg_eval_vertices(h, x, u_np)
        return st

    step_e2e()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_cycles = 0
    for _ in range(args.steps):
        e2e_cycles += step_e2e().cycles
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_all = reduce_over_ranks(1e3 * e2e_s, e2e_cycles, ws, dev)
    e2e_value = n * nrhs * e2e_all / (e2e_ms / 1e3)

    # plain FP64 GPU multigrid on the same mesh: ms to the same tolerance
    fp64_steps = max(1, min(3, args.steps))
    step(L.LBMG_FP64)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record()
    fp64_cycles = 0
    for _ in range(fp64_steps):
        fp64_cycles += step(L.LBMG_FP64).cycles
    g1.record()
    torch.cuda.synchronize()
    fp64_ms = g0.elapsed_time(g1) / fp64_steps

    # the other solver on the same steps: ms to the same tolerance, mixed and FP64
    other = "pcg" if args.solver == "vcycle" else "vcycle"
    other_solve = L.lbmg_solve_pcg if other == "pcg" else L.lbmg_solve
    other_res = {}
    for name, prec in (("mixed", L.LBMG_MIXED), ("fp64", L.LBMG_FP64)):
        def ostep():
            L.lbmg_assemble(h, t)
            L.lbmg_project_rhs(h, f_dev, rhs)
            x.zero_()
            code, st = other_solve(h, rhs, x, tol, max_cycles, prec)
            L.lbmg_eval_vertices(h, x, u)
            return code, st
        ostep()
        torch.cuda.synchronize()
        g0.record()
        its, ok = 0, True
        for _ in range(fp64_steps):
            code, st = ostep()
            its += st.cycles
            ok = ok and code == L.LBMG_OK
        g1.record()
        torch.cuda.synchronize()
        other_res[name] = {"ms_to_tol": g0.elapsed_time(g1) / fp64_steps, "cycles_per_step": its / fp64_steps,
                           "converged": ok}

    # conformalized mean-curvature flow (Section 5.3): a few steps of the library's flow loop
    # (area weights of the current positions, assembly, projection, warm-started solve, vertex
    # evaluation, all on the device), the unit of the paper's Table 1
    learned, params = None, None
    if not args.no_learned and args.solver == "vcycle" and not args.persistent:
        params, hist, train_s = learned_train(L, dev, args.learned_steps, args.learned_lr)
        learned = learned_compare(L, h, step, args.steps, params, hist, train_s, args)
        learned["vs_plain_mixed"] = (ms_per_step / learned["learned"]["ms_to_tol"]) if ws == 1 else None

    def flow(k, with_learned):
        """k steps of the library's flow loop from the build-time positions, after one untimed step"""
        if with_learned:
            L.lbmg_learned_params(h, params)
        L.lbmg_learned_enable(h, with_learned)
        X = torch.tensor(V, device=dev)
        xc = torch.zeros((n, 3), dtype=torch.float64, device=dev)
        Xn = torch.zeros_like(X)
        solver = 1 if args.solver == "pcg" else 0
        L.lbmg_cmcf_step(h, X, t, xc, tol, max_cycles, L.LBMG_MIXED, Xn, solver=solver)
        X, Xn = Xn, X
        torch.cuda.synchronize()
        g0.record()
        ccyc, fb = 0, 0
        for _ in range(k):
            code, st = L.lbmg_cmcf_step(h, X, t, xc, tol, max_cycles, L.LBMG_MIXED, Xn, solver=solver)
            ccyc += st.cycles
            fb = max(fb, st.learned_fallback)
            X, Xn = Xn, X
        g1.record()
        torch.cuda.synchronize()
        L.lbmg_set_area_weights(h, None)
        L.lbmg_learned_enable(h, False)
        return {"ms_per_step": g0.elapsed_time(g1) / k, "cycles_per_step": ccyc / k, "fallback": fb}

    # conformalized mean-curvature flow (Section 5.3): a few steps of the library's flow loop
    # (area weights of the current positions, assembly, projection, warm-started solve, vertex
    # evaluation, all on the device), the unit of the paper's Table 1; also with the learned
    # correction when it was trained
    cmcf = None
    if args.cmcf_steps > 0:
        cmcf = {"steps": args.cmcf_steps, "delta": t, "solver": args.solver, "precision": "mixed",
                "warm_start": True, **flow(args.cmcf_steps, False)}
        if params is not None:
            cmcf["learned"] = flow(args.cmcf_steps, True)

    # roofline of the dominant kernel (the finest-level Gauss-Seidel colour), timed live with
    # CUDA events on its stream: the timed steps run each solve as one graph launch, whose
    # conditional loop cannot hold event records, so the same step is replayed with the host
    # stopping test (one graph per cycle, events around the finest pre- and post-smoothing)
    a_cnt, p_cnt, per_cycle, fixed = L.lbmg_launch_counts(h, L.LBMG_MIXED)
    opts = L.lbmg_default_options()
    sweeps = opts.nu1 + opts.nu2
    peak, peak_kind = _peaks()
    R = 4 if nrhs > 2 else nrhs
    if args.persistent:
        cyc_bytes, fixed_bytes = solve_bytes(h, sweeps, nrhs)
        launch_bytes = cyc_bytes * (cycles / args.steps) + fixed_bytes
        avg_launch_ms = solve_ms / args.steps
        roof_cycles = cycles / args.steps
        kernel = f"solve_persistent_kernel<float,{R}> (whole mixed solve, one launch)"
        key = f"solve_persistent_{workload}"
    else:
        L.lbmg_set_host_check(h, 1)
        roof_smooth, roof_cycles = 0.0, 0
        for _ in range(2):
            st = step()
            roof_smooth, roof_cycles = st.ms_fine_smooth, st.cycles
        L.lbmg_set_host_check(h, 0)
        # algorithmic bytes per colour launch (one eighth of a sweep): nnz (4 B value + 4 B
        # column) + n nrhs (4 B right-hand side + 4 B x read + 4 B x write)
        launch_bytes = (nnz * 8 + n * nrhs * 12) / 8
        avg_launch_ms = roof_smooth / max(roof_cycles * sweeps * 8, 1)
        tpr, tpb = shapes[str(D)][0]
        kname = "pk_row_kernel" if tpr == 4 else "smooth_colour_kernel"
        kernel = f"{kname}<float,{R},GS> (finest level, one colour, {tpr} threads per row, {tpb} threads/block)"
        key = f"{kname}_gs_{workload}"
    achieved = launch_bytes / (avg_launch_ms * 1e-3) / 1e9 if avg_launch_ms > 0 else 0.0
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tr = json.load(fh).get(key)
            # counters apply only to the kernel instance they were taken from
            same = args.persistent or (tr and [tr.get("threads_per_row"), tr.get("threads_per_block")] ==
                                       list(shapes[str(D)][0]))
            if tr and same:
                traffic = tr["bytes_per_launch"]
    except Exception:
        pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kernel, "peak_kind": peak_kind, "bytes_per_launch": launch_bytes,
                "avg_launch_ms": avg_launch_ms,
                "timing": "CUDA events in the per-cycle graph around the finest smoothing of a replayed step "
                          f"({roof_cycles} cycles x {sweeps} sweeps x 8 colour launches and their gaps)",
                "solve_ms_per_step": solve_ms / args.steps}

    gpu_launches = args.steps * (a_cnt + p_cnt + fixed + 1) + cycles * per_cycle

    cpu_baseline = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        v1, dt1, n1 = oracle_baseline(V, F, depth, d0, t, 1)
        vp, dtp, npc = oracle_baseline(V, F, depth, d0, t, cores)
        cpu_baseline = {"value": vp, "unit": UNIT, "cores": cores, "kind": "oracle",
                        "sample": f"{SAMPLE_CYCLES} FP64 lexicographic-GS V-cycles x 3 right-hand sides per core, "
                                  f"each core on its own stretch of {SAMPLE_TRIS} consecutive triangles of the same "
                                  f"mesh on its grid (depth {depth}, coarsest depth {d0}, about {int(np.mean(npc))} "
                                  f"finest functions each), spawned processes started together; {dtp:.1f} s",
                        "single_core": {"value": v1, "cores": 1, "seconds": dt1, "finest_functions": n1[0]}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 relax / f64 assembly, residual with f64 values as f32 pairs", "data": "synthetic",
            "config": {"workload": workload, "triangles": int(F.shape[0]), "depth": depth, "min_depth": d0,
                       "dofs_finest": n, "nnz_finest": nnz, "fragments_finest": nfrag, "nrhs": nrhs, "t": t,
                       "tol": tol, "precision": "mixed", "l2": "inputs larger than L2 (assembly streams >0.5 GB/step)",
                       "cycle": f"{args.cycle.upper()}({args.nu},{args.nu})",
                       "assembly": ("every step: the finest entries gathered from the pieces' local integrals (mass "
                                    "scaled by the current area weights), the Galerkin products of every coarser "
                                    "level, A = M + tL and its packed and FP32 copies; the pieces' moments and local "
                                    "integrals depend only on the build-time geometry and are computed by the first "
                                    "assembly (setup)"),
                       "parallelism": "replicas" if ws > 1 else "single",
                       "solve": ("persistent (one cooperative launch)" if args.persistent else
                                 "one graph launch per solve (conditional loop, device stopping test)"),
                       "dependent_launch": not args.no_pdl and not args.persistent,
                       "launch_shapes_mixed": {d: {"sweep": list(v[0]), "residual": list(v[1])}
                                               for d, v in shapes.items()},
                       "tuned_us_per_sweep_and_residual": tuned_us},
            "setup_s": {"hierarchy_build_and_upload": t_build, "autotune": t_tune,
                        "pieces_cut_on": "gpu" if args.gpu_clip else "host cores"},
            "ms_to_tol_mixed": ms_per_step, "ms_to_tol_fp64": fp64_ms, "solver": args.solver,
            "other_solver": {"solver": other, **other_res}, "learned": learned, "cmcf": cmcf,
            "cycles_per_step": cycles / args.steps, "fp64_cycles_per_step": fp64_cycles / fp64_steps,
            "max_rel_residual": rel,
            "roofline": roofline, "cpu_baseline": cpu_baseline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(nv * nrhs * 8),
                    "d2h_bytes_per_step": int(nv * nrhs * 8)},
            "gpu_launches": int(gpu_launches), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    L.lbmg_destroy(h)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

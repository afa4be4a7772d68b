#!/usr/bin/env python
"""Benchmark of the trust-region / Steihaug-CG homogenisation solver on one GB300.

Workload (N=1): the 256^3 random-sphere RVE -- 144 non-overlapping spheres,
radius U[4, 10] voxels, seed 0, stiff elastic spheres (E=10, nu=0.2) in a
damaging matrix (E=1, nu=0.3, kappa0=1e-4, kappaf=1e-3) -- under uniaxial
mean strain eps_zz ramped in increments of 5e-5 (2e-3 over 40 increments),
the other five mean components stress-free.  FP32 fields, FP64 reductions,
relative residual |G:sigma|/|sigma| <= 1e-6.

A bench *step* is one load increment (Algorithm 2) from a fixed reference
state (the unloaded cell, reset with rve_set_state at the start of every
step, which re-evaluates the constitutive law): uniform predictor,
constitutive update, gradient, and trust-region Newton iterations, each one
a Steihaug-CG solve (Hessian-vector products: tangent + forward FFT +
projection + inverse FFT, CG reductions and updates) followed by the trial
constitutive evaluation, the first-order incremental-energy ratio test and
the new gradient.  value = voxels x Hessian-vector products / time (all
ranks), ms_per_step = the load-step time.  The first increment stays below
the damage threshold; later increments localise a crack band and take
10^4-10^5 products each, too long for a bench run of minutes.

--workload asr times the same kind of step on the cell read as an ASR-like
concrete model (Sec. 3.3): the spheres as damaging aggregates in a damaging
cement paste, single gel voxels inside the aggregates expanding by 5e-4 per
step through the per-phase eigenstrain of Algorithm 2, all mean components
stress-free.

--workload lbfgs solves the default load step by L-BFGS (the quasi-Newton
method the first-order incremental energy makes usable, with Eq. (18) in its
line search) and by the trust-region solver, and prints the L-BFGS step time
with the trust-region time beside it.

Roofline: the dominant kernel's average launch time comes from CUDA events
recorded by the library around every launch inside the timed region;
algorithmic bytes per launch are the compulsory reads + writes of that pass.

--impl reference times the FP64 CPU oracle (the repo's plain restatement of
the method, single thread): each step is one Hessian-vector product on a
bounded sample of the workload, the 128^3 cell of the same sphere model
(48 spheres) with a damage snapshot D ~ U[0, 0.9] on the matrix, so that
--steps 10 --warmup 3 ends within a few minutes.  The GPU arm's cpu_baseline
times one oracle product on the full 256^3 cell.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-Hv/s at 256³ (% HBM roofline); load-step time, warm start vs plain @1e-6"
UNIT = "voxel-Hv/s"
N = 256
INC = 5e-5
MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)
FREE = [1, 1, 0, 1, 1, 1]
WORKLOAD = ("256^3 random-sphere RVE (144 spheres, r~U[4,10], seed 0; spheres E=10 nu=0.2 elastic, matrix "
            "E=1 nu=0.3 damaging kappa0=1e-4 kappaf=1e-3), uniaxial eps_zz increments 5e-5 (40 to 2e-3), "
            "other components stress-free, trust-region Newton + Steihaug CG to rel. residual 1e-6")
# ASR-like cell (Sec. 3.3): Table 2's aggregate / cement paste / ASR product constants (E in GPa,
# kappa0 = f_t / E, zero stiffness at 10 kappa0), gel voxels expanding by the paper's medium step
ASR_STEP = 5e-4
ASR_PHASES = [(12.0, 0.3, True, 2.5e-4, 2.5e-3), (59.0, 0.3, True, 10.0 / 59000.0, 100.0 / 59000.0),
              (11.0, 0.18, False, 0.0, 0.0)]
ASR_WORKLOAD = ("256^3 ASR-like cell: the 144 spheres of the load-step workload as aggregates (E=59 nu=0.3, "
                "damaging, kappa0=f_t/E=1.69e-4, kappaf=10 kappa0) in a cement paste (E=12 nu=0.3, kappa0=2.5e-4, "
                "kappaf=10 kappa0), 288 single gel voxels drawn inside the aggregates (E=11 nu=0.18, elastic) "
                "with a stress-free expansion of 5e-4 per normal component (eigenstrain -5e-4, Algorithm 2), "
                "every mean component stress-free (free expansion); a step = that expansion increment from the "
                "unloaded cell, trust-region Newton + Steihaug CG to rel. residual 1e-6")


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=N, help="grid size (default 256)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-onset", action="store_true", help="skip the damage-onset step of the default line")
    p.add_argument("--workload", default="rve256",
                   choices=["rve256", "asr", "lbfgs", "onset", "batch96", "warmstart", "hv", "control"],
                   help="rve256: the 256^3 sphere cell (default); asr: the same cell as an ASR-like "
                        "aggregate / paste / gel model loaded by gel eigenstrain; lbfgs: the default load step "
                        "solved by L-BFGS and by trust-region Newton-CG; onset: a load step at the onset of "
                        "damage with the secant and the symmetric consistent Hessian; batch96: 96 cells of "
                        "uneven sizes; "
                        "warmstart: train the spectral neural operator, then learned vs plain load steps; "
                        "hv: Hessian-vector products alone (damage snapshot, compatible input), several sizes; "
                        "control: device-side vs host-stepped Steihaug-CG control at 32^2 and 128^3")
    p.add_argument("--lbfgs-memory", type=int, default=5, help="lbfgs: (s, y) pairs kept")
    p.add_argument("--hv-sizes", default="128,256,384", help="hv: cube edge lengths")
    p.add_argument("--onset-sizes", default="128,256", help="onset: cube edge lengths")
    p.add_argument("--hv-precisions", default="32,64", help="hv: 32 and / or 64")
    p.add_argument("--ws-train-seconds", type=float, default=120.0,
                   help="warmstart: time budget of the training-data generation (plain solves at 64^3)")
    p.add_argument("--ws-iters", type=int, default=4000, help="warmstart: Adam iterations")
    p.add_argument("--ws-hessian", type=int, default=1, choices=[0, 1],
                   help="warmstart: Hessian of every solve (0 secant, 1 symmetric consistent tangent)")
    p.add_argument("--ws-eval", default="128,128,192", help="warmstart: held-out evaluation grids")
    p.add_argument("--probe", choices=["step", "fno"], default=None,
                   help="untimed small case for profilers: 'step' = one load step of a 256x256x128 sphere cell, "
                        "'fno' = three training iterations of the spectral neural operator at 64^3, batch 4")
    p.add_argument("--passes", type=int, default=0, choices=[0, 1, 2, 3],
                   help="rve_solver_opts.passes of the timed solver: 0 compiled five passes (default), 3 compiled "
                        "with the cluster x+y passes, 2 unfused CG, 1 generic")
    p.add_argument("--host-loop", action="store_true",
                   help="step the Steihaug-CG iterations from the host in every timed step (the same kernels as "
                        "the device-side graph loop, each a separate launch; for profilers, which do not take "
                        "the kernels inside conditional graph nodes)")
    p.add_argument("--probe-dims", default="256,256,128",
                   help="probe step: grid (nx,ny,nz); 256,128,256 gives the length-256 z pass the benchmark runs")
    p.add_argument("--batch-hessian", type=int, default=1, choices=[0, 1],
                   help="batch96: Hessian of the batched solves (0 secant, 1 symmetric consistent tangent)")
    p.add_argument("--batch-increments", type=int, default=0,
                   help="batch96: after the timed step, run this many increments of the load path from the "
                        "unloaded cells and report converged members per increment (the configuration's 30)")
    p.add_argument("--batch-max-nr", type=int, default=50,
                   help="Newton cap per member for batch96 (bounds the work of members that localise)")
    return p.parse_args()


# ----------------------------------------------------------------- helpers
def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash():
    """Hash of the sources of the kernels whose DRAM counters
    profiles/traffic.json holds (spectral passes, constitutive and CG vector
    kernels).  The network, the batched solver, the allocation-free
    projection, the L-BFGS and homogenisation kernels and the host-side control loop
    (rve_api.cu: entry points and one-thread scalar kernels) live in files of
    their own and do not enter it."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2207_10657_gb300", "csrc")
    skip = {"fno.cu", "batch.cu", "noalloc.cu", "lbfgs.cu", "lbfgs.cuh", "homogenize.cu", "homogenize.cuh",
            "consistent.cu", "consistent.cuh", "rve_api.cu"}
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")) and fn not in skip:
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(fn.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel, n):
    """DRAM bytes per launch of `kernel` at size n from the committed ncu
    summary, or None if absent or taken on different kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("kernel_hash") != _kernel_hash():
        return None
    rec = d.get("kernels", {}).get(f"{kernel}@{n}")
    return None if rec is None else rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

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
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(dist, ms, count, device):
    """Whole-job timing over the ranks of a replicas run: the slowest rank's
    time (MAX) and the units all ranks processed (SUM).  dist None: one rank."""
    if dist is None:
        return float(ms), float(count)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(count)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), float(c[0])


# ------------------------------------------------------------ CPU oracle
def _oracle_hv_setup(n):
    import numpy as np
    import oracle
    from synth import random_spheres, damage_snapshot, random_field
    dims = (n, n, n)
    pm = random_spheres(dims, count=144 if n >= 256 else 48, rmin=4.0, rmax=10.0, seed=0)
    D = damage_snapshot(pm, dmax=0.9, seed=1).astype(np.float64)
    v = random_field(6, dims, seed=2)
    rve = oracle.RVE(pm, [oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3), oracle.Phase(10.0, 0.2)])
    return rve, D, v


def _oracle_hv_time(n, reps=1):
    rve, D, v = _oracle_hv_setup(n)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        rve.hessp(D, v)
        ts.append(time.perf_counter() - t0)
    return ts


def _oracle_hv_worker(args):
    """One spawned process: set up the oracle's product on an n^3 cell, wait
    for the others, time one product."""
    n, barrier = args
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    rve, D, v = _oracle_hv_setup(n)
    barrier.wait()
    t0 = time.perf_counter()
    rve.hessp(D, v)
    return time.perf_counter() - t0


def _oracle_hv_all_cores(n):
    """The oracle's product timed on every host core at once: one
    single-threaded process per core (spawned: this process has a CUDA
    context), each on its own copy of the n^3 cell.  Returns (voxel-Hv/s of
    all processes together, processes, slowest time)."""
    import multiprocessing as mp
    procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(procs)
        with ctx.Pool(procs) as pool:
            ts = pool.map(_oracle_hv_worker, [(n, barrier)] * procs)
    return procs * n ** 3 / max(ts), procs, max(ts)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    n = min(args.n, 128)
    rve, D, v = _oracle_hv_setup(n)
    for _ in range(args.warmup):
        rve.hessp(D, v)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rve.hessp(D, v)
    dt = time.perf_counter() - t0
    val = args.steps * n ** 3 / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [n, n, n]},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"one FP64 Hessian-vector product per step on the {n}^3 cell of the same "
                                   "sphere model (damage snapshot D~U[0,0.9] on the matrix), numpy, 1 thread"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ GPU arm
HV_PASSES = ("xfwd_tangent", "y_fwd", "z_proj", "y_inv", "x_inv")


def _pass_bytes(n, pass_name):
    """Algorithmic (compulsory) DRAM bytes of one launch of a pass at n^3, FP32."""
    nvox = n ** 3
    spec = 6 * n * n * (n // 2 + 1) * 8  # half spectrum, 6 complex components
    field = 6 * nvox * 4
    return {
        "xfwd_tangent": field + nvox * (1 + 4) + spec,
        "y_fwd": 2 * spec,
        "z_proj": 2 * spec,
        "y_inv": 2 * spec,
        # CG products: the x-inverse applies z += alpha d, r += alpha Hd (reads z, r, d;
        # writes z, r) instead of storing Hd
        "x_inv": spec + 5 * field,
        "x_inv_plain": spec + field,  # the product alone (rve_hessp): the half spectrum in, H v out
        "trial": nvox * (24 + 24 + 4 + 24 + 4 + 1 + 24 + 4 + 4),
        "cg_vec": nvox * 96,  # direction update: reads z, r, d, writes d
    }.get(pass_name)


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    torch.cuda.set_device(local)
    from paper_2207_10657_gb300 import build as _build
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    from paper_2207_10657_gb300 import RVESolver, binding
    from synth import gel_sites, random_spheres

    n = args.n
    dims = (n, n, n)
    nvox = n ** 3
    nsph = 144 if n >= 256 else 48
    pm = random_spheres(dims, count=nsph, rmin=4.0, rmax=10.0, seed=0)
    asr = args.workload == "asr"
    st = torch.cuda.Stream()
    if asr:
        pm = gel_sites(pm, 2 * nsph, host=1, site=2, seed=3)
        R0 = 10.0 * (nvox ** 0.5) * ASR_STEP
        with torch.cuda.stream(st):
            s = RVESolver(dims, pm, ASR_PHASES, precision=32, stream=st, eta_eq=1e-6, eta_cg=1e-2, max_nr=400,
                          R0=R0, Rmax=R0, passes=args.passes)
        s.set_eigenstrain([[0.0] * 6, [0.0] * 6, [-ASR_STEP] * 3 + [0.0] * 3])
        dE, free, workload = [0.0] * 6, [1] * 6, ASR_WORKLOAD
    else:
        with torch.cuda.stream(st):
            s = RVESolver(dims, pm, [MATRIX, STIFF], precision=32, stream=st, eta_eq=1e-6, eta_cg=1e-2,
                          max_nr=400, passes=args.passes)
        dE, free, workload = [0.0, 0.0, INC, 0.0, 0.0, 0.0], FREE, WORKLOAD
    if args.host_loop:
        binding.rve_set_device_loop(s.h, False)
    eps0 = s.field(0.0)  # reference state: the unloaded cell

    def step():
        s.set_state(eps0)
        return s.solve_step(dE, free_mask=free, raise_on_error=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---------------- timed region: K load steps (device-resident inputs).
    # The Steihaug iterations run as device-side graph loops here.
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    hv0, l0, y0 = s.hv_count, s.launch_count, s.sync_count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(st)
    timed = []
    for _ in range(args.steps):
        timed.append(step())
    ev1.record(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop() if sampler else None
    hv = s.hv_count - hv0
    launches = s.launch_count - l0
    syncs = s.sync_count - y0
    ms_max, hv_all = reduce_over_ranks(dist, ms, hv, "cuda")
    value = hv_all * nvox / (ms_max / 1e3)

    # ---------------- per-pass device times: the same steps again with CUDA
    # events around every pass launch (this steps the Steihaug iterations
    # from the host, since events cannot be recorded inside the device loop)
    binding.rve_pass_timing(s.h, True)
    y1 = s.sync_count
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(st)
    for _ in range(args.steps):
        step()
    ev3.record(st)
    torch.cuda.synchronize()
    ms_host = ev2.elapsed_time(ev3)
    syncs_host = s.sync_count - y1
    stats = binding.rve_pass_stats(s.h)
    binding.rve_pass_timing(s.h, False)

    # ---------------- end to end through the public API with host buffers:
    # per step, the reference strain field is copied from pinned host memory,
    # the load step runs (dE is a host argument of rve_solve_step), and the
    # converged strain field is read back to pinned host memory.
    host_in = torch.zeros((6,) + pm.shape, dtype=torch.float32).pin_memory()
    host_out = torch.empty((6,) + pm.shape, dtype=torch.float32).pin_memory()
    dev_in = s.field()
    dev_out = s.field()
    e2e_steps = max(1, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    hv_e0 = s.hv_count
    for _ in range(e2e_steps):
        with torch.cuda.stream(st):
            dev_in.copy_(host_in, non_blocking=True)
        s.set_state(dev_in)
        s.solve_step(dE, free_mask=free, raise_on_error=False)
        binding.rve_get_state(s.h, dev_out.data_ptr())
        with torch.cuda.stream(st):
            host_out.copy_(dev_out, non_blocking=True)
        st.synchronize()
    e2e_s = time.perf_counter() - t0
    hv_e = s.hv_count - hv_e0
    e2e_max, hv_e_all = reduce_over_ranks(dist, e2e_s, hv_e, "cuda")
    e2e_val = hv_e_all * nvox / e2e_max

    # ---------------- roofline of the dominant pass
    dom = max((k for k in stats if stats[k][0] > 0), key=lambda k: stats[k][1])
    cnt, tot = stats[dom]
    avg_s = tot / cnt / 1e3
    bytes_launch = _pass_bytes(n, dom)
    peak, peak_kind = _peaks()
    achieved = bytes_launch / avg_s / 1e9
    traffic = _traffic(dom, n)
    # passes that launched: with the x and y passes merged (Nx = Ny compiled sizes)
    # the y passes run inside the x launches and their spectrum stays in L2
    hv_passes = [k for k in HV_PASSES if stats[k][0] > 0]
    hv_only_ms = sum(stats[k][1] for k in hv_passes)
    hv_bytes = sum(_pass_bytes(n, k) for k in hv_passes)
    nprod = max(stats["z_proj"][0], 1)
    # DRAM bytes of the same passes from the committed ncu record (None if it
    # was taken on other kernel sources)
    ncu_parts = [_traffic(k, n) for k in hv_passes]
    ncu_bytes = sum(ncu_parts) if ncu_parts and all(x is not None for x in ncu_parts) else None

    # ---------------- a load step at the damage onset (past kappa0), where the
    # Newton iterations and not the product dominate: both Hessians
    onset = None
    if rank == 0 and not asr and not args.no_onset:
        onset, _ = _onset_measure(n, 1, 1, st, args.passes)
        onset = {"workload": ONSET_WORKLOAD, **onset}

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        # bounded oracle sample on the host cores (one FP64 Hv of the same workload)
        try:
            for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
                os.environ.setdefault(var, "1")
            ts = _oracle_hv_time(n, reps=1)
            n_all = min(n, 128)
            v_all, procs, t_all = _oracle_hv_all_cores(n_all)
            cpu = {"value": v_all, "unit": UNIT, "cores": procs, "kind": "oracle",
                   "sample": f"one FP64 Hessian-vector product in each of {procs} single-threaded processes at "
                             f"once (one per host core), each on its own {n_all}^3 cell of the same sphere model "
                             f"(damage snapshot D~U[0,0.9]), numpy; slowest process {t_all:.1f} s",
                   "one_core": {"value": nvox / ts[0], "unit": UNIT, "cores": 1,
                                "sample": f"one FP64 Hessian-vector product of the {n}^3 workload, numpy, "
                                          f"1 thread, {ts[0]:.1f} s"}}
        except Exception as ex:  # report, do not hide
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "grid": [n, n, n], "parallelism": f"replicas x{ws}",
                   "passes": args.passes, "host_loop": bool(args.host_loop),
                   "l2": "inputs larger than L2 (each 6-component FP32 field is 403 MB > 129 MB L2)",
                   "hv_per_step": hv / args.steps,
                   "nr_iters_per_step": [r["nr_iters"] for r in timed],
                   "cg_iters_per_step": [r["cg_iters"] for r in timed],
                   "converged": [r["converged"] for r in timed],
                   "mean_stress_zz": [r["mean_stress"][2] for r in timed],
                   "mean_strain_volumetric": [sum(r["mean_strain"][:3]) for r in timed],
                   "onset_step": onset,
                   "host_waits_per_step": syncs / args.steps,
                   "host_stepped_cg": {"ms_per_step": ms_host / args.steps,
                                       "host_waits_per_step": syncs_host / args.steps},
                   "hv_only_ms": hv_only_ms / nprod,
                   "hv_only_voxel_hv_per_s": nvox / (hv_only_ms / nprod / 1e3),
                   "pass_ms_per_launch": {k: (v[1] / v[0] if v[0] else None) for k, v in stats.items()}},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_launch},
        "hv_roofline": {"bound": "hbm", "passes": hv_passes,
                        "what": "one CG iteration's product: the passes that launched -- the five separate passes "
                                "(default), or with --passes 3 the x+y forward cluster pass (as x_fwd), the z pass "
                                "and the y+x inverse cluster pass (as x_inv) -- with the Steihaug iterate / "
                                "residual update of the inverse x pass (its reads of z, r, d and writes of z, r) "
                                "counted",
                        "achieved": hv_bytes / (hv_only_ms / nprod / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": hv_bytes / (hv_only_ms / nprod / 1e3) / 1e9 / peak,
                        "algorithmic_bytes_per_product": hv_bytes,
                        "product_alone_bytes": hv_bytes - _pass_bytes(n, "x_inv") + _pass_bytes(n, "x_inv_plain"),
                        "ncu_dram_bytes_per_product": ncu_bytes,
                        "ncu_frac": (ncu_bytes / (hv_only_ms / nprod / 1e3) / 1e9 / peak) if ncu_bytes else None},
        "compulsory_fraction": {"bytes_per_voxel": 53, "frac": 53 * nvox / (hv_only_ms / nprod / 1e3) / 1e9 / peak},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 6 * nvox * 4,
                "d2h_bytes_per_step": 6 * nvox * 4},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    s.close()
    if dist:
        dist.destroy_process_group()
    return 0


BATCH_WORKLOAD = ("96 RVEs of uneven sizes in one batched solver: 48 2D square grids N^2, N drawn from the even "
                  "5-smooth sizes in [64, 512] (random discs, area fraction U[0.1, 0.4]) and 48 3D grids N^3, N from "
                  "the even 5-smooth sizes in [32, 96] (random spheres, volume fraction U[0.1, 0.3]); each with its "
                  "own seeded microstructure and a random unit load direction (full strain control) scaled so 30 "
                  "increments reach Frobenius norm 2e-3; one step = the first increment of every member from the "
                  "unloaded state")


def batch96_members(seed=0):
    import numpy as np
    from synth import five_smooth_sizes, random_circles, random_spheres
    rng = np.random.default_rng(seed)
    s2 = [n for n in five_smooth_sizes(64, 512) if n % 2 == 0]
    s3 = [n for n in five_smooth_sizes(32, 96) if n % 2 == 0]
    dims, pms, dEs = [], [], []
    for k in range(96):
        if k < 48:
            n = int(rng.choice(s2))
            d = (n, n)
            pm = random_circles(d, target_frac=float(rng.uniform(0.1, 0.4)), rmin=n / 32, rmax=n / 10,
                                seed=1000 + k)
            nc = 3
        else:
            n = int(rng.choice(s3))
            d = (n, n, n)
            pm = random_spheres(d, count=None, rmin=n / 16, rmax=n / 8, seed=1000 + k,
                                target_frac=float(rng.uniform(0.1, 0.3)))
            nc = 6
        a = rng.standard_normal(nc)
        a *= 2e-3 / 30 / np.linalg.norm(a)
        dims.append(d)
        pms.append(pm)
        dEs.append(list(a))
    return dims, pms, dEs


def run_batch(args):
    import torch
    from paper_2207_10657_gb300 import RVEBatch, RVESolver, build as _build
    _build.build()
    dims, pms, dEs = batch96_members()
    nvox = [int(np_prod(d)) for d in dims]
    free = [[0] * (3 if len(d) == 2 else 6) for d in dims]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b = RVEBatch(dims, pms, [MATRIX, STIFF], stream=st, eta_eq=1e-6, eta_cg=1e-2, max_nr=args.batch_max_nr,
                     hessian=args.batch_hessian)
        tuned = b.autotune(reps=3)

    def step():
        b.reset()
        return b.solve_step(dEs, free, raise_on_error=False)

    for w in range(args.warmup):
        t0 = time.perf_counter()
        r = step()
        print(f"batch warm-up {w}: {time.perf_counter() - t0:.2f} s, converged "
              f"{sum(x['converged'] for x in r)}/{len(r)}, max nr {max(x['nr_iters'] for x in r)}",
              file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    hv0, l0 = b.hv_count, b.launch_count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    reps = []
    for _ in range(args.steps):
        reps = step()
    ev1.record(st)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    print(f"batch timed: {ms / args.steps:.1f} ms/step", file=sys.stderr, flush=True)
    # voxel-Hv: each member's products times its voxels
    per_step = sum(r["hv_products"] * nv for r, nv in zip(reps, nvox))
    value = per_step * args.steps / (ms / 1e3)
    launches = b.launch_count - l0
    path = None
    if args.batch_increments > 0:
        # the load path: increments accumulate from the unloaded cells
        b.reset()
        path = []
        for k in range(args.batch_increments):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            rk = b.solve_step(dEs, free, raise_on_error=False)
            e1.record(st)
            torch.cuda.synchronize()
            nr = [x["nr_iters"] for x in rk]
            path.append({"increment": k + 1, "converged": sum(1 for x in rk if x["converged"]),
                         "nr_mean": sum(nr) / len(nr), "nr_max": max(nr),
                         "hv_mean": sum(x["hv_products"] for x in rk) / len(rk), "ms": e0.elapsed_time(e1)})
            print(f"batch path increment {k + 1}: {path[-1]}", file=sys.stderr, flush=True)
    b.close()
    # the same members solved one after another with single-cell contexts
    singles = []
    with torch.cuda.stream(st):
        for d, pm in zip(dims, pms):
            singles.append(RVESolver(d, pm, [MATRIX, STIFF], precision=32, stream=st, eta_eq=1e-6, eta_cg=1e-2,
                                     max_nr=args.batch_max_nr, hessian=args.batch_hessian))
    zero = [s.field(0.0) for s in singles]
    for s, z, de, fm in zip(singles, zero, dEs, free):
        s.set_state(z)
        s.solve_step(de, free_mask=fm, raise_on_error=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hv_single = 0
    for s, z, de, fm in zip(singles, zero, dEs, free):
        s.set_state(z)
        r = s.solve_step(de, free_mask=fm, raise_on_error=False)
        hv_single += r["hv_products"] * int(np_prod(s.dims))
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    for s in singles:
        s.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "members": len(dims), "total_voxels": sum(nvox),
                   "converged": sum(1 for r in reps if r["converged"]),
                   "hv_per_member_mean": sum(r["hv_products"] for r in reps) / len(reps),
                   "sequential_single_contexts_ms": t_single * 1e3,
                   "sequential_single_contexts_voxel_hv_per_s": hv_single / t_single,
                   "batched_speedup": (t_single * 1e3) / (ms / args.steps),
                   "hessian": "consistent" if args.batch_hessian else "secant",
                   "max_nr": args.batch_max_nr, "path": path,
                   "autotune": tuned},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_lbfgs(args):
    """The default load step (256^3 sphere cell, first increment from the
    unloaded state) solved by L-BFGS with the first-order energy line search
    and by trust-region Newton-CG, timed alike (CUDA events, K steps)."""
    import torch
    from paper_2207_10657_gb300 import RVESolver, build as _build
    from synth import random_spheres
    _build.build()
    n = args.n
    dims = (n, n, n)
    pm = random_spheres(dims, count=144 if n >= 256 else 48, rmin=4.0, rmax=10.0, seed=0)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = RVESolver(dims, pm, [MATRIX, STIFF], precision=32, stream=st, eta_eq=1e-6, eta_cg=1e-2, max_nr=400)
    dE = [0.0, 0.0, INC, 0.0, 0.0, 0.0]
    eps0 = s.field(0.0)

    def lb_step():
        s.set_state(eps0)
        return s.solve_step_lbfgs(dE, free_mask=FREE, memory=args.lbfgs_memory, max_iter=5000,
                                  raise_on_error=False)

    def tr_step():
        s.set_state(eps0)
        return s.solve_step(dE, free_mask=FREE, raise_on_error=False)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = s.launch_count
        ev0.record(st)
        reps = [fn() for _ in range(args.steps)]
        ev1.record(st)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / args.steps, reps, s.launch_count - l0

    sampler = ClockSampler(0)
    sampler.start()
    lb_ms, lb_reps, lb_launch = timed(lb_step)
    clocks = sampler.stop()
    tr_ms, tr_reps, _ = timed(tr_step)
    s.close()
    line = {
        "metric": "load-step time at 256³: L-BFGS (first-order energy line search) vs trust-region Newton-CG",
        "value": lb_ms, "unit": "ms/load step", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": lb_ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + "; the same load step by L-BFGS (memory "
                   f"{args.lbfgs_memory}) and by the trust-region solver",
                   "l2": "inputs larger than L2 (each 6-component FP32 field is 403 MB > 129 MB L2)",
                   "lbfgs_iters_per_step": [r["nr_iters"] for r in lb_reps],
                   "lbfgs_trials_per_step": [r["cg_iters"] for r in lb_reps],
                   "lbfgs_halvings_per_step": [r["rejected"] for r in lb_reps],
                   "lbfgs_converged": [r["converged"] for r in lb_reps],
                   "lbfgs_mean_stress_zz": [r["mean_stress"][2] for r in lb_reps],
                   "trust_region_ms_per_step": tr_ms,
                   "trust_region_hv_per_step": [r["hv_products"] for r in tr_reps],
                   "trust_region_mean_stress_zz": [r["mean_stress"][2] for r in tr_reps],
                   "speedup_over_trust_region": tr_ms / lb_ms},
        "gpu_launches": lb_launch, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_control(args):
    """Host-wait cost of Algorithm 1's control: the same load steps with the
    Steihaug iterations as device-side graph loops and stepped from the host
    (rve_set_device_loop), on the 2D configuration-1 cell (32^2 plane strain,
    centred inclusion, the first three increments of 1e-4, FP32) and on the
    128^3 sphere cell (the default first increment, FP32)."""
    import numpy as np
    import torch
    from paper_2207_10657_gb300 import RVESolver, binding, build as _build
    from synth import circular_inclusion, random_spheres
    _build.build()
    st = torch.cuda.Stream()
    cases = []
    pm2 = circular_inclusion((32, 32), 0.3)
    R2 = 10 * np.sqrt(32 * 32) * 1e-4
    cases.append(("2D 32^2 plane strain, centred inclusion (vol. frac 0.3), eps_xx += 1e-4 three times from "
                  "the unloaded cell, other components stress-free",
                  (32, 32), pm2, [MATRIX, (10.0, 0.3, False, 0.0, 0.0)], [[1e-4, 0, 0]] * 3, [0, 1, 1],
                  dict(R0=R2, Rmax=R2, max_nr=400, max_cg=500)))
    pm3 = random_spheres((128, 128, 128), count=48, rmin=4.0, rmax=10.0, seed=0)
    cases.append(("128^3 sphere cell (48 spheres), the default first increment eps_zz += 5e-5",
                  (128, 128, 128), pm3, [MATRIX, STIFF], [[0, 0, INC, 0, 0, 0]], FREE, dict(max_nr=400)))
    out = []
    for name, dims, pm, phases, incs, free, opts in cases:
        res = {}
        for mode in ("device", "host"):
            # a fresh context per mode: the trust radius carries over between load steps
            with torch.cuda.stream(st):
                s = RVESolver(dims, pm, phases, precision=32, stream=st, eta_eq=1e-6, eta_cg=1e-2, **opts)
                eps0 = s.field(0.0)
            binding.rve_set_device_loop(s.h, mode == "device")

            def path():
                s.set_state(eps0)
                return [s.solve_step(dE, free_mask=free, raise_on_error=False) for dE in incs]

            for _ in range(args.warmup):
                path()
            torch.cuda.synchronize()
            y0 = s.sync_count
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(st)
            reps = [path() for _ in range(args.steps)]
            ev1.record(st)
            torch.cuda.synchronize()
            cg = sum(r["cg_iters"] for rr in reps for r in rr)
            res[mode] = {"ms_per_path": ev0.elapsed_time(ev1) / args.steps,
                         "host_waits_per_path": (s.sync_count - y0) / args.steps, "cg_iters_per_path": cg / args.steps}
            s.close()
        d, h = res["device"], res["host"]
        out.append({"case": name, "device_loop": d, "host_stepped": h,
                    "host_overhead_us_per_cg_iteration": 1e3 * (h["ms_per_path"] - d["ms_per_path"])
                    / max(d["cg_iters_per_path"], 1)})
    line = {"metric": "load-path time with device-side vs host-stepped Steihaug-CG control",
            "value": out[0]["device_loop"]["ms_per_path"], "unit": "ms per load path (32^2 case)", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "control", "cases": out}}
    print(json.dumps(line), flush=True)
    return 0


ONSET_WORKLOAD = ("random-sphere cells (48 spheres at 128^3, 144 at 256^3, r~U[4,10], seed 0; the materials of the "
                  "load-step workload), uniaxial eps_zz (other components stress-free): after a first increment of 5e-5 "
                  "(damage starts), a step = the next increment of 5e-6 from that state (reset every step), "
                  "trust-region Newton + Steihaug CG to rel. residual 1e-6, with the secant Hessian and with the "
                  "symmetric consistent tangent")


def _onset_measure(n, steps, warmup, st, passes=0):
    """One load step at the damage onset of the n^3 sphere cell (48 spheres
    at 128^3, 144 at 256^3), timed with the secant and with the symmetric
    consistent Hessian from the same converged first increment."""
    import torch
    from paper_2207_10657_gb300 import RVESolver
    from synth import random_spheres
    dE1, dE2 = [0.0, 0.0, 5e-5, 0.0, 0.0, 0.0], [0.0, 0.0, 5e-6, 0.0, 0.0, 0.0]
    dims = (n, n, n)
    pm = random_spheres(dims, count=144 if n >= 256 else 48, rmin=4.0, rmax=10.0, seed=0)
    R0 = 10.0 * (n ** 3) ** 0.5 * 5e-5
    out, fields, launches = {}, {}, 0
    for name, h in (("secant", 0), ("consistent", 1)):
        with torch.cuda.stream(st):
            s = RVESolver(dims, pm, [MATRIX, STIFF], precision=32, stream=st, eta_eq=1e-6, eta_cg=1e-2,
                          max_nr=2000, R0=R0, Rmax=R0, hessian=h, passes=passes)
        first = s.solve_step(dE1, free_mask=FREE, raise_on_error=False)
        ref = s.get_state()
        eps0, kap0 = ref["eps"].clone(), ref["kappa"].clone()

        def step():
            s.set_state(eps0, kap0)
            return s.solve_step(dE2, free_mask=FREE, raise_on_error=False)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hv0, l0 = s.hv_count, s.launch_count
        ev0.record(st)
        reps = [step() for _ in range(steps)]
        ev1.record(st)
        torch.cuda.synchronize()
        launches += s.launch_count - l0
        fin = s.get_state()
        fields[name] = (fin["eps"].double().cpu(), fin["kappa"].double().cpu())
        out[name] = {"ms": ev0.elapsed_time(ev1) / steps, "hv": (s.hv_count - hv0) / steps,
                     "first_nr": first["nr_iters"], "first_converged": first["converged"],
                     "nr_iters": [r["nr_iters"] for r in reps], "converged": [r["converged"] for r in reps],
                     "rel_residual": [r["rel_residual"] for r in reps],
                     "mean_stress": reps[-1]["mean_stress"],
                     "damaged_voxels": int((fields[name][1] > 1e-4).sum().item())}
        s.close()
    c, sc = out["consistent"], out["secant"]
    ds = sum((a - b) ** 2 for a, b in zip(c["mean_stress"], sc["mean_stress"])) ** 0.5
    ns = sum(b ** 2 for b in sc["mean_stress"]) ** 0.5
    (ec, kc), (es, ks) = fields["consistent"], fields["secant"]
    dc, dsec = kc > 1e-4, ks > 1e-4
    near = (kc - 1e-4).abs() <= 1e-7
    return {"consistent": c, "secant": sc, "speedup_over_secant": sc["ms"] / c["ms"],
            "mean_stress_rel_diff": ds / ns if ns > 0 else None,
            "strain_field_rel_l2_diff": float((ec - es).norm() / es.norm()),
            "damaged_set_differences": int((dc != dsec).sum()),
            "damaged_set_differences_beyond_1e-3_of_kappa0": int(((dc != dsec) & ~near).sum()),
            "voxel_hv_per_s_consistent": c["hv"] * n ** 3 / (c["ms"] / 1e3)}, launches


def run_onset(args):
    """One load step at the damage onset with the secant and with the
    symmetric consistent Hessian (the converged state of a first increment
    is the reference state of every timed step), on the sphere cells of
    --onset-sizes (48 spheres at 128^3, 144 at 256^3, r ~ U[4, 10])."""
    import torch
    from paper_2207_10657_gb300 import build as _build
    _build.build()
    st = torch.cuda.Stream()
    sizes, launches = {}, 0
    for n in [int(x) for x in args.onset_sizes.split(",")]:
        sizes[str(n)], nl = _onset_measure(n, args.steps, args.warmup, st, args.passes)
        launches += nl
    first = sizes[sorted(sizes, key=int)[0]]
    line = {
        "metric": "load-step time at the damage onset: symmetric consistent vs secant Hessian",
        "value": first["consistent"]["ms"], "unit": "ms/load step (smallest size)", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": first["consistent"]["ms"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": ONSET_WORKLOAD, "sizes": sizes},
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    return 0


WS_WORKLOAD = ("learned warm start: 4-layer spectral neural operator (width 32, modes kx<16, |ky|,|kz|<=8, BF16 "
               "operands, FP32 accumulation) trained on plain-solver load steps of seeded 64^3 sphere cells (48 "
               "spheres, r~U[2,5]) under uniaxial eps_zz increments of 1e-5 (other components stress-free), then "
               "load steps of held-out cells (48 spheres, r~U[4,10] at 128^3, scaled with the grid) solved from the "
               "same converged states by the plain method, the learned start and the previous-increment start, "
               "each to rel. residual 1e-6")


HV_WORKLOAD = ("Hessian-vector products alone on the sphere cells of the load-step workload (48 spheres at "
               "128^3, 144 at 256^3 and 384^3, r ~ U[4, 10], seed 0), damage snapshot D ~ U[0, 0.9] on the matrix "
               "(seed 1), input v = G:(N(0,1) field, seed 2); 20 untimed products, then 200 timed one by one with "
               "CUDA events on the solver's stream")


def run_hv(args):
    import numpy as np
    import torch
    from paper_2207_10657_gb300 import RVESolver, build as _build
    from synth import damage_snapshot, random_field, random_spheres
    _build.build()
    peak, peak_kind = _peaks()
    for n in (int(x) for x in args.hv_sizes.split(",")):
        dims = (n, n, n)
        nvox = n ** 3
        pm = random_spheres(dims, count=48 if n <= 128 else 144, rmin=4.0, rmax=10.0, seed=0)
        D = damage_snapshot(pm, dmax=0.9, seed=1)
        for prec in (int(x) for x in args.hv_precisions.split(",")):
            dt = torch.float32 if prec == 32 else torch.float64
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                s = RVESolver(dims, pm, [MATRIX, STIFF], precision=prec, stream=st)
                s.set_damage(torch.from_numpy(D).to(device="cuda", dtype=dt))
                v = s.project(torch.from_numpy(random_field(6, dims, seed=2)).to(device="cuda", dtype=dt))
                out = s.field()
            for _ in range(20):
                s.hessp(v, out)
            st.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(200)]
            for e0, e1 in ev:
                e0.record(st)
                s.hessp(v, out)
                e1.record(st)
            st.synchronize()
            ms = np.array([e0.elapsed_time(e1) for e0, e1 in ev])
            es = prec // 8  # bytes per real
            spec = 6 * n * n * (n // 2 + 1) * 2 * es
            field = 6 * nvox * es
            # plain product: x-forward (v, phase, damage -> spectrum), three spectral passes, x-inverse
            byts = (field + nvox * (1 + es) + spec) + 3 * 2 * spec + (spec + field)
            med = float(np.median(ms))
            print(json.dumps({
                "metric": "voxel-Hv/s (Hessian-vector product alone)", "value": nvox / (med / 1e3), "unit": UNIT,
                "grid": [n, n, n], "dtype": f"f{prec}", "ms_median": med, "ms_p10": float(np.percentile(ms, 10)),
                "ms_p90": float(np.percentile(ms, 90)), "products": len(ms),
                "roofline": {"bound": "hbm", "achieved": byts / (med / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                             "frac": byts / (med / 1e3) / 1e9 / peak, "algorithmic_bytes": byts,
                             "peak_source": peak_kind},
                "config": {"workload": HV_WORKLOAD}}), flush=True)
            s.close()
            del v, out
            torch.cuda.empty_cache()
    return 0


def run_warmstart(args):
    import numpy as np
    import torch
    from paper_2207_10657_gb300 import build as _build
    from paper_2207_10657_gb300.learned import SpectralOperator, compare_warm_start, generate_samples, train
    from synth import random_spheres
    _build.build()
    phases = [MATRIX, STIFF]
    dE = [0.0, 0.0, 1e-5, 0.0, 0.0, 0.0]
    opts = dict(eta_eq=1e-6, eta_cg=1e-2, hessian=args.ws_hessian)

    def cell(n, seed):
        return random_spheres((n, n, n), count=48, rmin=4.0 * n / 128, rmax=10.0 * n / 128, seed=seed)

    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        net = SpectralOperator(layers=4, modes=16, seed=0, stream=st)
        t0 = time.perf_counter()
        Xs, Ts, log = generate_samples(net, [cell(64, 1000 + i) for i in range(2000)], phases, dE, FREE, 8,
                                       max_samples=2000, time_budget_s=args.ws_train_seconds, max_nr=100, **opts)
        t_gen = time.perf_counter() - t0
        t0 = time.perf_counter()
        hist = train(net, Xs, Ts, (64, 64, 64), args.ws_iters, batch=4, lr=2e-3, seed=0)
        st.synchronize()
        t_train = time.perf_counter() - t0
        zero = float(np.mean([float((T ** 2).mean()) for T in Ts]))
        l0 = net.launch_count
        recs = []
        for k, n in enumerate(int(x) for x in args.ws_eval.split(",")):
            for r in compare_warm_start(net, cell(n, 5000 + k), phases, dE, FREE, 6, max_nr=150, **opts):
                r["grid"] = n
                recs.append(r)
    ok = [r for r in recs if all(r[a]["converged"] for a in ("plain", "learned", "previous"))]
    if not ok:
        print(json.dumps({"metric": METRIC, "value": None, "error": "no evaluation step converged in every arm"}))
        return 1
    tot = {a: sum(r[a]["ms"] for r in ok) for a in ("plain", "learned", "previous")}
    hv = {a: sum(r[a]["hv"] for r in ok) for a in ("plain", "learned", "previous")}
    dsig = max(abs(r["learned"]["mean_stress"][2] - r["plain"]["mean_stress"][2]) / abs(r["plain"]["mean_stress"][2])
               for r in ok)
    line = {
        "metric": METRIC, "value": tot["learned"] / len(ok), "unit": "ms/load step (learned warm start)",
        "n_gpus": 1, "steps": len(ok), "warmup": 0, "ms_per_step": tot["learned"] / len(ok),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32 solver / bf16 network",
        "data": "synthetic",
        "config": {"workload": WS_WORKLOAD, "eval_grids": args.ws_eval,
                   "hessian": "symmetric consistent" if args.ws_hessian else "secant",
                   "train_samples": len(Xs), "train_generation_s": t_gen, "train_iters": args.ws_iters,
                   "train_s": t_train, "train_ms_per_iter": t_train / args.ws_iters * 1e3,
                   "loss_zero_prediction": zero, "loss_last_100": float(np.mean(hist[-100:])),
                   "plain_ms_per_step": tot["plain"] / len(ok), "previous_ms_per_step": tot["previous"] / len(ok),
                   "speedup_learned_vs_plain": tot["plain"] / tot["learned"],
                   "hv_total": hv, "max_rel_stress_diff_learned_vs_plain": dsig,
                   "steps": [{"grid": r["grid"], "step": r["step"],
                              **{a: {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r[a].items()
                                     if k != "mean_stress"} for a in ("plain", "learned", "previous")}}
                             for r in recs]},
        "network_gpu_launches_in_eval": net.launch_count - l0,
    }
    print(json.dumps(line), flush=True)
    net.close()
    return 0


def np_prod(d):
    out = 1
    for x in d:
        out *= int(x)
    return out


def run_probe(args):
    """Small untimed cases whose kernels an ncu capture can take in full."""
    import numpy as np
    import torch
    from paper_2207_10657_gb300 import build as _build
    _build.build()
    if args.probe == "step":
        from paper_2207_10657_gb300 import RVESolver, binding
        from synth import random_spheres
        dims = tuple(int(x) for x in args.probe_dims.split(","))
        pm = random_spheres(dims, count=100, rmin=4, rmax=10, seed=0)
        s = RVESolver(dims, pm, [MATRIX, STIFF], precision=32, eta_eq=1e-6, eta_cg=1e-2, max_nr=50,
                      passes=args.passes)
        # the CG iterations stepped from the host: the same kernels, each a
        # separate launch a profiler can take (the device loop's are graph nodes)
        binding.rve_set_device_loop(s.h, False)
        r = s.solve_step([0, 0, INC, 0, 0, 0], free_mask=FREE, raise_on_error=False)
        torch.cuda.synchronize()
        print("probe step", r["converged"], r["hv_products"], s.launch_count)
        s.close()
    else:
        from paper_2207_10657_gb300.learned import SpectralOperator
        net = SpectralOperator(layers=4, modes=16, seed=0)
        rng = np.random.default_rng(0)
        X = torch.from_numpy(rng.standard_normal((4, 64, 64, 64, 16)).astype(np.float32)).cuda()
        T = torch.from_numpy(rng.standard_normal((4, 64, 64, 64, 6)).astype(np.float32)).cuda()
        for _ in range(3):
            net.loss_grad(X, T, (64, 64, 64))
            net.adam_step(1e-3)
        torch.cuda.synchronize()
        print("probe fno", net.launch_count)
        net.close()
    return 0


def main():
    args = _args()
    if args.probe:
        return run_probe(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch96":
        return run_batch(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "hv":
        return run_hv(args)
    if args.workload == "lbfgs":
        return run_lbfgs(args)
    if args.workload == "control":
        return run_control(args)
    if args.workload == "onset":
        return run_onset(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
